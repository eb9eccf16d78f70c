"""The learned initial guess inside the pressure solve: harvested pairs are
exact, the solve with the guess still meets the tolerance, and a briefly
trained network reduces the SRJ work on a channel it was not trained on."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GRID = (32, 16, 32)


def _cfg():
    from paper_1511_07800_gb300 import learn
    return learn.workload("os_instability", grid=GRID)


def test_harvested_pairs_satisfy_the_poisson_equation(stp_lib):
    """r = b - L p_prev and dp = p - p_prev, so r - L dp = b - L p, which the
    solve drove below 1e-8 ||b||; FP32 storage of r and dp adds ~1e-7."""
    torch = pytest.importorskip("torch")
    from paper_1511_07800_gb300 import learn
    cfg = _cfg()
    R, DP = learn.harvest(cfg, seeds=[5], steps_per_seed=4, precision="fp64")
    for i in range(4):
        r = R[i].double().contiguous()
        dp = DP[i].double().contiguous()
        res = torch.zeros_like(r)
        n = stp_lib.poisson_residual_noalloc(cfg, dp, r, res)
        assert n <= 1e-6 * float(r.norm()), (i, n, float(r.norm()))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_learned_guess_solves_to_tolerance(stp_lib, orc, precision):
    """With an untrained (random) network as the guess, every solve still
    converges to ptol, and the step agrees with the plain step to that level."""
    torch = pytest.importorskip("torch")
    from oracle import unet
    from paper_1511_07800_gb300 import learn
    cfg = _cfg()
    net = stp_lib.UNet(1, *GRID)
    net.set_params(unet.init_params(11).astype(np.float32))
    fields = {}
    for mode in ("plain", "learned"):
        with stp_lib.Channel(cfg, precision=precision) as ch:
            ch.set_fields(*learn.varied_fields(cfg, 3))
            ch.step(2)
            if mode == "learned":
                ch.set_learned_guess(net)
            for _ in range(3):
                st = ch.step(1)
                assert st["converged"] and st["rel_res"] <= cfg["ptol"]
            if mode == "learned":
                ch.set_learned_guess(None)
            fields[mode] = ch.get_fields()
    for k in ("u", "v", "w"):
        a, b = fields["plain"][k], fields["learned"][k]
        assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max(), k
    net.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_learned_preconditioner_solves_to_tolerance(stp_lib, orc, precision):
    """The network as a preconditioner (stp_set_learned_mode 1: applied to
    the residual at every refinement pass in FP32, before every SRJ cycle in
    FP64), untrained: every solve still converges to ptol, the step agrees
    with the plain step to that level, and the host-driven solve takes the
    same path as the graph."""
    torch = pytest.importorskip("torch")
    from oracle import unet
    from paper_1511_07800_gb300 import learn
    cfg = _cfg()
    net = stp_lib.UNet(1, *GRID)
    net.set_params(unet.init_params(12).astype(np.float32))
    fields, sweeps = {}, {}
    for mode in ("plain", "precond", "precond_host"):
        import os
        if mode == "precond_host":
            os.environ["STP_HOST_SOLVE"] = "1"
        try:
            with stp_lib.Channel(cfg, precision=precision) as ch:
                ch.set_fields(*learn.varied_fields(cfg, 4))
                ch.step(2)
                if mode != "plain":
                    ch.set_learned_guess(net)
                    ch.set_learned_mode(1)
                sw = 0
                for _ in range(3):
                    st = ch.step(1)
                    assert st["converged"] and st["rel_res"] <= cfg["ptol"], mode
                    sw += st["sweeps"]
                fields[mode], sweeps[mode] = ch.get_fields(), sw
        finally:
            os.environ.pop("STP_HOST_SOLVE", None)
    for k in ("u", "v", "w"):
        a, b = fields["plain"][k], fields["precond"][k]
        assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max(), k
        assert np.array_equal(fields["precond"][k], fields["precond_host"][k]), k
    assert sweeps["precond"] == sweeps["precond_host"]
    net.close()


def test_trained_guess_cuts_the_fp64_solve_time(stp_lib, orc):
    """What the trained network gains.  Trained on 600 pairs harvested from
    ten instability channels at 128 x 64 x 128 (the workload's grid), then
    used as the initial guess of every FP64 pressure solve of an unseen
    channel: the solves to 1e-8 take at least 15 % fewer SRJ sweeps and at
    least 1.1 times less GPU time than the plain solves from the previous
    pressure, the network's forward included (measured: 1216 against 1600
    sweeps, 1.25x).  In FP64 a guess that removes most of the error saves
    whole SRJ cycles; in FP32 with refinement a pass gains about 1e-3 from
    any start, so the guess saves no pass (not asserted; printed)."""
    torch = pytest.importorskip("torch")
    from paper_1511_07800_gb300 import learn
    grid = (128, 64, 128)
    cfg = learn.workload("os_instability", grid=grid)
    R, DP = learn.harvest(cfg, seeds=range(10), steps_per_seed=60)
    K = learn.output_scale(R, DP, 4, grid)
    net = stp_lib.UNet(4, *grid)
    net.set_params(learn.he_init(0))
    net.set_output_scale(K)
    learn.train(net, R, DP, 1500, 4, 1e-3)
    learn.train(net, R, DP, 500, 4, 3e-4)
    one = stp_lib.UNet(1, *grid)
    one.set_params(net.get_params())
    one.set_output_scale(K)
    net.close()
    del R, DP
    res = learn.compare_modes(cfg, one, seed=50, nsteps=8, precision="fp64")
    print("learned vs plain (FP64):", res)
    assert res["guess"]["converged"] and res["plain"]["converged"]
    assert res["guess"]["sweeps"] <= 0.85 * res["plain"]["sweeps"], res
    assert res["guess"]["speedup"] >= 1.1, res
    res32 = learn.compare_modes(cfg, one, seed=50, nsteps=4, precision="fp32")
    print("learned vs plain (FP32 + refinement):", res32)
    one.close()
