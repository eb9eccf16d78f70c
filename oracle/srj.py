"""SRJ relaxation schedule -- TEST INFRASTRUCTURE ONLY (part of the oracle).

Sec. 3.4 of the paper: each sweep of a cycle of M Jacobi-SOR sweeps uses its
own relaxation factor omega_k, and the cycle repeats until convergence.  The
paper takes the factors from an external script that is not available, so
the schedule here is built from the mathematics of the method:

* Error components of the Jacobi-preconditioned operator D^-1(-L) with
  eigenvalue mu are multiplied by (1 - omega mu) per sweep, so a cycle
  multiplies them by G(mu) = prod_k (1 - omega_k mu).
* The M factors that minimise max |G| over [mu_min, mu_max] are the
  reciprocals of the Chebyshev points of that interval (the many-level limit
  of SRJ); then G(mu) = T_M((mu_max+mu_min-2mu)/(mu_max-mu_min)) /
  T_M((mu_max+mu_min)/(mu_max-mu_min)).
* The order within the cycle pairs each factor with its mirror root
  (recursive doubling, M a power of two) so that no partial product grows
  far beyond the largest single factor.

mu_min and mu_max come from the separable structure of the discrete Poisson
operator: Fourier modes in the periodic x and y directions, and for each
(x, y) wavenumber a small generalized symmetric eigenproblem in z solved with
scipy.  For z-line Jacobi (each z column solved exactly, Sec. 3.4's
relaxation applied to whole lines) the operator splits the same way.
"""
import numpy as np
import scipy.linalg


def z_grid(nz, Lz, stretch):
    """Face heights (tanh clustering toward both walls when stretch > 0)."""
    s = np.arange(nz + 1) / nz
    if stretch > 0:
        zf = 0.5 * Lz * (1.0 + np.tanh(stretch * (2 * s - 1)) / np.tanh(stretch))
    else:
        zf = Lz * s
    zf[0], zf[-1] = 0.0, Lz
    return zf


def _z_operator(nz, Lz, stretch):
    zf = z_grid(nz, Lz, stretch)
    dz = np.diff(zf)
    zc = 0.5 * (zf[1:] + zf[:-1])
    hz = np.diff(zc)                                  # between centres k-1, k (k=1..nz-1)
    cup = np.zeros(nz)
    cdn = np.zeros(nz)
    cup[:-1] = 1.0 / (hz * dz[:-1])
    cdn[1:] = 1.0 / (hz * dz[1:])
    # -L_z, made symmetric by the cell widths: W(-L_z)
    A = np.diag(dz * (cup + cdn))
    off = -1.0 / hz
    A += np.diag(off, 1) + np.diag(off, -1)
    return dz, cup, cdn, A


def jacobi_bounds(nx, ny, nz, Lx, Ly, Lz, stretch=0.0):
    """(mu_min, mu_max): smallest non-zero and largest eigenvalue of D^-1(-L)."""
    dx, dy = Lx / nx, Ly / ny
    dz, cup, cdn, A0 = _z_operator(nz, Lz, stretch)
    S = 2 / dx**2 + 2 / dy**2 + cup + cdn
    B = np.diag(dz * S)

    def ev(a):
        return scipy.linalg.eigh(A0 + a * np.diag(dz), B, eigvals_only=True)

    lx = lambda m: 4 / dx**2 * np.sin(np.pi * m / nx) ** 2
    ly = lambda n: 4 / dy**2 * np.sin(np.pi * n / ny) ** 2
    cands = [ev(0.0)[1]]
    if nx > 1:
        cands.append(ev(lx(1))[0])
    if ny > 1:
        cands.append(ev(ly(1))[0])
    mu_min = min(cands)
    mu_max = ev(lx(nx // 2) + ly(ny // 2))[-1]
    return float(mu_min), float(mu_max)


def line_bounds(nx, ny, nz, Lx, Ly, Lz, stretch=0.0):
    """(mu_min, mu_max) for z-line Jacobi: the smallest non-zero and the
    largest eigenvalue of A^-1(-L), A = -L_z + (2/dx^2 + 2/dy^2) I the
    operator of one z column with its x-y diagonal.  -L is the Kronecker sum
    of -L_z (eigenvalues tau, from the symmetric generalized problem
    W(-L_z) phi = tau W phi, W = diag(dz)) and the periodic x-y operator
    (eigenvalues lam = 4/dx^2 sin^2(pi m/nx) + 4/dy^2 sin^2(pi n/ny)); A
    shares the eigenvectors, so every eigenvalue is (tau + lam)/(tau + dxy).
    All (tau, lam) pairs but the constant mode are enumerated."""
    dx, dy = Lx / nx, Ly / ny
    dz, cup, cdn, A0 = _z_operator(nz, Lz, stretch)
    tau = scipy.linalg.eigh(A0, np.diag(dz), eigvals_only=True)
    dxy = 2 / dx**2 + 2 / dy**2
    lam = (4 / dx**2 * np.sin(np.pi * np.arange(nx) / nx) ** 2)[:, None] + \
        (4 / dy**2 * np.sin(np.pi * np.arange(ny) / ny) ** 2)[None, :]
    lam = lam.ravel()
    mu = (tau[:, None] + lam[None, :]) / (tau[:, None] + dxy)
    mu[0, 0] = np.inf          # the constant mode (tau_0 = 0, lam = 0) is the null space
    mu_min = mu.min()
    mu[0, 0] = -np.inf
    return float(mu_min), float(mu.max())


def stable_order(M):
    """Odd numbers 1..2M-1 in the recursive mirror-pair order (M = 2^p)."""
    assert M >= 1 and (M & (M - 1)) == 0, "cycle length must be a power of two"
    th, m = [1], 1
    while m < M:
        th = [x for t in th for x in (t, 4 * m - t)]
        m *= 2
    return th


def chebyshev_schedule(mu_min, mu_max, M):
    """omega_1..omega_M: reciprocals of the Chebyshev points of [mu_min, mu_max]."""
    mid, half = 0.5 * (mu_max + mu_min), 0.5 * (mu_max - mu_min)
    return np.array([1.0 / (mid + half * np.cos(t * np.pi / (2 * M))) for t in stable_order(M)])


def cycle_factor(mu_min, mu_max, M):
    """max |G| over [mu_min, mu_max] for the Chebyshev cycle: 1/T_M(x0)."""
    x0 = (mu_max + mu_min) / (mu_max - mu_min)
    return 1.0 / np.cosh(M * np.arccosh(x0))


def default_cycle_length(mu_min, mu_max, target=0.01, mmax=1024):
    """Smallest power of two whose cycle reduces every error mode by `target`."""
    M = 2
    while M < mmax and cycle_factor(mu_min, mu_max, M) > target:
        M *= 2
    return M


def schedule_for(nx, ny, nz, Lx, Ly, Lz, stretch=0.0, M=0, line=False):
    """(omega, mu_min, mu_max) for point (default) or z-line Jacobi sweeps."""
    mn, mx = (line_bounds if line else jacobi_bounds)(nx, ny, nz, Lx, Ly, Lz, stretch)
    if M <= 0:
        M = default_cycle_length(mn, mx)
    return chebyshev_schedule(mn, mx, M), mn, mx
