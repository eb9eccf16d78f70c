/*
 * stp.h -- C ABI of the GB300 projection step for incompressible channel flow.
 *
 * One handle holds one channel on one GPU: a 3-D MAC grid, periodic in x and
 * y, with no-slip walls at z = 0 and z = Lz (arXiv 1511.07800, Sec. 2.1 and
 * Fig. "computational domain").  A time step is the projection method of
 * Sec. 3.1:
 *   nu_T     Smagorinsky eddy viscosity with van Driest damping (Sec. 2.2)
 *   N^n      -u.grad u + d_j(nu_T d_i u_j) + f   (Eq. more_conv; AB3)
 *   u*       Crank-Nicolson on d_j(nu_T d_j u_i) (Eq. more_diff)
 *   b        div u* / dt                          (Eq. presdiv)
 *   p        L p = b by Scheduled Relaxation Jacobi (Sec. 3.4)
 *   u^{n+1}  u* - dt grad p                       (Eq. project u_p_1)
 *
 * Layouts (all arrays x fastest, C order, double on the ABI):
 *   u, v, p, nu_t : [nz][ny][nx]   u(i) at x = i dx, v(j) at y = j dy,
 *                                  p, nu_t at cell centres
 *   w             : [nz+1][ny][nx] w(k) at z = zf[k]; the planes k = 0 and
 *                                  k = nz are the walls and must be zero
 *
 * Pointers: `where` = STP_HOST for host memory, STP_DEVICE for memory on the
 * handle's device.  The library never keeps a caller pointer after a call
 * returns; it owns all its device memory and frees it in stp_destroy.
 *
 * The pressure solve runs as one CUDA graph steered from the device (graph
 * conditional nodes), one kernel per SRJ sweep.  With STP_PERSISTENT=1 at
 * stp_init an FP32 cycle instead runs as one persistent cooperative kernel
 * with bounded grid barriers between its sweeps (slower on GB300: kept as an
 * option); each barrier wait gives up after STP_BARRIER_WAIT SM clock cycles
 * (read at every stp_step / stp_poisson_solve call; default 2e9, about one
 * second), and the call then returns STP_ETIMEOUT.  With
 * STP_LINE_PERSISTENT=1 at stp_init an FP32 z-line cycle runs as one
 * cooperative launch in which every 32 x 4-column tile waits only for its
 * four x-y neighbour tiles to finish the previous sweep (bitwise the same
 * results as the shared-memory lock-step kernel below; the same bounded
 * waits; STP_WAIT_SKEW=<n> makes every tile wait for a sweep count no
 * neighbour reaches, so that tests can make those waits run out).  An FP32
 * z-line sweep on rows of a multiple of 32 cells and columns of 2 to 192
 * levels solves each column in registers, level chunk by level chunk
 * (Sec. 3.4's line relaxation with the twisted elimination split into
 * chunked recurrences); elsewhere, or with STP_LINE_VARIANT=0 at stp_init,
 * a block stages its columns in shared memory and solves them in lock
 * step.  The two round differently (a few units in the last place).  The FP32 sweep kernel's tile shape (z levels per thread, rows
 * per block) is picked on first use by timing the variants on the grid
 * (STP_SWEEP_VARIANT=<0..11> forces one; variants 6..8 pack warps along the
 * plane for rows shorter than 128 cells, 9..11 run two sweeps per launch on
 * a shared-memory tile; STP_TUNE_LOG=1 prints the timings to stderr).  With STP_HOST_SOLVE=1 at
 * stp_init the same kernels are driven from the host instead, one host
 * round trip per SRJ cycle (for profilers that cannot see kernels inside
 * conditional graphs).
 *
 * Errors: every int-returning call returns STP_OK (0) or a negative STP_E*
 * code; stp_last_error gives a one-line message.  No call aborts the process.
 * Calls on one handle must not overlap (one handle per host thread).
 */
#ifndef STP_H
#define STP_H

#ifdef __cplusplus
extern "C" {
#endif

#define STP_OK 0
#define STP_EINVAL (-1)        /* bad argument, size or configuration           */
#define STP_ENOMEM (-2)        /* device or host allocation failed              */
#define STP_ECUDA (-3)         /* a CUDA runtime call failed                    */
#define STP_ENOTCONVERGED (-4) /* pressure solve hit its sweep cap              */
#define STP_EDIVERGED (-5)     /* NaN/Inf in a residual or the velocity         */
#define STP_ECFL (-6)          /* U_max dt > 0.1 dx (Eq. cfl_cond), if checked   */
#define STP_ETIMEOUT (-7)      /* a bounded device-side wait ran out              */

#define STP_HOST 0
#define STP_DEVICE 1

#define STP_FP64 0        /* every field and sweep in FP64                       */
#define STP_FP32_REFINE 1 /* FP32 fields and sweeps; FP64 pressure, norms and an
                             FP64 iterative-refinement loop around FP32 SRJ       */

typedef struct stp_config {
    int nx, ny, nz;          /* cells; nx, ny >= 3, nz >= 2                      */
    double Lx, Ly, Lz;       /* box; z in [0, Lz]                                */
    double nu;               /* molecular viscosity 1/Re                         */
    double dt;               /* time step                                        */
    int forcing;             /* 0: constant body force fx (= -dp/dx) on u;
                                1: constant bulk velocity ubulk (flux fix-up)     */
    double fx;
    double ubulk;
    int les;                 /* 1: nu_T = nu + (cs Delta phi_w)^2 |S|            */
    double cs;               /* Smagorinsky constant (0.1)                       */
    double vd_a;             /* van Driest constant A (25)                       */
    double re_tau;           /* friction Reynolds number used in d+ = d Re_tau/(Lz/2) */
    double stretch;          /* 0: uniform z; gamma > 0: zf = Lz/2 (1 + tanh(gamma(2k/nz-1))/tanh gamma) */
    int precision;           /* STP_FP64 or STP_FP32_REFINE                     */
    double ptol;             /* pressure: stop when ||b - Lp||_2 <= ptol ||b||_2 */
    int pmaxit;              /* cap on SRJ sweeps per solve                      */
    int cn_sweeps;           /* Jacobi sweeps of the CN system; 0: automatic
                                (the count whose contraction bound reaches the
                                storage precision: 1e-12 in FP64, 2^-24 in FP32) */
    int srj_m;               /* SRJ cycle length; 0: automatic (power of two)    */
    const double *srj_omega; /* optional schedule omega_1..omega_M (M = srj_m);
                                NULL: Chebyshev schedule built by the library     */
    double inner_tol;        /* FP32 inner solve: relative reduction per
                                refinement pass (default 1e-3)                    */
    int cfl_check;           /* 1: return STP_ECFL when U_max dt > 0.1 dx         */
    int device;              /* CUDA device ordinal                              */
    void *stream;            /* cudaStream_t to run on; NULL: the library's own  */
    int zline;               /* pressure sweeps: 0 point Jacobi-SOR (Sec. 3.4);
                                1 z-line Jacobi-SOR: each z column solved exactly
                                (Thomas) with the x-y neighbours held, SRJ
                                weights from the line-Jacobi spectrum (suits
                                wall-stretched grids)                            */
    int cn_zline;            /* Crank-Nicolson system: 0 point Jacobi sweeps;
                                1 z-line Jacobi: each z column solved exactly
                                (Thomas) with the x-y neighbours of the previous
                                iterate (Sec. 3.1 names no solver; the wall-
                                normal couplings of a stretched grid then cost
                                no sweeps: automatic count from the x-y
                                couplings alone); needs ny <= 65535 (else
                                stp_init returns STP_EINVAL)                      */
} stp_config;

typedef struct stp_step_stats {
    int poisson_sweeps;      /* SRJ sweeps of the last step (inner sweeps in FP32) */
    int refine_passes;       /* FP64 refinement passes of the last step         */
    int converged;           /* 1 if every pressure solve met ptol               */
    double rel_residual;     /* ||b - Lp|| / ||b|| at the end of the last solve  */
    double ubulk;            /* volume mean of u after the last step             */
    double umax;             /* max |u| after the last step                      */
    double dpdx;             /* implied -dp/dx of the flux fix-up (forcing 1)    */
    long long step;          /* steps taken since stp_set_fields                 */
    long long launches;      /* kernels run by this stp_step call (host launches
                                plus the kernels of the solve graphs)             */
    long long solve_sweeps;  /* SRJ sweeps of all solves of this call           */
    double solve_ms;         /* GPU time of those solves (CUDA events on the
                                handle's stream around each solve graph; includes
                                the once-per-cycle residual checks and, in FP32
                                mode, the refinement kernels)                     */
} stp_step_stats;

typedef struct stp_solve_stats {
    int sweeps;              /* SRJ sweeps (inner sweeps in FP32)               */
    int refine_passes;       /* FP64 refinement passes                          */
    int converged;           /* 1 if ||rhs - Lp|| <= tol ||rhs||                */
    double rel_residual;     /* ||rhs - Lp|| / ||rhs|| at the end               */
    double solve_ms;         /* GPU time of the solve (CUDA events on the
                                handle's stream around the solve graph)          */
} stp_solve_stats;

typedef struct stp_handle stp_handle;

/* Fill `cfg` with defaults: 32^3 unit-Re channel, FP64, ptol 1e-8,
   automatic CN sweeps and SRJ schedule, Cs 0.1, A 25, Re_tau 180. */
void stp_config_defaults(stp_config *cfg);

/* Create a handle: validates cfg (STP_EINVAL), selects cfg->device, allocates
   every device buffer (STP_ENOMEM), builds the SRJ schedule.  Fields start at
   zero.  On failure *out is NULL and stp_last_error(NULL) explains. */
int stp_init(const stp_config *cfg, stp_handle **out);

/* Free the handle and its device memory (NULL is a no-op). */
void stp_destroy(stp_handle *h);

/* Message of the last failed call on h (h NULL: last stp_init failure of the
   calling thread).  Valid until the next call on h. */
const char *stp_last_error(const stp_handle *h);

/* Copy initial fields in (Sec. 2.1 layout above).  p may be NULL (zero).
   Resets the Adams-Bashforth history (the next step is forward Euler, the
   one after AB2) and the step counter.  STP_EINVAL if a wall plane of w is
   non-zero. */
int stp_set_fields(stp_handle *h, const double *u, const double *v, const double *w, const double *p,
                   int where);

/* Copy the current fields out.  Any pointer may be NULL.  nu_t receives the
   total viscosity nu_T of the last step (nu without LES). */
int stp_get_fields(stp_handle *h, double *u, double *v, double *w, double *p, double *nu_t, int where);

/* Advance nsteps projection steps (Sec. 3.1), each with its pressure solved
   to ptol from the previous pressure.  Blocks until done.  Returns
   STP_ENOTCONVERGED if a solve hit pmaxit (the step still completes),
   STP_EDIVERGED on NaN/Inf in a residual or the velocity, STP_ETIMEOUT when
   a bounded device-side wait ran out, STP_ECFL when cfl_check is set and
   violated.  On STP_EDIVERGED and STP_ETIMEOUT the step that failed is
   undone: the fields, the Adams-Bashforth history and the step counter are
   those of the last good step (each step first copies u, v, w, p on the
   device).  stats (nullable) describes the last step. */
int stp_step(stp_handle *h, int nsteps, stp_step_stats *stats);

/* ------------------------------------------------------------------------
 * Batched channels: many independent channels (each its own stp_handle,
 * of any size and configuration, all on one device) advanced together by
 * one CUDA graph launch.  The graph holds a device-side WHILE loop over the
 * steps; its body has one branch per channel (velocity kernels, the
 * channel's own device-steered pressure solve, the correction), so the
 * channels run concurrently and the host neither launches nor waits
 * between steps.  Every pressure solve still meets its channel's ptol.
 * ------------------------------------------------------------------------ */
typedef struct stp_batch stp_batch;

typedef struct stp_batch_stats {
    long long steps;         /* steps taken by every channel in this call      */
    long long cells;         /* total cells over the channels                  */
    long long sweeps;        /* SRJ sweeps over all channels and steps         */
    int converged;           /* 1 if every solve of every channel met its ptol  */
    double gpu_ms;           /* GPU time of the launch (CUDA events)           */
    long long kernels;       /* kernels the launch ran                         */
} stp_batch_stats;

/* The handles stay owned by the caller and must outlive the batch; they
   must not be stepped on their own while the batch runs.  stream NULL: the
   batch's own stream. */
int stp_batch_create(stp_handle *const *handles, int n, void *stream, stp_batch **out);
void stp_batch_destroy(stp_batch *b);
const char *stp_batch_last_error(const stp_batch *b);

/* LES statistics (Sec. 6).  The velocities are taken at the cell centres
   (uc, vc, wc: the mean of the two faces of each component) and averaged
   over x, y and the accumulated samples.
   stp_stats_reset: clear the sums (the first call allocates two small
   buffers); kc is the level of the two-point correlations, -1 for nz/2.
   stp_stats_accumulate: add the current fields, asynchronously on the
   handle's stream (call it between steps).
   stp_stats_read (synchronises): moments [9][nz] = per level the means of
   uc, vc, wc, uc^2, vc^2, wc^2, uc vc, uc wc, vc wc; corr [3][nx] = the
   streamwise correlations R(d) = <q(x + d dx) q(x)> - <q>^2 of u, v (on their
   faces) and wc at level kc; either may be NULL.  FP64 sums in a fixed
   order. */
int stp_stats_reset(stp_handle *h, int kc);
int stp_stats_accumulate(stp_handle *h);
int stp_stats_read(stp_handle *h, double *moments, double *corr, long long *nsamples, int *kc);

/* The FP32 sweep tile variant the autotuner picked for this handle's grid
   (0..8, see above; -1 before the first solve, 0 in FP64) and, when it was
   timed, its time per sweep in microseconds (*us may be NULL). */
int stp_sweep_tile(const stp_handle *h, float *us);

/* The z-line sweep kernel of a handle with line relaxation (Sec. 3.4):
   1 for the register-chunked FP32 kernel (rows of a multiple of 32 cells,
   columns of 2 to 192 levels), 0 for the shared-memory lock-step kernel
   (FP64, other grids, or STP_LINE_VARIANT=0 at stp_init); -1 for point
   sweeps or a NULL handle.  No GPU work. */
int stp_line_kernel(const stp_handle *h);

/* Lock-step groups of the batch (built at the first stp_batch_step).
   Channels of at most 2^17 cells in FP32 with refinement that share the SRJ
   cycle length M (at least two of them, rows a multiple of 4 cells, no
   learned guess) are solved together: every kernel of their pressure solve covers all of them
   in one launch, each channel keeping its own schedule, residuals and
   stopping decisions, so its results are bitwise those of its own solve.
   Environment, read when the graph is built: STP_BATCH_GROUPS=0 keeps every
   channel on its own solve; STP_BATCH_GROUP_MAX_CHANNEL=<n> sets the channel
   size limit (-1: none); groups are split into parts whose inner
   working set (12 bytes a cell) fills at most half the L2, or at most n
   cells with STP_BATCH_GROUP_CELLS=<n> (0: no split);
   STP_BATCH_GROUP_CHAIN=1 runs the groups' solves one after another
   instead of side by side. */
typedef struct stp_batch_group {
    int channels, M;
    int variant;        /* FP32 sweep tile variant picked by timing the group   */
    long long cells;
    float sweep_us;     /* measured grouped sweep, every channel active (0: not timed) */
} stp_batch_group;

/* Number of groups; fills out[0 .. min(n, max_groups)) when out is not NULL. */
int stp_batch_groups(const stp_batch *b, int max_groups, stp_batch_group *out);

/* Advance every channel nsteps steps in one graph launch; per_channel
   (nullable, n entries) receives each channel's stats of its last step. */
int stp_batch_step(stp_batch *b, int nsteps, stp_batch_stats *stats, stp_step_stats *per_channel);

/* Checkpoint: the whole state of the time stepper (velocities, pressure,
   the two Adams-Bashforth history levels, the history depth and the step
   counter) as one opaque host buffer of stp_state_size() doubles, its
   fields kept in the handle's precision (an FP32 handle packs its FP32
   arrays two values to a double; the pressure is FP64 in both);
   stp_set_state resumes bitwise where stp_get_state was taken (same
   configuration and precision; another grid or precision: STP_EINVAL). */
long long stp_state_size(const stp_handle *h);
int stp_get_state(stp_handle *h, double *buf);
int stp_set_state(stp_handle *h, const double *buf);

/* Solve L p = rhs (Sec. 3.4 SRJ; Eq. presdiv operator with Neumann walls)
   to ||rhs - Lp||_2 <= tol ||rhs||_2 starting from p_inout, capped at maxit
   sweeps (0: pmaxit).  L is singular (its null space is the constants), so
   rhs [nz][ny][nx] must have zero volume-weighted mean: the call returns
   STP_EINVAL, before any sweep, when |sum rhs dV| > 1e-9 sum |rhs| dV.
   p_inout receives the solution with its volume-weighted mean set to zero.
   Uses the handle's buffers: the current pressure field is overwritten. */
int stp_poisson_solve(stp_handle *h, const double *rhs, double *p_inout, double tol, int maxit, int where,
                      stp_solve_stats *stats);

/* Terms of the step evaluated on the current fields, for checks:
     STP_TERM_VISCOSITY  a = nu_T                         (Sec. 2.2)
     STP_TERM_EXPLICIT   a,b,c = N = -u.grad u + d_j(nu_T d_i u_j) + f
     STP_TERM_DIFFUSION  a,b,c = d_j(nu_T d_j u_i)        (nu_T from the
                         current fields)
     STP_TERM_DIVERGENCE a = D u                          (Eq. presdiv)
     STP_TERM_LAPLACIAN  a = L p                          (L = D G)
   b, c are w-shaped ([nz+1]) where the term is a velocity. */
#define STP_TERM_VISCOSITY 1
#define STP_TERM_EXPLICIT 2
#define STP_TERM_DIFFUSION 3
#define STP_TERM_DIVERGENCE 4
#define STP_TERM_LAPLACIAN 5
int stp_eval(stp_handle *h, int term, double *a, double *b, double *c, int where);

/* The SRJ schedule (Sec. 3.4) the library would use for cfg: the Chebyshev
   factors of [mu_min, mu_max] for the Jacobi-preconditioned operator, in the
   mirror-pair order.  M = 0 picks the cycle length; omega needs room for
   1024 values.  Host only. */
int stp_srj_schedule(const stp_config *cfg, int M, double *omega, int *M_out, double *mu_min, double *mu_max);

/* ------------------------------------------------------------------------
 * Learned pressure guess: a 3-D U-Net (4 levels of 16, 32, 64, 128
 * channels, two 3x3x3 convolutions with ReLU per level, 2x2x2 mean pooling,
 * nearest upsampling with skip concatenation, 1x1x1 linear output).
 * Convolutions are periodic in x and y and zero-padded in z.  BF16 weights
 * and activations on the tensor cores with FP32 accumulation; FP32 master
 * weights, gradients and Adam state.  Inputs and outputs are FP32
 * [n][nz][ny][nx] device arrays.  The paper's solver has no learned part:
 * this follows the extension that asks for a learned initial guess of the
 * SRJ pressure iteration, trained on (residual, correction) pairs that the
 * solver itself produces.
 * ------------------------------------------------------------------------ */
typedef struct stp_unet stp_unet;

/* Number of parameters (one flat FP32 vector: per layer, in the order
   enc1a, enc1b, ..., enc4b, dec3a, dec3b, dec2a, dec2b, dec1a, dec1b, out,
   weights [c_out][c_in][taps] (tap = (kz*3 + ky)*3 + kx) then bias). */
long long stp_unet_param_count(void);

/* Network for up to nmax samples of nz x ny x nx (each a multiple of 8, at
   least 8) on the current device; stream NULL: its own stream.  Parameters
   start at zero: set them with stp_unet_set_params.  Its 3x3x3 convolutions
   run on tcgen05 where a level's shape allows (STP_UNET_TC=0 at create:
   mma.sync everywhere), a block computing 1, 2 or 4 z planes chosen by the
   layer's shape (STP_UNET_TC_PLANES=<1|2|4> forces a count where it is
   valid; the forward output does not depend on it).  The mma.sync ones take
   64, 32, 16 or 8 output channels a block by grid size (STP_UNET_MMA_NT=
   <8|4|2|1> forces a width where the channels allow; results do not depend
   on it either). */
int stp_unet_create(int nmax, int nz, int ny, int nx, void *stream, stp_unet **out);
void stp_unet_destroy(stp_unet *net);
const char *stp_unet_last_error(const stp_unet *net);

/* Copy the FP32 parameters in (resets the Adam state) or out. */
int stp_unet_set_params(stp_unet *net, const float *theta, int where);
int stp_unet_get_params(stp_unet *net, float *theta, int where);

/* y = U(x) for nb <= nmax samples (device arrays). */
int stp_unet_forward(stp_unet *net, const float *x, float *y, int nb);

/* Mean squared error of U(x) against target and its gradient with respect
   to the parameters (grad: device FP32 [param_count], nullable). */
int stp_unet_gradient(stp_unet *net, const float *x, const float *target, int nb, float *grad, float *loss);

/* One Adam step (beta 0.9, 0.999, eps 1e-8) on the MSE loss; *loss gets the
   loss before the step. */
int stp_unet_train_step(stp_unet *net, const float *x, const float *target, int nb, float lr, float *loss);

/* Training on solver pairs: r = residual of the previous pressure, dp = the
   exact correction (see stp_set_harvest).  Each sample is scaled by the RMS
   s of its r: the network maps r/s to K dp/s, K the output scale (default
   1; set it so that K dp/s is of order one).  One Adam step per call;
   stp_unet_eval_pairs gives the loss without a step. */
int stp_unet_set_output_scale(stp_unet *net, float k);
int stp_unet_train_pairs(stp_unet *net, const float *r, const float *dp, int nb, float lr, float *loss);
int stp_unet_eval_pairs(stp_unet *net, const float *r, const float *dp, int nb, float *loss);

/* One 3x3x3 convolution of the network on its own, for checks of the
   convolution kernels against an independent definition.  layer is the
   parameter-order index 0..13 (enc1a .. dec1b); it runs at its level's size
   for nb samples, on the kernel the network itself uses for that layer
   (tcgen05 or mma.sync, planes per block as the network picks them).
   Arrays are device FP32, channels last [nb][d][h][w][c]; inputs are
   rounded to BF16 on entry, as the network stores its activations.
     mode 0  forward: out [.., cout] = relu(conv(a) + bias), the BF16 values
             the network stores (layer 0 takes its 1-channel input a in
             FP32, as the network does); b unused
     mode 1  data gradient (layers 1..13): out [.., cin] =
             conv^T(a) * (b > 0), a the gradient of the output [.., cout],
             b a mask [.., cin] (NULL: none), stored in BF16
     mode 2  weight gradient: out [cout*cin*27 + cout] = dW ([o][c][tap])
             then db, for the input a [.., cin] and the output gradient
             b [.., cout]; FP32
   Allocates temporaries and synchronises.  Errors: STP_EINVAL (bad layer,
   mode or nb), STP_ENOMEM, STP_ECUDA, STP_ETIMEOUT. */
#define STP_UNET_FORWARD 0
#define STP_UNET_DATA_GRAD 1
#define STP_UNET_WEIGHT_GRAD 2
int stp_unet_layer(stp_unet *net, int layer, int mode, const float *a, const float *b, float *out, int nb);

/* Use net (NULL: none) as the learned initial guess of every pressure solve
   of h: with s = RMS(r) of the solve's starting residual r, the correction
   s U(r / s) is added to p before the SRJ iteration (once per solve, in
   both precisions).  The SRJ iteration always finishes to ptol.
   The network must match the grid (nz, ny, nx); the handle keeps the
   pointer, which must stay valid while set. */
int stp_set_learned_guess(stp_handle *h, stp_unet *net);

/* How the network of stp_set_learned_guess enters the solve:
     0  (default) initial guess, once per solve, as above;
     1  preconditioner: applied to the current residual throughout the
        solve.  In FP32 with refinement every refinement pass starts its
        inner SRJ solve of L d = r from d = s U(r / s) (s = RMS(r)) instead
        of zero; in FP64, before the sweeps of every SRJ cycle,
        p += s U(r / s) with r = b - L p.  The SRJ iteration still decides
        convergence and finishes to ptol.
   Rebuilds the solve graph. */
int stp_set_learned_mode(stp_handle *h, int mode);

/* Record training pairs of every pressure solve of h into caller device
   arrays (FP32 [nz][ny][nx], NULL: stop): r_out = b - L p_prev at the start
   of the solve, dp_out = p - p_prev after it. */
int stp_set_harvest(stp_handle *h, float *r_out, float *dp_out);

/* ||b - L p||_2 of the pressure equation for caller-owned device arrays p
   and b ([nz][ny][nx], FP64), without allocating anything.  The paper has
   no counterpart: it is for callers that hold their own device buffers but
   may not allocate device memory, for example a host program that has
   handed all device memory to its own pool allocator, or a time-critical
   loop that cannot accept the device-wide synchronisation cudaMalloc and
   cudaFree can cause.  L is the operator of stp_poisson_solve on the grid
   given by nx, ny, nz, Lx, Ly, Lz and stretch (as in stp_config).
     r_out    optional device array [nz][ny][nx] that receives b - L p
     norm_out host pointer that receives the norm
     stream   cudaStream_t of the current device (NULL: the default stream);
              the call synchronises it before returning
   Scratch memory is one fixed device array inside the library (held by
   every GPU that loads the library until the process exits), limited to
   nz <= 4096 and ceil(nx/32) * ceil(ny/8) * nz <= 65536; larger grids are
   rejected with STP_EINVAL.  The first call on a device looks up the
   array's device address; under CUDA's lazy module loading (the default)
   that first call can also load the library's device code, array included, onto the
   device, a one-time allocation made by the CUDA runtime (to have it
   happen earlier, set CUDA_MODULE_LOADING=EAGER or make one call during
   set-up).  All calls share the array: calls whose work overlaps on the GPU
   race and must be serialised by the caller.  Errors: STP_EINVAL,
   STP_ECUDA; stp_last_error(NULL) gives the message. */
int stp_poisson_residual_noalloc(int nx, int ny, int nz, double Lx, double Ly, double Lz, double stretch,
                                 const double *p, const double *b, double *r_out, double *norm_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* STP_H */
