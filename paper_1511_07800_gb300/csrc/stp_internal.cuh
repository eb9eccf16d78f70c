// Internal declarations of the GB300 projection-step library: device geometry,
// the handle, deterministic reductions and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include <string>
#include <vector>

#include "../../include/stp.h"

namespace stp {

// ---------------------------------------------------------------------------
// Grid metrics.  z is stretched or uniform; x and y are uniform.  Every 1-D
// array lives in device memory (read through the read-only path).
//   dz[k]   cell width            k < nz
//   hz[c]   centre-to-centre distance across face c (c = 1..nz-1)
//   dzf[c]  distance between the two u-values that straddle face c; at a wall
//           the ghost is the mirror image of the first centre (dzf = dz)
// ---------------------------------------------------------------------------
template <typename T>
struct Geom {
  int nx, ny, nz;
  T idx, idy;      // 1/dx, 1/dy
  T idx2, idy2;    // 1/dx^2, 1/dy^2
  T hidx, hidy;    // 1/(2dx), 1/(2dy)
  T idxdy;         // 1/(dx dy)
  const T* idz;    // [nz]    1/dz
  const T* ihz;    // [nz+1]  1/hz (interior faces)
  const T* idzf;   // [nz+1]  1/dzf
  const T* i2dzc;  // [nz]    1/(distance between the centres (or ghosts) above and below)
  const T* idzw;   // [nz+1]  1/(dz[c] + dz[c-1]) at interior faces
  const T* cup;    // [nz]    Poisson coupling to k+1 (0 at the top wall)
  const T* cdn;    // [nz]    Poisson coupling to k-1 (0 at the bottom wall)
  const T* iS;     // [nz]    1/(2/dx^2 + 2/dy^2 + cup + cdn)
  const T* S;      // [nz]    2/dx^2 + 2/dy^2 + cup + cdn
  const T* lm2;    // [nz]    (Cs Delta phi_w)^2 per level (LES)
  const T* dzv;    // [nz]    dz
  const T* li;     // [nz]    z-line Thomas: 1/m_k, m_k the k-th pivot of A = -L_z + (2/dx^2 + 2/dy^2) I
  const T* lu;     // [nz]    z-line Thomas: cup_k/m_k
  // z-line twisted factorisation of the same A, eliminated from both walls
  // towards the twist level t = nz/2 (top-down pivots m_k above it,
  // bottom-up pivots m'_k below, gamma_t at it):
  const T* tli;    // [nz]    1/m_k (k < t), 1/gamma_t (k = t), 1/m'_k (k > t)
  const T* tlf;    // [nz]    elimination: cdn_k/m_k (k < t), cdn_t/gamma_t, cup_k/m'_k (k > t)
  const T* tlb;    // [nz]    substitution: cup_k/m_k (k < t), cup_t/gamma_t, cdn_k/m'_k (k > t)
  // FP32 only (null in FP64): {cup_k, cdn_k, tli_k, tlf_k} packed per level,
  // one 16-byte load for the z-line sweep's level coefficients
  const float4* lz4;
};

// Number of metric arrays packed into one device allocation per precision.
constexpr int kMetricArrays = 16;

// Reduction workspace (device).  Every reducing kernel writes one partial per
// block, then the last block to finish sums the partials in block order, so
// results do not depend on scheduling.
struct Red {
  double* partial;    // [2 * max_blocks]
  unsigned* counter;  // [1], returns to 0 after each reduction
  double* sc;         // scalars, see SC_* below
  int* flag;          // flags, see FL_* below
  unsigned* gcount;   // [max_blocks / 64 + 1] arrival counters of groups of 64 blocks (0 between reductions)
};

enum {
  SC_BNORM = 0,     // ||b||_2 of the current Poisson right-hand side
  SC_RES = 1,       // ||r||_2 at the last check
  SC_INNER_REF = 2, // ||r||_2 of the outer residual (inner solve reference)
  SC_BULK = 3,      // volume mean of u after the correction
  SC_UMAX = 4,      // max |u| after the correction
  SC_SHIFT = 5,     // flux fix-up added to u
  SC_RES_INNER = 6, // inner residual at the last inner check
  SC_VSUM = 7,      // volume sum of a field (stp_poisson_solve's mean checks)
  SC_VABS = 8,      // volume sum of its absolute value
  SC_BMEAN = 9,     // a volume mean of b to remove in the refinement residual (0: b from the step telescopes)
  SC_COUNT = 10
};
enum { FL_DONE = 0, FL_INNER_DONE = 1, FL_BAD = 2, FL_COUNT = 4 };

// grid-wide barrier state of the persistent SRJ cycle kernel (device)
struct GridBar {
  unsigned* count;  // arrivals in the current barrier
  unsigned* gen;    // completed barriers
  int* err;         // set when a wait timed out
};

struct Launch {
  dim3 grid, block;
  unsigned nblocks;
};

// Device-resident control block of the pressure solves.  The host writes
// the parameters once per call; the check kernels update the state and set
// the graph conditionals; k_begin folds the previous solve into the totals.
struct SolveCtl {
  // parameters
  double tol;        // ||b - L p|| <= tol ||b||
  double inner_tol;  // FP32 inner solve: reduce the refinement residual by this
  int max_sweeps;    // cap on SRJ sweeps per solve
  int max_passes;    // cap on refinement passes per solve
  int M;             // SRJ cycle length
  int kpc;           // kernels that run the M sweeps of a cycle
  // state of the current solve
  int sweeps, passes, cycles_inner, converged, bad, pad1;
  double prev, res, res_inner;
  long long kernels;  // kernels run by the solve graph
  int go;             // last decision of a check kernel (1: run the cycle / pass)
  int pad2;
  // totals over the earlier solves of this call
  long long tot_sweeps, tot_kernels;
  int solves, nonconv;
  // longest wait of a grid barrier of the persistent SRJ cycle, in SM clock
  // cycles (about one second by default; STP_BARRIER_WAIT overrides it)
  long long bar_wait;
  // added to the sweep count a persistent z-line tile waits for (0; a
  // positive value, from STP_WAIT_SKEW, asks for a count nothing reaches,
  // so that a test can make the bounded waits run out)
  int wait_skew;
  int pad3;
};

// ---------------------------------------------------------------------------
// Kernel launchers (kernels_step.cu, kernels_poisson.cu).  T is the storage
// and arithmetic type of the velocity fields (double or float).
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_viscosity(const Geom<T>& g, const T* u, const T* v, const T* w, T nu0, T* nu,
                             cudaStream_t s);

// Adams-Bashforth history: three slots per component; step n (the number
// of steps taken since the fields were set, read on the device) writes
// N^n into slot n % 3 and reads N^{n-1}, N^{n-2} from the others, with
// forward Euler at n = 0, AB2 at n = 1 and AB3 after.
template <typename T>
struct Hist {
  T* u[3];
  T* v[3];
  T* w[3];
  const int* step;
};

template <typename T>
cudaError_t launch_momentum(const Geom<T>& g, bool les, const T* u, const T* v, const T* w, const T* nu,
                            T nu0, T fx, Hist<T> H, T dt, T* ru, T* rv, T* rw, cudaStream_t s);

// end of a step: (*step)++
cudaError_t launch_step_end(int* step, cudaStream_t s);

template <typename T>
cudaError_t launch_cn_sweep(const Geom<T>& g, bool les, const T* nu, T nu0, T hdt, const T* ru, const T* rv,
                            const T* rw, const T* au, const T* av, const T* aw, T* ou, T* ov, T* ow,
                            cudaStream_t s);

// One z-line Jacobi sweep of the same system (columns solved by Thomas,
// x-y neighbours from a); scratch holds 3 (nz + 1) nx ny pairs of T.
template <typename T>
cudaError_t launch_cn_line(const Geom<T>& g, bool les, const T* nu, T nu0, T hdt, const T* ru, const T* rv,
                           const T* rw, const T* au, const T* av, const T* aw, T* ou, T* ov, T* ow, void* scratch,
                           const T* piv, cudaStream_t s);
// 1/pivot of every z column's Crank-Nicolson matrix (once per step, before
// the sweeps that pass piv to launch_cn_line; columns of 2 to 192 levels)
template <typename T>
cudaError_t launch_cn_pivots(const Geom<T>& g, bool les, const T* nu, T nu0, T hdt, T* piv, cudaStream_t s);
bool cn_chunk_ok(int nz);

// b = D u / dt (FP64 arithmetic in both precisions), ||b||^2 reduced into
// sc[SC_BNORM] (as the norm), flags reset; sc[SC_BMEAN] = 0 (b telescopes).
template <typename T>
cudaError_t launch_divergence_rhs(const Geom<T>& g, const T* u, const T* v, const T* w, double idt, double* b,
                                  Red red, double Lz, cudaStream_t s);

// Terms for checks (stp_eval).
template <typename T>
cudaError_t launch_explicit_only(const Geom<T>& g, bool les, const T* u, const T* v, const T* w, const T* nu,
                                 T nu0, T fx, T* Nu, T* Nv, T* Nw, cudaStream_t s);
template <typename T>
cudaError_t launch_diffusion_only(const Geom<T>& g, bool les, const T* u, const T* v, const T* w, const T* nu,
                                  T nu0, T* Du, T* Dv, T* Dw, cudaStream_t s);

// One z-line Jacobi-SOR sweep: out = p - omega A^-1 (b - L p), A the z
// column operator -L_z + (2/dx^2 + 2/dy^2) I (Thomas with the pivots li, lu).
template <typename T>
cudaError_t launch_line_sweep(const Geom<T>& g, const T* p, const T* b, T omega, T* out, cudaStream_t s,
                              int variant);
// whether the register-chunked FP32 line sweep (variant 1) takes the grid
bool line_chunk_ok(int nx, int nz);

// One Jacobi-SOR sweep of L p = b with factor omega: out = p - omega (b - Lp)/S.
template <typename T>
cudaError_t launch_sweep(const Geom<T>& g, const T* p, const T* b, T omega, T* out, cudaStream_t s);
template <>
cudaError_t launch_sweep<float>(const Geom<float>&, const float*, const float*, float, float*, cudaStream_t);
template <>
cudaError_t launch_sweep<double>(const Geom<double>&, const double*, const double*, double, double*, cudaStream_t);

// FP32 sweep variant used by launch_sweep<float> on this host thread
// (chosen by the autotuner in api.cu).
void set_sweep_variant(int v);
int sweep_variant_count();
bool sweep_variant_ok(int v, int nx, int ny, int nz);
// variants 9..11 run two sweeps per launch (launch_sweep_pair, cycles of a
// multiple of 4 sweeps only); launch_sweep falls back to variant 0 for them
bool sweep_variant_is_pair(int v);
cudaError_t launch_sweep_pair(const Geom<float>& g, const float* p, const float* b, float om_a, float om_b,
                              float* out, cudaStream_t s);

// ||b - L p|| and the once-per-cycle decision (mode 0: FP64 solve, mode 1:
// FP32 inner solve); sets the WHILE (h_loop) and IF (h_body) conditionals.
// Outside a graph (graph == 0) the decision is only written to ctl->go.
template <typename T>
cudaError_t launch_check(const Geom<T>& g, const T* p, const T* b, int mode, SolveCtl* ctl, Red red, int graph,
                         cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_body, cudaStream_t s);

// Refinement residual r = b - L p (FP64, stored FP32) and the pass decision.
cudaError_t launch_outer(const Geom<double>& g, const double* p, const double* b, float* r32, SolveCtl* ctl, Red red,
                         int after_pass, int graph, cudaGraphConditionalHandle h_loop, cudaStream_t s);
// One SRJ cycle of M FP32 sweeps (A -> B -> A ...) in one cooperative
// launch of nblocks x 1024 threads (nblocks from cycle_grid_f32).
int cycle_grid_f32(int device);
cudaError_t launch_cycle_f32(const Geom<float>& g, float* A, float* B, const float* b, const float* omega, int M,
                             GridBar bar, SolveCtl* ctl, int nblocks, cudaStream_t s);
// One SRJ cycle of M FP32 z-line sweeps in one cooperative launch, tiles
// synchronised with their x-y neighbours through flags (ints, one a tile,
// zero at the start of a call).  line_cycle_rows: the tile's rows, 0 when
// the grid cannot run it (then the per-sweep kernels run).
int line_cycle_rows(const Geom<float>& g, int device);
int line_cycle_tiles(const Geom<float>& g, int rb);
cudaError_t launch_line_cycle_f32(const Geom<float>& g, int rb, float* A, float* B, const float* b,
                                  const float* omega, int M, int* flags, SolveCtl* ctl, cudaStream_t s);
// start of a refinement pass: d = 0 and the inner loop armed
cudaError_t launch_pass_begin(float* d, size_t n, int graph, cudaGraphConditionalHandle h_loop, cudaStream_t s);
// p += d
cudaError_t launch_addcorr(double* p, const float* d, size_t n, cudaStream_t s);
// out = a - b (FP64 in, FP32 out)
cudaError_t launch_difference(const double* a, const double* b, float* out, size_t n, cudaStream_t s);
// start of a solve: fold the previous solve into the totals, reset the state
// (in a graph it also arms the WHILE handle h_loop of an FP64 solve)
cudaError_t launch_begin(SolveCtl* ctl, int graph, cudaGraphConditionalHandle h_loop, cudaStream_t s);

// ---------------------------------------------------------------------------
// Grouped FP32 pressure solves (kernels_group.cu).  In the batched step the
// channels that share an SRJ cycle length M are solved in lock step: each
// kernel of the solve covers the tiles of every channel of the group in one
// launch (block -> channel by a search over the channels' first tiles), and
// each channel keeps its own schedule, residuals, counters and stopping
// decisions, so it computes exactly what its own solve computes.  A channel
// that has stopped skips its tiles.  The channel deciding last in a kernel
// sets the graph conditionals: the loops run while any channel continues.
// ---------------------------------------------------------------------------
struct GChan {
  Geom<float> g32;
  Geom<double> g64;
  double* p;
  const double* b;
  float* d1;           // inner correction (cycle input and output)
  float* d2;           // its ping-pong partner
  float* r32;          // refinement residual (inner right-hand side)
  const float* omega;  // [M] FP32 schedule
  SolveCtl* ctl;
  Red red;
};

struct GState {
  unsigned arrived;     // channels that have decided in the current kernel
  unsigned n_go;        // of those, the ones that continue
  unsigned part_pass;   // channels in the current refinement pass
  unsigned part_inner;  // channels in the current inner SRJ loop
  long long kernels;    // grouped kernels run (all solves since the counter was cleared)
};

struct Group {
  const GChan* ch;  // [n]
  const int* soff;  // [n+1] first 32 x 8 one-level tile of each channel (residuals, element-wise work)
  const int* voff;  // [n+1] first sweep tile of each channel (sweep variant kz x by)
  int* pass_on;     // [n] channel in the current refinement pass
  int* inner_on;    // [n] channel in the current inner SRJ loop
  GState* gs;
  int n, M;
  int stiles, vtiles;
  int variant;      // FP32 sweep tile variant (as set_sweep_variant numbers them)
};

// tile counts of one channel: one-level 32 x 8 tiles, and sweep tiles of a variant
int group_scalar_tiles(int nx, int ny, int nz);
int group_sweep_tiles(int variant, int nx, int ny, int nz);
cudaError_t launch_group_begin(const Group& G, cudaStream_t s);
cudaError_t launch_group_outer(const Group& G, int after_pass, cudaGraphConditionalHandle h_pass, cudaStream_t s);
cudaError_t launch_group_pass_begin(const Group& G, cudaGraphConditionalHandle h_loop, cudaStream_t s);
cudaError_t launch_group_check(const Group& G, cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_body,
                               cudaStream_t s);
cudaError_t launch_group_sweep(const Group& G, int m, cudaStream_t s);
cudaError_t launch_group_addcorr(const Group& G, cudaStream_t s);

// LES statistics (les_stats.cu): plane sums of the kStatMoments moments of
// the cell-centred velocities per level (mom[m * nz + k]) and streamwise
// two-point products of u, v, wc at level kc (corr[c * nx + d]), added to the
// buffers.
constexpr int kStatMoments = 9;
template <typename T>
cudaError_t launch_les_stats(int nx, int ny, int nz, int kc, const T* u, const T* v, const T* w, double* mom,
                             double* corr, cudaStream_t s);

// batched step: counter[0] = steps done, counter[1] = steps wanted
cudaError_t launch_batch_begin(int* counter, cudaGraphConditionalHandle h_steps, cudaStream_t s);
cudaError_t launch_batch_end(int* counter, cudaGraphConditionalHandle h_steps, cudaStream_t s);

// Velocity correction (Eq. project u_p_1) with walls; reduces the volume
// mean of u and max |u|.  The pressure is FP64 in both modes; ihz64 and dz64
// are the FP64 metrics 1/hz and dz.
template <typename T>
cudaError_t launch_correct_impl(const Geom<T>& g, const double* p, double dt, T* u, T* v, T* w,
                                const double* ihz64, const double* dz64, double inv_vol, Red red, cudaStream_t s);

// u += target - sc[SC_BULK] (constant-flux fix-up).
template <typename T>
cudaError_t launch_flux_shift(const Geom<T>& g, T* u, double target, Red red, cudaStream_t s);

cudaError_t launch_laplacian(const Geom<double>& g, const double* p, double* out, cudaStream_t s);

template <typename Td, typename Ts>
cudaError_t launch_convert(Td* dst, const Ts* src, size_t n, cudaStream_t s);

// Volume sums sum a dz and sum |a| dz of a cell-centred FP64 field into
// sc[SC_VSUM], sc[SC_VABS]; a -= (its volume-weighted mean), read from
// sc[SC_VSUM] on the device (Lz the box height).
cudaError_t launch_vsum(const Geom<double>& g, const double* a, Red red, cudaStream_t s);
cudaError_t launch_sub_vmean(const Geom<double>& g, double* a, double Lz, Red red, cudaStream_t s);

// ||a||_2 of a double array into sc[slot].
cudaError_t launch_norm(const double* a, size_t n, int slot, Red red, cudaStream_t s);

// learned guess (unet.cu)
bool unet_matches(const stp_unet* n, int nz, int ny, int nx);
int unet_guess(stp_unet* n, const float* r, const double* norm, float* d, cudaStream_t st, int* kernels);

// Raise a kernel's dynamic shared-memory limit on the current device the
// first time it is launched there (the attribute is per device; `done`
// holds one bit per device, devices 0-31; setting it twice is harmless).
template <typename K>
inline cudaError_t smem_limit_once(K kern, int bytes, std::atomic<unsigned>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned bit = 1u << (dev & 31);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

}  // namespace stp
