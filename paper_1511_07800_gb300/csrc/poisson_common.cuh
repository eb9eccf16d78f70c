// Device pieces of the pressure solve shared by the per-channel kernels
// (kernels_poisson.cu) and the grouped kernels of the batched step
// (kernels_group.cu): the residual at a point, the FP32 SRJ cell update, one
// FP32 sweep tile, and the per-solve decisions.  Sharing them keeps a
// channel's arithmetic and its stopping decisions bitwise the same in both.
//
// L p = D G p on the MAC grid (Sec. 3.4, Eq. presdiv): periodic in x and y,
// zero flux through the walls,
//   (L p)_k = [(p_{i+1} - p_i) - (p_i - p_{i-1})]/dx^2 + (same in y)
//             + cup_k (p_{k+1} - p_k) - cdn_k (p_k - p_{k-1}).
#pragma once

#include "device_util.cuh"
#include "stp_internal.cuh"

namespace stp {
namespace {

// b - L p at one point, difference form (arithmetic in T)
template <typename T>
__device__ __forceinline__ T point_residual(const Geom<T>& g, const T* __restrict__ p, const T* __restrict__ b,
                                            int i, int j, int k, T* pc_out) {
  const int nx = g.nx, plane = g.nx * g.ny;
  const int ip = i == nx - 1 ? 0 : i + 1, im = i == 0 ? nx - 1 : i - 1;
  const int jp = j == g.ny - 1 ? 0 : j + 1, jm = j == 0 ? g.ny - 1 : j - 1;
  const int row = k * plane;
  const int q = row + j * nx + i;
  const T pc = __ldg(p + q);
  T lap = g.idx2 * ((__ldg(p + row + j * nx + ip) - pc) + (__ldg(p + row + j * nx + im) - pc)) +
          g.idy2 * ((__ldg(p + row + jp * nx + i) - pc) + (__ldg(p + row + jm * nx + i) - pc));
  if (k < g.nz - 1) lap += __ldg(g.cup + k) * (__ldg(p + q + plane) - pc);
  if (k > 0) lap += __ldg(g.cdn + k) * (__ldg(p + q - plane) - pc);
  *pc_out = pc;
  return __ldg(b + q) - lap;
}

// b - L p at one point in FP64, neighbour-sum form: b - (sum_nb c p_nb -
// S p), eight FP64 operations against twelve for the difference form (GB300
// issues FP64 at 1/64 of the FP32 rate).  It rounds with the size of S p
// rather than of the differences, which for a pressure of order one is far
// below the refinement's 1e-8; the FP32 refinement residual uses it, the FP64
// solve keeps the difference form (its sweep counts are compared with the
// oracle's).
__device__ __forceinline__ double point_residual_sum(const Geom<double>& g, const double* __restrict__ p,
                                                     const double* __restrict__ b, int i, int j, int k) {
  const int nx = g.nx, plane = g.nx * g.ny;
  const int ip = i == nx - 1 ? 0 : i + 1, im = i == 0 ? nx - 1 : i - 1;
  const int jp = j == g.ny - 1 ? 0 : j + 1, jm = j == 0 ? g.ny - 1 : j - 1;
  const int row = k * plane;
  const int q = row + j * nx + i;
  double nb = g.idx2 * (__ldg(p + row + j * nx + ip) + __ldg(p + row + j * nx + im));
  nb = fma(g.idy2, __ldg(p + row + jp * nx + i) + __ldg(p + row + jm * nx + i), nb);
  if (k < g.nz - 1) nb = fma(__ldg(g.cup + k), __ldg(p + q + plane), nb);
  if (k > 0) nb = fma(__ldg(g.cdn + k), __ldg(p + q - plane), nb);
  return fma(__ldg(g.S + k), __ldg(p + q), __ldg(b + q) - nb);
}

// One FP32 SRJ update in difference form with a fixed rounding sequence
// (explicit round-to-nearest operations), shared by every FP32 sweep kernel
// so that all of them produce bitwise the same values.
__device__ __forceinline__ float srj_cell_f32(float pc, float xl, float xr, float nn, float ss, float uu, float dd,
                                              float bb, float idx2, float idy2, float cup, float cdn, float iS,
                                              float om) {
  float lap = __fmul_rn(idx2, __fadd_rn(__fsub_rn(xr, pc), __fsub_rn(xl, pc)));
  lap = __fmaf_rn(idy2, __fadd_rn(__fsub_rn(nn, pc), __fsub_rn(ss, pc)), lap);
  lap = __fmaf_rn(cup, __fsub_rn(uu, pc), lap);
  lap = __fmaf_rn(cdn, __fsub_rn(dd, pc), lap);
  return __fmaf_rn(-om, __fmul_rn(__fsub_rn(bb, lap), iS), pc);
}

// One tile of an FP32 sweep: 32 lanes x 4 cells along x (float4), BY rows,
// KZ consecutive z levels per thread (the z neighbours inside the column
// come from registers).  Tile (bx, by, bz) of a grid of
// ceil(nx/128) x ceil(ny/BY) x nz/KZ tiles; nx a multiple of 4, nz of KZ.
// Lanes past the end of a row (or rows past ny) read a clamped, in-bounds
// element, take part in the shuffles and store nothing.  Waits for the
// previous kernel (programmatic dependent launch) before reading p.
template <int KZ, int BY>
__device__ __forceinline__ void sweep_z_tile(const Geom<float>& g, const float* __restrict__ p,
                                             const float* __restrict__ b, float omega, float* __restrict__ out,
                                             int bx, int by, int bz) {
  const int lane = threadIdx.x;
  const int nx = g.nx, ny = g.ny, nx4 = nx >> 2;
  const int x4 = bx * kBX + lane;
  const int j = by * BY + threadIdx.y, k0 = bz * KZ;
  const bool active = x4 < nx4 && j < ny;
  const int xx = x4 < nx4 ? x4 : nx4 - 1;
  const int jj = j < ny ? j : ny - 1;
  // 32-bit float4-unit offsets (fields of fewer than 2^32 cells)
  const unsigned plane4 = (unsigned)nx4 * ny;
  const unsigned rc = (unsigned)jj * nx4 + xx;                             // unit within a level
  const unsigned rn = (unsigned)(jj == ny - 1 ? 0 : jj + 1) * nx4 + xx;    // row j+1
  const unsigned rs = (unsigned)(jj == 0 ? ny - 1 : jj - 1) * nx4 + xx;    // row j-1
  const int xl = xx == 0 ? nx - 1 - 4 * xx : -1, xr = xx == nx4 - 1 ? 4 - nx : 4;  // x-neighbour cells, wrapped
  const unsigned u0 = (unsigned)k0 * plane4;
  const float idx2 = g.idx2, idy2 = g.idy2;
  cudaGridDependencySynchronize();
  const float4* P = reinterpret_cast<const float4*>(p);
  const float4* Bq = reinterpret_cast<const float4*>(b);
  float4 c[KZ + 2];
#pragma unroll
  for (int q = 0; q < KZ; q++) c[q + 1] = __ldg(P + (u0 + q * plane4 + rc));
  c[0] = k0 > 0 ? __ldg(P + (u0 - plane4 + rc)) : c[1];
  c[KZ + 1] = k0 + KZ < g.nz ? __ldg(P + (u0 + KZ * plane4 + rc)) : c[KZ];
#pragma unroll
  for (int q = 0; q < KZ; q++) {
    const int k = k0 + q;
    const unsigned lev = u0 + q * plane4;
    const float cup = __ldg(g.cup + k), cdn = __ldg(g.cdn + k), iS = __ldg(g.iS + k);
    const float4 cc = c[q + 1], zu = c[q + 2], zd = c[q];
    float left = __shfl_up_sync(0xffffffffu, cc.w, 1);
    float right = __shfl_down_sync(0xffffffffu, cc.x, 1);
    const float* pc = p + 4 * (lev + rc);  // first cell of this thread's unit
    if (lane == 0 || xx == 0) left = __ldg(pc + xl);
    if (lane == kBX - 1 || xx == nx4 - 1) right = __ldg(pc + xr);
    const float4 yn = __ldg(P + (lev + rn));
    const float4 ys = __ldg(P + (lev + rs));
    const float4 bq = __ldg(Bq + (lev + rc));
    auto cell = [&](float pcv, float xlv, float xrv, float nn, float ss, float uu, float dd, float bb) {
      return srj_cell_f32(pcv, xlv, xrv, nn, ss, uu, dd, bb, idx2, idy2, cup, cdn, iS, omega);
    };
    float4 o;
    o.x = cell(cc.x, left, cc.y, yn.x, ys.x, zu.x, zd.x, bq.x);
    o.y = cell(cc.y, cc.x, cc.z, yn.y, ys.y, zu.y, zd.y, bq.y);
    o.z = cell(cc.z, cc.y, cc.w, yn.z, ys.z, zu.z, zd.z, bq.z);
    o.w = cell(cc.w, cc.z, right, yn.w, ys.w, zu.w, zd.w, bq.w);
    if (active) reinterpret_cast<float4*>(out)[lev + rc] = o;
  }
}

// One tile of an FP32 sweep with warps packed along the plane: the channel
// is cut into z-slabs of KZ levels, and the float4 units of a slab's plane
// (nx/4 x ny of them, p = j nx/4 + x4) are taken 256 at a time in the
// order slab, then p.  Tile t holds units 256 t .. 256 t + 255 of that
// sequence, so a warp is full whatever the row length (rows shorter than a
// warp share it); a thread owns one unit at KZ levels.  Requires nx a
// multiple of 4, nz of KZ and nx/4 * ny of 32 (a warp never straddles two
// slabs).  x-neighbours come from the adjacent lanes when they hold the
// same row, else by a scalar load (the periodic wrap, and lanes 0 and 31).
template <int KZ>
__device__ __forceinline__ void sweep_flat_tile(const Geom<float>& g, const float* __restrict__ p,
                                                const float* __restrict__ b, float omega, float* __restrict__ out,
                                                int t) {
  const int lane = threadIdx.x;
  const int nx = g.nx, ny = g.ny, nx4 = nx >> 2;
  const int plane4 = nx4 * ny;
  const int nunits = (g.nz / KZ) * plane4;
  const int f0 = t * (kBX * kBY) + threadIdx.y * kBX + lane;
  const bool active = f0 < nunits;  // whole warps (nunits is a multiple of 32)
  const int f = active ? f0 : nunits - 1;
  const int slab = f / plane4, pi = f - slab * plane4;
  const int j = pi / nx4, x4 = pi - j * nx4;
  const int k0 = slab * KZ;
  // 32-bit float4-unit offsets (fields of fewer than 2^32 cells)
  const unsigned rn = (unsigned)(j == ny - 1 ? 0 : j + 1) * nx4 + x4;
  const unsigned rs = (unsigned)(j == 0 ? ny - 1 : j - 1) * nx4 + x4;
  const int xl = x4 == 0 ? nx - 1 : -1, xr = x4 == nx4 - 1 ? 4 - nx : 4;  // x-neighbour cells, wrapped
  const unsigned u0 = (unsigned)k0 * plane4;
  const float idx2 = g.idx2, idy2 = g.idy2;
  cudaGridDependencySynchronize();
  const float4* P = reinterpret_cast<const float4*>(p);
  const float4* Bq = reinterpret_cast<const float4*>(b);
  float4 c[KZ + 2];
#pragma unroll
  for (int q = 0; q < KZ; q++) c[q + 1] = __ldg(P + (u0 + q * plane4 + pi));
  c[0] = k0 > 0 ? __ldg(P + (u0 - plane4 + pi)) : c[1];
  c[KZ + 1] = k0 + KZ < g.nz ? __ldg(P + (u0 + KZ * plane4 + pi)) : c[KZ];
#pragma unroll
  for (int q = 0; q < KZ; q++) {
    const int k = k0 + q;
    const unsigned lev = u0 + q * plane4;
    const float cup = __ldg(g.cup + k), cdn = __ldg(g.cdn + k), iS = __ldg(g.iS + k);
    const float4 cc = c[q + 1], zu = c[q + 2], zd = c[q];
    float left = __shfl_up_sync(0xffffffffu, cc.w, 1);
    float right = __shfl_down_sync(0xffffffffu, cc.x, 1);
    const float* pc = p + 4 * (lev + pi);  // first cell of this thread's unit
    if (lane == 0 || x4 == 0) left = __ldg(pc + xl);
    if (lane == kBX - 1 || x4 == nx4 - 1) right = __ldg(pc + xr);
    const float4 yn = __ldg(P + (lev + rn));
    const float4 ys = __ldg(P + (lev + rs));
    const float4 bq = __ldg(Bq + (lev + pi));
    auto cell = [&](float pcv, float xlv, float xrv, float nn, float ss, float uu, float dd, float bb) {
      return srj_cell_f32(pcv, xlv, xrv, nn, ss, uu, dd, bb, idx2, idy2, cup, cdn, iS, omega);
    };
    float4 o;
    o.x = cell(cc.x, left, cc.y, yn.x, ys.x, zu.x, zd.x, bq.x);
    o.y = cell(cc.y, cc.x, cc.z, yn.y, ys.y, zu.y, zd.y, bq.y);
    o.z = cell(cc.z, cc.y, cc.w, yn.z, ys.z, zu.z, zd.z, bq.z);
    o.w = cell(cc.w, cc.z, right, yn.w, ys.w, zu.w, zd.w, bq.w);
    if (active) reinterpret_cast<float4*>(out)[lev + pi] = o;
  }
}

// FP32 sweep variants, as set_sweep_variant numbers them:
//   0        one level per thread, 32 x 8 threads over 128 x 8 cells
//   1 .. 5   (KZ, BY) = (2,8), (4,8), (2,4), (4,4), (8,4): KZ levels per
//            thread, 32 x BY threads
//   6 .. 8   warps packed along the plane (sweep_flat_tile), KZ = 2, 4, 8
//   9 .. 11  two sweeps per launch on a shared-memory tile of TY rows x
//            TZ levels x all of x (k_sweep_f32_pair), (TY, TZ) = (8,4),
//            (4,4), (4,8); used only for cycles of a multiple of 4 sweeps
constexpr int kSweepVariants = 12;
__host__ __device__ constexpr int sweep_kz(int v) {
  return v == 0 ? 1 : v == 1 ? 2 : v == 2 ? 4 : v == 3 ? 2 : v == 4 ? 4 : v == 5 ? 8 : v == 6 ? 2 : v == 7 ? 4
         : v == 8 ? 8 : v == 9 ? 4 : v == 10 ? 4 : 8;
}
__host__ __device__ constexpr int sweep_by(int v) { return (v >= 3 && v <= 5) || v == 10 || v == 11 ? 4 : 8; }
__host__ __device__ constexpr bool sweep_flat(int v) { return v >= 6 && v <= 8; }
__host__ __device__ constexpr bool sweep_pair(int v) { return v >= 9; }

// shared memory of a pair-sweep tile: input p with two ghost rows and
// levels on each side, b and the first sweep's result with one
__host__ __device__ constexpr size_t pair_smem_bytes(int ty, int tz, int nx) {
  return (size_t)((tz + 4) * (ty + 4) + 2 * (tz + 2) * (ty + 2)) * (nx / 4) * 16;
}
constexpr size_t kPairSmemMax = 227 * 1024;

// Start of a solve: fold the previous solve into the totals, reset the state.
__device__ __forceinline__ void begin_solve_state(SolveCtl* ctl) {
  if (ctl->solves > 0) {
    ctl->tot_sweeps += ctl->sweeps;
    ctl->tot_kernels += ctl->kernels;
    ctl->nonconv += ctl->converged ? 0 : 1;
  }
  ctl->solves += 1;
  ctl->sweeps = 0;
  ctl->passes = 0;
  ctl->cycles_inner = 0;
  ctl->converged = 0;
  ctl->prev = 0.0;
  ctl->kernels = 1;
}

// Once-per-cycle decision from res = ||b - L p|| of the cycle's input.
// MODE 0: FP64 solve, stop at res <= tol ||b||; MODE 1: FP32 inner solve of
// the refinement, stop at max(inner_tol ||r||, tol ||b|| / 2) or when a
// cycle gains less than 10 %.  Both stop at the sweep cap and on NaN/Inf.
// Returns true to run the cycle's M sweeps.  Also returns the reduction
// counter to zero.
template <int MODE>
__device__ __forceinline__ bool cycle_decide(SolveCtl* ctl, const Red& red, double res) {
  const double nb = red.sc[SC_BNORM];
  bool stop;
  ctl->kernels += 1;
  if (ctl->bad) {
    stop = true;  // a cycle kernel gave up waiting (ctl->bad = 2)
  } else if (!(res == res) || isinf(res)) {
    ctl->bad = 1;
    stop = true;
  } else if (MODE == 0) {
    ctl->res = res;
    ctl->converged = res <= ctl->tol * nb;
    stop = ctl->converged || ctl->sweeps >= ctl->max_sweeps;
  } else {
    const double target = fmax(ctl->inner_tol * red.sc[SC_INNER_REF], 0.5 * ctl->tol * nb);
    const bool stall = ctl->cycles_inner > 0 && res > 0.9 * ctl->prev;
    ctl->res_inner = res;
    stop = res <= target || stall || ctl->sweeps >= ctl->max_sweeps;
    ctl->prev = res;
  }
  if (!stop) {
    ctl->sweeps += ctl->M;
    ctl->cycles_inner += 1;
    ctl->kernels += ctl->kpc;
  }
  *red.counter = 0u;
  ctl->go = stop ? 0 : 1;
  return !stop;
}

// Refinement-pass decision from res = ||b - L p|| in FP64 (the residual
// after a pass when after_pass).  Returns true to run another pass.
__device__ __forceinline__ bool pass_decide(SolveCtl* ctl, const Red& red, double res, int after_pass) {
  const double nb = red.sc[SC_BNORM];
  ctl->kernels += 1 + (after_pass ? 1 : 0);  // this kernel and the correction before it
  if (after_pass) ctl->passes += 1;
  ctl->res = res;
  red.sc[SC_INNER_REF] = res;
  ctl->cycles_inner = 0;
  ctl->prev = 0.0;
  bool stop;
  if (ctl->bad) {
    stop = true;
  } else if (!(res == res) || isinf(res)) {
    ctl->bad = 1;
    stop = true;
  } else {
    ctl->converged = res <= ctl->tol * nb;
    stop = ctl->converged || ctl->sweeps >= ctl->max_sweeps || ctl->passes >= ctl->max_passes;
  }
  *red.counter = 0u;
  ctl->go = stop ? 0 : 1;
  return !stop;
}

}  // namespace
}  // namespace stp
