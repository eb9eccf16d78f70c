// Pressure-Poisson kernels (arXiv 1511.07800, Sec. 3.4 and Eq. presdiv).
//
// L p = D G p on the MAC grid: periodic in x and y, zero flux through the
// walls (Neumann):
//   (L p)_k = [(p_{i+1} - p_i) - (p_i - p_{i-1})]/dx^2 + (same in y)
//             + cup_k (p_{k+1} - p_k) - cdn_k (p_k - p_{k-1}),
// cup_k = 1/(hz_{k+1} dz_k) (0 at the top), cdn_k = 1/(hz_k dz_k) (0 at the
// bottom), S_k = 2/dx^2 + 2/dy^2 + cup_k + cdn_k.
//
// Jacobi-SOR (Eq. Jacobi-SOR in 3-D): p' = (1 - omega) p + omega p^J with
// p^J = (sum_nb c p_nb - b)/S.  Since p^J - p = -(b - L p)/S, the sweep is
// written p' = p - omega (b - L p)/S with L p in difference form, which in
// FP32 avoids the cancellation of sum_nb c p_nb against S p.
//
// The solve is driven on the device: a residual-check kernel decides, once
// per SRJ cycle, whether to run the cycle's M sweeps, and sets the graph
// conditionals (WHILE over cycles, IF around the sweeps) -- see api.cu.
#include <algorithm>

#include "device_util.cuh"
#include "poisson_common.cuh"
#include "stp_internal.cuh"

namespace stp {

namespace {
// FP32: difference form (no cancellation against S p).
__global__ void __launch_bounds__(kBX* kBY) k_sweep_f32(Geom<float> g, const float* __restrict__ p,
                                                         const float* __restrict__ b, float omega,
                                                         float* __restrict__ out) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const int nx = g.nx, plane = g.nx * g.ny;
  const int ip = i == nx - 1 ? 0 : i + 1, im = i == 0 ? nx - 1 : i - 1;
  const int jp = j == g.ny - 1 ? 0 : j + 1, jm = j == 0 ? g.ny - 1 : j - 1;
  const int row = k * plane, q = row + j * nx + i;
  const float pc = __ldg(p + q);
  const float uu = k < g.nz - 1 ? __ldg(p + q + plane) : pc, dd = k > 0 ? __ldg(p + q - plane) : pc;
  out[q] = srj_cell_f32(pc, __ldg(p + row + j * nx + im), __ldg(p + row + j * nx + ip), __ldg(p + row + jp * nx + i),
                        __ldg(p + row + jm * nx + i), uu, dd, __ldg(b + q), g.idx2, g.idy2, __ldg(g.cup + k),
                        __ldg(g.cdn + k), __ldg(g.iS + k), omega);
}

// FP64: the neighbour-sum form p + omega (p^J - p), p^J = (sum_nb c p_nb - b)/S,
// which needs fewest FP64 operations (the FP64 sweep is bound by FP64
// arithmetic on this part, not by memory).
__global__ void __launch_bounds__(kBX* kBY) k_sweep_f64(Geom<double> g, const double* __restrict__ p,
                                                         const double* __restrict__ b, double omega,
                                                         double* __restrict__ out) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const int nx = g.nx, plane = g.nx * g.ny;
  const int ip = i == nx - 1 ? 0 : i + 1, im = i == 0 ? nx - 1 : i - 1;
  const int jp = j == g.ny - 1 ? 0 : j + 1, jm = j == 0 ? g.ny - 1 : j - 1;
  const int row = k * plane;
  const int q = row + j * nx + i;
  const double pc = __ldg(p + q);
  double nb = g.idx2 * (__ldg(p + row + j * nx + ip) + __ldg(p + row + j * nx + im)) +
              g.idy2 * (__ldg(p + row + jp * nx + i) + __ldg(p + row + jm * nx + i));
  if (k < g.nz - 1) nb += __ldg(g.cup + k) * __ldg(p + q + plane);
  if (k > 0) nb += __ldg(g.cdn + k) * __ldg(p + q - plane);
  const double pj = (nb - __ldg(b + q)) * __ldg(g.iS + k);
  out[q] = pc + omega * (pj - pc);
}

// Vectorised sweeps: each thread owns 4 consecutive cells of a row (float4
// in FP32, double2 pairs in FP64); the x-neighbours across lanes come by
// warp shuffle, so a cell costs one vector load per stencil direction
// instead of eight scalar loads and their index arithmetic.  Lanes past the
// end of a row (or rows past ny) read a clamped, in-bounds element, take
// part in the shuffles and store nothing.  Launched as programmatic
// dependents: set-up overlaps the previous kernel's tail, and
// cudaGridDependencySynchronize waits for its results before any read of p.
// FP32 sweep with KZ consecutive z levels per thread (the z neighbours
// inside the column come from registers, and a thread has KZ rows of loads
// in flight) and BY rows per block (sweep_z_tile).  nz must be a multiple of
// KZ.  Identical arithmetic per cell for every (KZ, BY).
template <int KZ, int BY>
__global__ void __launch_bounds__(kBX* BY) k_sweep_f32_z(Geom<float> g, const float* __restrict__ p,
                                                          const float* __restrict__ b, float omega,
                                                          float* __restrict__ out) {
  sweep_z_tile<KZ, BY>(g, p, b, omega, out, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <int KZ>
__global__ void __launch_bounds__(kBX* kBY) k_sweep_f32_flat(Geom<float> g, const float* __restrict__ p,
                                                             const float* __restrict__ b, float omega,
                                                             float* __restrict__ out) {
  sweep_flat_tile<KZ>(g, p, b, omega, out, blockIdx.x);
}

// 16-byte asynchronous copy global -> shared, and the wait for all of them
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Two consecutive SRJ sweeps (omega_a, then omega_b) in one launch.  A block
// owns TY rows x TZ levels x all of x of the output.  It stages p on its
// tile widened by two rows and two levels on each side (rows wrap
// periodically; levels past a wall are not needed: the wall cell uses its
// own value, as in every sweep kernel) and b widened by one, computes the
// first sweep on the tile widened by one into shared memory, then the
// second sweep on the tile itself into global memory.  The widened part of
// the first sweep repeats what the neighbouring blocks compute, with the
// same inputs and the same cell function, so the result is bitwise that of
// two single sweeps.  b is constant over a cycle and is copied before the
// wait for the previous launch; p after it.
template <int TY, int TZ>
__global__ void __launch_bounds__(256) k_sweep_f32_pair(Geom<float> g, const float* __restrict__ p,
                                                         const float* __restrict__ b, float om_a, float om_b,
                                                         float* __restrict__ out) {
  extern __shared__ float4 sm[];
  constexpr int RY0 = TY + 4, RZ0 = TZ + 4, RY1 = TY + 2, RZ1 = TZ + 2;
  const int nx = g.nx, ny = g.ny, nz = g.nz, nx4 = nx >> 2;
  float4* P0 = sm;                    // [RZ0][RY0][nx4]  p, levels k0-2.., rows j0-2..
  float4* B1 = P0 + RZ0 * RY0 * nx4;  // [RZ1][RY1][nx4]  b, levels k0-1.., rows j0-1..
  float4* P1 = B1 + RZ1 * RY1 * nx4;  // [RZ1][RY1][nx4]  first sweep, same region as B1
  const int j0 = blockIdx.x * TY, k0 = blockIdx.y * TZ;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const float4* Pg = reinterpret_cast<const float4*>(p);
  const float4* Bg = reinterpret_cast<const float4*>(b);
  const float idx2 = g.idx2, idy2 = g.idy2;
  const int n1 = RZ1 * RY1 * nx4;
  for (int q = tid; q < n1; q += nthr) {
    const int x4 = q % nx4, r = q / nx4, yt = r % RY1, zt = r / RY1;
    const int k = k0 - 1 + zt;
    if (k < 0 || k >= nz) continue;
    const int j = ((j0 - 1 + yt) % ny + ny) % ny;
    cp_async16(B1 + q, Bg + ((size_t)k * ny + j) * nx4 + x4);
  }
  cudaGridDependencySynchronize();
  const int n0 = RZ0 * RY0 * nx4;
  for (int q = tid; q < n0; q += nthr) {
    const int x4 = q % nx4, r = q / nx4, yt = r % RY0, zt = r / RY0;
    const int k = k0 - 2 + zt;
    if (k < 0 || k >= nz) continue;
    const int j = ((j0 - 2 + yt) % ny + ny) % ny;
    cp_async16(P0 + q, Pg + ((size_t)k * ny + j) * nx4 + x4);
  }
  cp_async_wait_all();
  __syncthreads();
  // first sweep: levels k0-1 .. k0+TZ (inside the walls), rows j0-1 .. j0+TY
  for (int q = tid; q < n1; q += nthr) {
    const int x4 = q % nx4, r = q / nx4, yt = r % RY1, zt = r / RY1;
    const int k = k0 - 1 + zt;
    if (k < 0 || k >= nz) continue;
    const float4* row = P0 + ((zt + 1) * RY0 + (yt + 1)) * nx4;
    const float4 c = row[x4];
    const float left = reinterpret_cast<const float*>(row + (x4 == 0 ? nx4 - 1 : x4 - 1))[3];
    const float right = reinterpret_cast<const float*>(row + (x4 == nx4 - 1 ? 0 : x4 + 1))[0];
    const float4 yn = row[nx4 + x4], ys = row[x4 - nx4];
    const float4 zu = k < nz - 1 ? row[RY0 * nx4 + x4] : c;
    const float4 zd = k > 0 ? row[x4 - RY0 * nx4] : c;
    const float4 bq = B1[q];
    const float cup = __ldg(g.cup + k), cdn = __ldg(g.cdn + k), iS = __ldg(g.iS + k);
    float4 o;
    o.x = srj_cell_f32(c.x, left, c.y, yn.x, ys.x, zu.x, zd.x, bq.x, idx2, idy2, cup, cdn, iS, om_a);
    o.y = srj_cell_f32(c.y, c.x, c.z, yn.y, ys.y, zu.y, zd.y, bq.y, idx2, idy2, cup, cdn, iS, om_a);
    o.z = srj_cell_f32(c.z, c.y, c.w, yn.z, ys.z, zu.z, zd.z, bq.z, idx2, idy2, cup, cdn, iS, om_a);
    o.w = srj_cell_f32(c.w, c.z, right, yn.w, ys.w, zu.w, zd.w, bq.w, idx2, idy2, cup, cdn, iS, om_a);
    P1[q] = o;
  }
  __syncthreads();
  // second sweep: the tile itself
  const int n2 = TZ * TY * nx4;
  for (int q = tid; q < n2; q += nthr) {
    const int x4 = q % nx4, r = q / nx4, yt = r % TY, zt = r / TY;
    const int k = k0 + zt;
    const int i1 = ((zt + 1) * RY1 + (yt + 1)) * nx4;
    const float4* row = P1 + i1;
    const float4 c = row[x4];
    const float left = reinterpret_cast<const float*>(row + (x4 == 0 ? nx4 - 1 : x4 - 1))[3];
    const float right = reinterpret_cast<const float*>(row + (x4 == nx4 - 1 ? 0 : x4 + 1))[0];
    const float4 yn = row[nx4 + x4], ys = row[x4 - nx4];
    const float4 zu = k < nz - 1 ? row[RY1 * nx4 + x4] : c;
    const float4 zd = k > 0 ? row[x4 - RY1 * nx4] : c;
    const float4 bq = B1[i1 + x4];
    const float cup = __ldg(g.cup + k), cdn = __ldg(g.cdn + k), iS = __ldg(g.iS + k);
    float4 o;
    o.x = srj_cell_f32(c.x, left, c.y, yn.x, ys.x, zu.x, zd.x, bq.x, idx2, idy2, cup, cdn, iS, om_b);
    o.y = srj_cell_f32(c.y, c.x, c.z, yn.y, ys.y, zu.y, zd.y, bq.y, idx2, idy2, cup, cdn, iS, om_b);
    o.z = srj_cell_f32(c.z, c.y, c.w, yn.z, ys.z, zu.z, zd.z, bq.z, idx2, idy2, cup, cdn, iS, om_b);
    o.w = srj_cell_f32(c.w, c.z, right, yn.w, ys.w, zu.w, zd.w, bq.w, idx2, idy2, cup, cdn, iS, om_b);
    reinterpret_cast<float4*>(out)[((size_t)k * ny + j0 + yt) * nx4 + x4] = o;
  }
}

template <bool PDL>
__global__ void __launch_bounds__(kBX* kBY) k_sweep_f64_v2(Geom<double> g, const double* __restrict__ p,
                                                            const double* __restrict__ b, double omega,
                                                            double* __restrict__ out) {
  const int lane = threadIdx.x;
  const int nx = g.nx, ny = g.ny, nx2 = nx >> 1;
  const int x2 = blockIdx.x * kBX + lane;
  const int j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  const bool active = x2 < nx2 && j < ny;
  const int xx = x2 < nx2 ? x2 : nx2 - 1;
  const int jj = j < ny ? j : ny - 1;
  const int jp = jj == ny - 1 ? 0 : jj + 1, jm = jj == 0 ? ny - 1 : jj - 1;
  const size_t plane2 = (size_t)nx2 * ny;
  const size_t rc = ((size_t)k * ny + jj) * nx2;
  const double cup = __ldg(g.cup + k), cdn = __ldg(g.cdn + k), iS = __ldg(g.iS + k);
  const double idx2 = g.idx2, idy2 = g.idy2;
  const bool has_up = k < g.nz - 1, has_dn = k > 0;
  if (PDL) cudaGridDependencySynchronize();
  const double2* P = reinterpret_cast<const double2*>(p);
  const double2 c = __ldg(P + rc + xx);
  double left = __shfl_up_sync(0xffffffffu, c.y, 1);
  double right = __shfl_down_sync(0xffffffffu, c.x, 1);
  const double* prow = p + rc * 2;
  if (lane == 0 || xx == 0) left = __ldg(prow + (2 * xx - 1 + nx) % nx);
  if (lane == kBX - 1 || xx == nx2 - 1) right = __ldg(prow + (2 * xx + 2) % nx);
  const double2 yn = __ldg(P + ((size_t)k * ny + jp) * nx2 + xx);
  const double2 ys = __ldg(P + ((size_t)k * ny + jm) * nx2 + xx);
  const double2 zu = has_up ? __ldg(P + rc + plane2 + xx) : c;
  const double2 zd = has_dn ? __ldg(P + rc - plane2 + xx) : c;
  const double2 bq = __ldg(reinterpret_cast<const double2*>(b) + rc + xx);
  auto cell = [&](double pc, double xl, double xr, double nn, double ss, double uu, double dd, double bb) {
    const double nbs = idx2 * (xr + xl) + idy2 * (nn + ss) + cup * uu + cdn * dd;
    const double pj = (nbs - bb) * iS;
    return pc + omega * (pj - pc);
  };
  double2 o;
  o.x = cell(c.x, left, c.y, yn.x, ys.x, zu.x, zd.x, bq.x);
  o.y = cell(c.y, c.x, right, yn.y, ys.y, zu.y, zd.y, bq.y);
  if (active) reinterpret_cast<double2*>(out)[rc + x2] = o;
}

// ---------------------------------------------------------------------------
// One whole SRJ cycle in a single cooperative launch (FP32): the M sweeps
// ping-pong between A and B with a grid barrier between consecutive sweeps,
// so the cycle costs one launch instead of M.  The grid is exactly the
// co-resident size (cooperative launch guarantees co-residency).  p is read
// with L2-coherent loads (__ldcg): another SM wrote it in the previous
// sweep.  Work: warps take chunks of 32 consecutive float4 units (4 cells of
// a row each) in a grid-stride loop; a unit's x-neighbours come from the
// adjacent lanes when they hold the same row, else by a scalar load.
// Every barrier wait is bounded (ctl->bar_wait clock cycles, about one
// second by default); on time-out the kernel sets ctl->bad = 2 and returns,
// and the check kernels then end the solve.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool grid_barrier(GridBar bar, unsigned nblocks, long long wait) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* vgen = bar.gen;
    const unsigned g0 = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar.count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(bar.count, 0u);
      __threadfence();
      atomicAdd(bar.gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g0) {
        if (clock64() - t0 > wait) {
          atomicExch(bar.err, 1);
          break;
        }
      }
    }
    __threadfence();
    if (*(volatile int*)bar.err) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void __launch_bounds__(1024, 1) k_cycle_f32(Geom<float> g, float* A, float* B, const float* __restrict__ b,
                                                       const float* __restrict__ omega, int M, GridBar bar,
                                                       SolveCtl* ctl) {
  const int nx = g.nx, ny = g.ny, nx4 = nx >> 2;
  const long long nunits = (long long)nx4 * ny * g.nz;
  const long long nchunks = (nunits + 31) / 32;
  const int lane = threadIdx.x & 31;
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const size_t plane4 = (size_t)nx4 * ny;
  const float idx2 = g.idx2, idy2 = g.idy2;
  const long long wait = __ldcg(&ctl->bar_wait);
  for (int m = 0; m < M; m++) {
    const float* src = (m & 1) ? B : A;
    float* dst = (m & 1) ? A : B;
    const float om = __ldg(omega + m);
    const float4* P = reinterpret_cast<const float4*>(src);
    for (long long ch = warp0; ch < nchunks; ch += nwarps) {
      const long long u0 = ch * 32 + lane;
      const bool active = u0 < nunits;
      const long long u = active ? u0 : nunits - 1;
      const int x4 = (int)(u % nx4);
      const long long rr = u / nx4;
      const int j = (int)(rr % ny), k = (int)(rr / ny);
      const int jp = j == ny - 1 ? 0 : j + 1, jm = j == 0 ? ny - 1 : j - 1;
      const size_t rc = ((size_t)k * ny + j) * nx4;
      const float cup = __ldg(g.cup + k), cdn = __ldg(g.cdn + k), iS = __ldg(g.iS + k);
      const float4 c = __ldcg(P + rc + x4);
      float left = __shfl_up_sync(0xffffffffu, c.w, 1);
      float right = __shfl_down_sync(0xffffffffu, c.x, 1);
      const float* prow = src + rc * 4;
      if (lane == 0 || x4 == 0) left = __ldcg(prow + (4 * x4 - 1 + nx) % nx);
      if (lane == 31 || x4 == nx4 - 1) right = __ldcg(prow + (4 * x4 + 4) % nx);
      const float4 yn = __ldcg(P + ((size_t)k * ny + jp) * nx4 + x4);
      const float4 ys = __ldcg(P + ((size_t)k * ny + jm) * nx4 + x4);
      const float4 zu = k < g.nz - 1 ? __ldcg(P + rc + plane4 + x4) : c;
      const float4 zd = k > 0 ? __ldcg(P + rc - plane4 + x4) : c;
      const float4 bq = __ldg(reinterpret_cast<const float4*>(b) + rc + x4);
      auto cell = [&](float pc, float xl, float xr, float nn, float ss, float uu, float dd, float bb) {
        return srj_cell_f32(pc, xl, xr, nn, ss, uu, dd, bb, idx2, idy2, cup, cdn, iS, om);
      };
      float4 o;
      o.x = cell(c.x, left, c.y, yn.x, ys.x, zu.x, zd.x, bq.x);
      o.y = cell(c.y, c.x, c.z, yn.y, ys.y, zu.y, zd.y, bq.y);
      o.z = cell(c.z, c.y, c.w, yn.z, ys.z, zu.z, zd.z, bq.z);
      o.w = cell(c.w, c.z, right, yn.w, ys.w, zu.w, zd.w, bq.w);
      if (active) reinterpret_cast<float4*>(dst)[rc + x4] = o;
    }
    if (m + 1 < M && !grid_barrier(bar, gridDim.x, wait)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) ctl->bad = 2;
      return;
    }
  }
}

// z-line Jacobi-SOR sweep (line relaxation of Sec. 3.4's SRJ): for every
// column (i, j), r = b - L p (difference form, arithmetic in T), the column
// system A delta = r with A = -L_z + (2/dx^2 + 2/dy^2) I by the Thomas
// algorithm (pivots precomputed per level: li = 1/m_k, lu = cup_k/m_k), and
// p' = p - omega delta; since A (p^L - p) = -(b - L p), this is
// p + omega (p^L - p) for the line value p^L.  One thread per column,
// consecutive threads along x (coalesced rows); the forward elimination
// stores its values in out, the back substitution overwrites them with p'.
template <typename T>
__global__ void __launch_bounds__(128) k_line_sweep(Geom<T> g, const T* __restrict__ p, const T* __restrict__ b,
                                                    T omega, T* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  cudaGridDependencySynchronize();
  if (i >= nx) return;
  const unsigned plane = (unsigned)nx * ny;
  const unsigned c0 = (unsigned)j * nx + i;
  const unsigned xp = (unsigned)j * nx + (i == nx - 1 ? 0 : i + 1), xm = (unsigned)j * nx + (i == 0 ? nx - 1 : i - 1);
  const unsigned yp = (unsigned)(j == ny - 1 ? 0 : j + 1) * nx + i, ym = (unsigned)(j == 0 ? ny - 1 : j - 1) * nx + i;
  const T idx2 = g.idx2, idy2 = g.idy2;
  T pm = T(0), pc = __ldg(p + c0), dprev = T(0);
#pragma unroll 4
  for (int k = 0; k < nz; k++) {
    const unsigned lev = (unsigned)k * plane;
    const T pu = k < nz - 1 ? __ldg(p + lev + plane + c0) : pc;
    T lap = idx2 * ((__ldg(p + lev + xp) - pc) + (__ldg(p + lev + xm) - pc)) +
            idy2 * ((__ldg(p + lev + yp) - pc) + (__ldg(p + lev + ym) - pc));
    if (k < nz - 1) lap += __ldg(g.cup + k) * (pu - pc);
    if (k > 0) lap += __ldg(g.cdn + k) * (pm - pc);
    const T r = __ldg(b + lev + c0) - lap;
    const T d = (r + __ldg(g.cdn + k) * dprev) * __ldg(g.li + k);
    out[lev + c0] = d;
    dprev = d;
    pm = pc;
    pc = pu;
  }
  T dnext = T(0);
#pragma unroll 4
  for (int k = nz - 1; k >= 0; k--) {
    const unsigned q = (unsigned)k * plane + c0;
    const T delta = out[q] + __ldg(g.lu + k) * dnext;
    out[q] = __ldg(p + q) - omega * delta;
    dnext = delta;
  }
}

// One direction of the twisted elimination or substitution on a column in
// shared memory: x_k = R_k + c_k x_(previous k) for the n levels
// k = k0, k0 + S, k0 + 2S, ..., each x_k stored over R_k; x enters as the
// value before k0.  R points at level k0 of the column (levels C apart), c
// at coefficient k0.  S and C are compile-time, so every access is a
// register plus an immediate offset.  Whole batches of B levels (8 in FP32,
// 4 in FP64, to keep two blocks an SM) run without bounds tests, their
// loads one batch ahead of the dependent multiply-adds (never touching a
// level being stored); the last n mod B levels run one at a time.
template <typename T, int S, int C>
__device__ __forceinline__ void line_chain(T* R, const T* __restrict__ c, int n, T x) {
  constexpr int B = sizeof(T) == 8 ? 4 : 8;
  int q = 0;
  if (n >= B) {
    T r[B], cc[B];
#pragma unroll
    for (int e = 0; e < B; e++) {
      r[e] = R[e * S * C];
      cc[e] = __ldg(c + e * S);
    }
    for (; q + 2 * B <= n; q += B) {
      T rn[B], cn[B];
#pragma unroll
      for (int e = 0; e < B; e++) {
        rn[e] = R[(B + e) * S * C];
        cn[e] = __ldg(c + (B + e) * S);
      }
#pragma unroll
      for (int e = 0; e < B; e++) {
        x = r[e] + cc[e] * x;
        R[e * S * C] = x;
      }
#pragma unroll
      for (int e = 0; e < B; e++) {
        r[e] = rn[e];
        cc[e] = cn[e];
      }
      R += B * S * C;
      c += B * S;
    }
#pragma unroll
    for (int e = 0; e < B; e++) {
      x = r[e] + cc[e] * x;
      R[e * S * C] = x;
    }
    R += B * S * C;
    c += B * S;
    q += B;
  }
  for (; q < n; q++) {
    x = *R + __ldg(c) * x;
    *R = x;
    R += S * C;
    c += S;
  }
}

// Phase 2 of the shared-memory line sweeps: the column systems A delta = r
// by the twisted factorisation (Thomas elimination from both walls, meeting
// at level t = nz/2), with R_k holding r_k times the twisted 1/pivot on
// entry and delta_k on exit.  Threads [0, C) take the upper part of their
// column (levels below t), threads [C, 2C) the lower part (above t); both
// chains are nz/2 levels, half of one-sided Thomas.  Called by every thread
// of the block (it holds block barriers); needs 2C <= blockDim.x.
template <typename T, int C>
__device__ __forceinline__ void line_solve_twisted(const Geom<T>& g, T* R) {
  const int nz = g.nz, t = nz >> 1;
  const int th = threadIdx.x, cl = th % C;
  const bool top = th < C, work = th < 2 * C;
  if (work) {
    if (top)
      line_chain<T, 1, C>(R + cl, g.tlf, t, T(0));  // d_k, k = 0 .. t-1
    else
      line_chain<T, -1, C>(R + (nz - 1) * C + cl, g.tlf + nz - 1, nz - 1 - t, T(0));  // e_k, k = nz-1 .. t+1
  }
  __syncthreads();
  T xt = T(0);
  if (work) {
    xt = R[t * C + cl];
    if (t > 0) xt += __ldg(g.tlf + t) * R[(t - 1) * C + cl];
    if (t < nz - 1) xt += __ldg(g.tlb + t) * R[(t + 1) * C + cl];
  }
  __syncthreads();
  if (work) {
    if (top) {
      R[t * C + cl] = xt;
      line_chain<T, -1, C>(R + (t - 1) * C + cl, g.tlb + t - 1, t, xt);  // delta_k, k = t-1 .. 0
    } else {
      line_chain<T, 1, C>(R + (t + 1) * C + cl, g.tlb + t + 1, nz - 1 - t, xt);  // delta_k, k = t+1 .. nz-1
    }
  }
  __syncthreads();
}

// The same sweep with the column work staged in shared memory.  A block
// owns C = 32 rb columns (32 consecutive x cells of rb rows) over all z
// levels, and 512 threads.  Phase 1: every thread computes r = b - L p for
// its column on one chunk of the levels (C columns x 512/C chunks, all
// independent) into R[k][column].  Phase 2: 2C threads solve the columns
// in shared memory by the twisted factorisation (line_solve_twisted).
// Phase 3: every thread writes p - omega delta for its column and chunk.
// The residual of each cell is formed as in k_line_sweep; the column solve
// eliminates from both walls instead of from the bottom one.
template <typename T, int RB>
__global__ void __launch_bounds__(512) k_line_sweep_smem(Geom<T> g, const T* __restrict__ p,
                                                         const T* __restrict__ b, T omega, T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char line_sm[];
  T* R = reinterpret_cast<T*>(line_sm);  // [nz][C]
  constexpr int rb = RB, C = 32 * RB, nchunk = 512 / C;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int nxb = (nx + 31) / 32;
  const int i0 = (blockIdx.x % nxb) * 32, j0 = (blockIdx.x / nxb) * rb;
  const int col = threadIdx.x % C, chunk = threadIdx.x / C;
  const int i = i0 + (col & 31), j = j0 + (col >> 5);
  const bool act = i < nx && j < ny;
  const int ic = i < nx ? i : nx - 1, jc = j < ny ? j : ny - 1;  // in-bounds stand-ins for inactive columns
  const unsigned plane = (unsigned)nx * ny;
  const unsigned c0 = (unsigned)jc * nx + ic;
  const unsigned xp = (unsigned)jc * nx + (ic == nx - 1 ? 0 : ic + 1), xm = (unsigned)jc * nx + (ic == 0 ? nx - 1 : ic - 1);
  const unsigned yp = (unsigned)(jc == ny - 1 ? 0 : jc + 1) * nx + ic, ym = (unsigned)(jc == 0 ? ny - 1 : jc - 1) * nx + ic;
  const int k0 = chunk * nz / nchunk, k1 = (chunk + 1) * nz / nchunk;
  const T idx2 = g.idx2, idy2 = g.idy2;
  cudaGridDependencySynchronize();
#pragma unroll 4
  for (int k = k0; k < k1; k++) {
    const unsigned lev = (unsigned)k * plane;
    const T pc = __ldg(p + lev + c0);
    T lap = idx2 * ((__ldg(p + lev + xp) - pc) + (__ldg(p + lev + xm) - pc)) +
            idy2 * ((__ldg(p + lev + yp) - pc) + (__ldg(p + lev + ym) - pc));
    if (k < nz - 1) lap += __ldg(g.cup + k) * (__ldg(p + lev + plane + c0) - pc);
    if (k > 0) lap += __ldg(g.cdn + k) * (__ldg(p + lev - plane + c0) - pc);
    R[k * C + col] = (__ldg(b + lev + c0) - lap) * __ldg(g.tli + k);  // r_k / pivot_k
  }
  __syncthreads();
  line_solve_twisted<T, C>(g, R);
  if (act) {
#pragma unroll 4
    for (int k = k0; k < k1; k++) {
      const unsigned q = (unsigned)k * plane + c0;
      out[q] = __ldg(p + q) - omega * R[k * C + col];
    }
  }
}

// The shared-memory line sweep with phases 1 and 3 on vector units (float4
// in FP32, double2 in FP64) of VW consecutive x cells: a thread handles one
// unit of one row over a chunk of levels, with vector loads of the centre,
// y and z neighbours and b, and scalar loads of the two x neighbours just
// outside the unit.  For nx a multiple of the vector width (aligned
// vectors); the last 32-cell segment of a row may be partial, its units past
// the row end reading the row's last unit (in bounds) and storing nothing.
// Phase 2 and the arithmetic per cell are those of k_line_sweep_smem.
template <typename T>
struct VecOf;
template <>
struct VecOf<float> {
  using V = float4;
  static constexpr int W = 4;
  __device__ static float get(const float4& v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }
  __device__ static void set(float4& v, int e, float x) {
    if (e == 0) v.x = x; else if (e == 1) v.y = x; else if (e == 2) v.z = x; else v.w = x;
  }
};
template <>
struct VecOf<double> {
  using V = double2;
  static constexpr int W = 2;
  __device__ static double get(const double2& v, int e) { return e == 0 ? v.x : v.y; }
  __device__ static void set(double2& v, int e, double x) {
    if (e == 0) v.x = x; else v.y = x;
  }
};

// loads of p in the line sweeps: through the read-only path, or (COH) from
// L2, for data that other blocks of the same kernel write (the persistent
// cycle below)
template <bool COH, typename V>
__device__ __forceinline__ V ldp(const V* a) {
  if constexpr (COH) return __ldcg(a);
  else return __ldg(a);
}

// One tile of the vector line sweep: 32 RB columns (32 x cells of RB rows),
// tile number `tile` (x tiles fastest), all three phases.  R is the block's
// shared column array.  PDL: wait for the previous kernel after the index
// set-up.
template <typename T, int RB, bool COH, bool PDL>
__device__ __forceinline__ void line_vec_tile(const Geom<T>& g, const T* __restrict__ p, const T* __restrict__ b,
                                              T omega, T* __restrict__ out, int tile, T* R) {
  using VT = VecOf<T>;
  using V = typename VT::V;
  constexpr int W = VT::W, UPR = 32 / W;  // vector units per 32-cell row segment
  constexpr int rb = RB, C = 32 * RB, U = UPR * RB, nchunk = 512 / U;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int nxb = (nx + 31) / 32;
  const int i0 = (tile % nxb) * 32, j0 = (tile / nxb) * rb;
  const int unit = threadIdx.x % U, chunk = threadIdx.x / U;
  const int jr = unit / UPR, xu = unit % UPR;
  const int i = i0 + W * xu, j = j0 + jr;
  const bool act = i < nx && j < ny;
  const int ic = i < nx ? i : nx - W, jc = j < ny ? j : ny - 1;  // in-bounds stand-ins for inactive units
  const unsigned plane = (unsigned)nx * ny;
  const unsigned c0 = (unsigned)jc * nx + ic;  // first cell of the unit
  const unsigned yp = (unsigned)(jc == ny - 1 ? 0 : jc + 1) * nx + ic, ym = (unsigned)(jc == 0 ? ny - 1 : jc - 1) * nx + ic;
  const unsigned xl = (unsigned)jc * nx + (ic == 0 ? nx - 1 : ic - 1), xr = (unsigned)jc * nx + (ic + W == nx ? 0 : ic + W);
  const int k0 = chunk * nz / nchunk, k1 = (chunk + 1) * nz / nchunk;
  const int col = jr * 32 + W * xu;
  const T idx2 = g.idx2, idy2 = g.idy2;
  if (PDL) cudaGridDependencySynchronize();
  // the unit's own values at levels k - 1 and k ride along in registers
  // (zd, c): each level loads only level k + 1 of the unit
  V c = {}, zd = {};
  if (k0 < k1) {
    c = ldp<COH>(reinterpret_cast<const V*>(p + (unsigned)k0 * plane + c0));
    zd = k0 > 0 ? ldp<COH>(reinterpret_cast<const V*>(p + (unsigned)(k0 - 1) * plane + c0)) : c;
  }
#pragma unroll 2
  for (int k = k0; k < k1; k++) {
    const unsigned lev = (unsigned)k * plane;
    const V yn = ldp<COH>(reinterpret_cast<const V*>(p + lev + yp));
    const V ys = ldp<COH>(reinterpret_cast<const V*>(p + lev + ym));
    const V zu = k < nz - 1 ? ldp<COH>(reinterpret_cast<const V*>(p + lev + plane + c0)) : c;
    const V bq = __ldg(reinterpret_cast<const V*>(b + lev + c0));
    const T left = ldp<COH>(p + lev + xl), right = ldp<COH>(p + lev + xr);
    const T cup = __ldg(g.cup + k), cdn = __ldg(g.cdn + k), li = __ldg(g.tli + k);
    V o;
#pragma unroll
    for (int e = 0; e < W; e++) {
      const T pc = VT::get(c, e);
      const T xrv = e == W - 1 ? right : VT::get(c, e + 1);
      const T xlv = e == 0 ? left : VT::get(c, e - 1);
      T lap = idx2 * ((xrv - pc) + (xlv - pc)) + idy2 * ((VT::get(yn, e) - pc) + (VT::get(ys, e) - pc));
      if (k < nz - 1) lap += cup * (VT::get(zu, e) - pc);
      if (k > 0) lap += cdn * (VT::get(zd, e) - pc);
      VT::set(o, e, (VT::get(bq, e) - lap) * li);
    }
    *reinterpret_cast<V*>(R + k * C + col) = o;
    zd = c;
    c = zu;
  }
  __syncthreads();
  line_solve_twisted<T, C>(g, R);
  if (act) {
#pragma unroll 2
    for (int k = k0; k < k1; k++) {
      const unsigned q = (unsigned)k * plane + c0;
      const V pv = ldp<COH>(reinterpret_cast<const V*>(p + q));
      const V dv = *reinterpret_cast<const V*>(R + k * C + col);
      V o;
#pragma unroll
      for (int e = 0; e < W; e++) VT::set(o, e, VT::get(pv, e) - omega * VT::get(dv, e));
      *reinterpret_cast<V*>(out + q) = o;
    }
  }
}

template <typename T, int RB>
__global__ void __launch_bounds__(512) k_line_sweep_vec(Geom<T> g, const T* __restrict__ p, const T* __restrict__ b,
                                                        T omega, T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char line_sm[];
  line_vec_tile<T, RB, false, true>(g, p, b, omega, out, blockIdx.x, reinterpret_cast<T*>(line_sm));
}

// The FP32 z-line sweep with every column solved in registers, in level
// chunks (no shared-memory column array, no serial chain over the column).
// The twisted factorisation of A is two first-order linear recurrences per
// column:
//   elimination  y_k = g_k + f_k y_{k-1}  (k < t, from the bottom wall)
//                y_k = g_k + f_k y_{k+1}  (k > t, from the top wall),
//   twist        x_t = g_t + tlf_t y_{t-1} + tlb_t y_{t+1},
//   substitution x_k = y_k + e_k x_{k+1}  (k < t),  x_k = y_k + e_k x_{k-1}  (k > t),
// with g = r tli, f = tlf, e = tlb.  The levels below t are cut into NCH/2
// chunks, t and the levels above it into NCH/2 more (the first of them, the
// twist chunk, starts at t).  Each thread owns one float4 unit (4 x cells)
// of one chunk, holds its g_k in registers, and runs each recurrence inside
// its chunk from zero; the value entering the chunk (its carry) then adds
// in times the running product of the chunk's coefficients:
//   y_k = z_k + (prod of f over the chunk up to k) y_in.
// The carries come from the chunk boundary values in shared memory, walked
// from the wall (elimination) or from the twist level (substitution).  In
// exact arithmetic this is the sequential elimination; the rounding differs
// by a few units in the last place.
// Block: 32 x cells of one row (8 units) x NCH chunks, one tile per block.
// Requires nx a multiple of 32 and chunks of at most LMAX levels.
template <int NCH, int LMAX>
__global__ void __launch_bounds__(8 * NCH, 4) k_line_sweep_chunk(Geom<float> g, const float* __restrict__ p,
                                                                  const float* __restrict__ b, float omega,
                                                                  float* __restrict__ out) {
  constexpr int U = 8, H = NCH / 2;
  __shared__ float4 ZB[NCH][U];  // chunk boundary values of the elimination
  __shared__ float4 WB[NCH][U];  // and of the substitution
  __shared__ float4 XT[U];       // x_t
  __shared__ float FB[NCH], EB[NCH];  // the chunks' coefficient products
  const int nx = g.nx, ny = g.ny, nz = g.nz, t = nz >> 1;
  const int nxb = nx >> 5;
  const int i = (blockIdx.x % nxb) * 32 + 4 * (threadIdx.x % U), j = blockIdx.x / nxb;
  const int u = threadIdx.x % U, c = threadIdx.x / U;
  const unsigned plane = (unsigned)nx * ny;
  const unsigned c0 = (unsigned)j * nx + i;
  const unsigned yp = (unsigned)(j == ny - 1 ? 0 : j + 1) * nx + i, ym = (unsigned)(j == 0 ? ny - 1 : j - 1) * nx + i;
  const unsigned xl = (unsigned)j * nx + (i == 0 ? nx - 1 : i - 1), xr = (unsigned)j * nx + (i + 4 == nx ? 0 : i + 4);
  // level range [k0, k1) of chunk c: [0, t) cut evenly from below, [t, nz)
  // cut with the first piece (holding t) never empty
  const bool lower = c < H;
  const int k0 = lower ? c * t / H : t + ((c - H) * (nz - t) + H - 1) / H;
  const int k1 = lower ? (c + 1) * t / H : (c + 1 == NCH ? nz : t + ((c - H + 1) * (nz - t) + H - 1) / H);
  const int L = k1 - k0;
  const bool twist = c == H;
  const float idx2 = g.idx2, idy2 = g.idy2;
  using VT = VecOf<float>;
  float4 G[LMAX];
  cudaGridDependencySynchronize();
  // g_k = (b - L p)_k tli_k on the chunk's levels (the unit's z neighbours
  // ride along in registers)
  {
    float4 cc = {}, zd = {};
    if (L > 0) {
      cc = __ldg(reinterpret_cast<const float4*>(p + (unsigned)k0 * plane + c0));
      zd = k0 > 0 ? __ldg(reinterpret_cast<const float4*>(p + (unsigned)(k0 - 1) * plane + c0)) : cc;
    }
#pragma unroll
    for (int q = 0; q < LMAX; q++) {
      if (q < L) {
        const int k = k0 + q;
        const unsigned lev = (unsigned)k * plane;
        const float4 yn = __ldg(reinterpret_cast<const float4*>(p + lev + yp));
        const float4 ys = __ldg(reinterpret_cast<const float4*>(p + lev + ym));
        const float4 zu = k < nz - 1 ? __ldg(reinterpret_cast<const float4*>(p + lev + plane + c0)) : cc;
        const float4 bq = __ldg(reinterpret_cast<const float4*>(b + lev + c0));
        const float left = __ldg(p + lev + xl), right = __ldg(p + lev + xr);
        const float4 cf = __ldg(g.lz4 + k);  // cup, cdn, tli, tlf
        const float cup = cf.x, cdn = cf.y, li = cf.z;
        float4 o;
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const float pc = VT::get(cc, e);
          const float xrv = e == 3 ? right : VT::get(cc, e + 1);
          const float xlv = e == 0 ? left : VT::get(cc, e - 1);
          float lap = idx2 * ((xrv - pc) + (xlv - pc)) + idy2 * ((VT::get(yn, e) - pc) + (VT::get(ys, e) - pc));
          if (k < nz - 1) lap += cup * (VT::get(zu, e) - pc);
          if (k > 0) lap += cdn * (VT::get(zd, e) - pc);
          VT::set(o, e, (VT::get(bq, e) - lap) * li);
        }
        G[q] = o;
        zd = cc;
        cc = zu;
      }
    }
  }
  auto axpy = [](float a, const float4& x, const float4& y) {  // a x + y
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
  };
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  // elimination inside the chunk from zero (upward below t, downward above
  // it; the twist level itself is not eliminated)
  {
    float4 z = zero;
    float F = 1.f;
    if (lower) {
#pragma unroll
      for (int q = 0; q < LMAX; q++)
        if (q < L) {
          const float f = __ldg(g.lz4 + k0 + q).w;
          z = axpy(f, z, G[q]);
          F *= f;
          G[q] = z;
        }
    } else {
#pragma unroll
      for (int q = LMAX - 1; q >= 0; q--)
        if (q < L && (q > 0 || !twist)) {
          const float f = __ldg(g.lz4 + k0 + q).w;
          z = axpy(f, z, G[q]);
          F *= f;
          G[q] = z;
        }
    }
    ZB[c][u] = z;
    if (u == 0) FB[c] = F;
  }
  __syncthreads();
  // carries of the elimination from the walls; the twist value
  {
    float4 carry = zero;
    if (lower) {
      for (int cc = 0; cc < c; cc++) carry = axpy(FB[cc], carry, ZB[cc][u]);
      float F = 1.f;
#pragma unroll
      for (int q = 0; q < LMAX; q++)
        if (q < L) {
          F *= __ldg(g.lz4 + k0 + q).w;
          G[q] = axpy(F, carry, G[q]);
        }
    } else {
      for (int cc = NCH - 1; cc > c; cc--) carry = axpy(FB[cc], carry, ZB[cc][u]);
      float F = 1.f;
#pragma unroll
      for (int q = LMAX - 1; q >= 0; q--)
        if (q < L && (q > 0 || !twist)) {
          F *= __ldg(g.lz4 + k0 + q).w;
          G[q] = axpy(F, carry, G[q]);
        }
      if (twist) {
        float4 ylow = zero;  // y_{t-1}
        for (int cc = 0; cc < H; cc++) ylow = axpy(FB[cc], ylow, ZB[cc][u]);
        const float4 yup = L >= 2 ? G[1] : carry;  // y_{t+1}
        const float ft = t > 0 ? __ldg(g.lz4 + t).w : 0.f, et = t < nz - 1 ? __ldg(g.tlb + t) : 0.f;
        G[0] = axpy(et, yup, axpy(ft, ylow, G[0]));
      }
    }
  }
  // substitution inside the chunk from zero (downward below t, upward above
  // it); the twist chunk publishes x_t and its top value
  {
    float4 w = zero;
    float E = 1.f;
    if (lower) {
#pragma unroll
      for (int q = LMAX - 1; q >= 0; q--)
        if (q < L) {
          const float e = __ldg(g.tlb + k0 + q);
          w = axpy(e, w, G[q]);
          E *= e;
          G[q] = w;
        }
    } else {
#pragma unroll
      for (int q = 0; q < LMAX; q++)
        if (q < L && (q > 0 || !twist)) {
          const float e = __ldg(g.tlb + k0 + q);
          w = axpy(e, w, G[q]);
          E *= e;
          G[q] = w;
        }
      if (twist) {
        w = axpy(E, G[0], w);  // x at the chunk's top level, absolute
        E = 0.f;
        XT[u] = G[0];
      }
    }
    WB[c][u] = w;
    if (u == 0) EB[c] = E;
  }
  __syncthreads();
  // carries of the substitution from the twist level; the update
  {
    float4 carry = twist ? G[0] : XT[u];
    if (lower) {
      for (int cc = H - 1; cc > c; cc--) carry = axpy(EB[cc], carry, WB[cc][u]);
      float E = 1.f;
#pragma unroll
      for (int q = LMAX - 1; q >= 0; q--)
        if (q < L) {
          E *= __ldg(g.tlb + k0 + q);
          G[q] = axpy(E, carry, G[q]);
        }
    } else {
      for (int cc = H; cc < c; cc++) carry = axpy(EB[cc], carry, WB[cc][u]);
      float E = 1.f;
#pragma unroll
      for (int q = 0; q < LMAX; q++)
        if (q < L && (q > 0 || !twist)) {
          E *= __ldg(g.tlb + k0 + q);
          G[q] = axpy(E, carry, G[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < LMAX; q++)
      if (q < L) {
        const unsigned a = (unsigned)(k0 + q) * plane + c0;
        const float4 pv = __ldg(reinterpret_cast<const float4*>(p + a));
        *reinterpret_cast<float4*>(out + a) = axpy(-omega, G[q], pv);
      }
  }
}

__device__ __forceinline__ int ld_acquire(const int* a) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* a, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

// A whole SRJ cycle of M FP32 z-line sweeps (A -> B -> A ...) in one
// cooperative launch, one block per tile of the vector line sweep.
// Instead of a grid barrier between sweeps, a tile waits only for the four
// tiles whose cells its stencil reads (x and y neighbours, periodic) to
// have finished the previous sweep: flags[t] counts the sweeps tile t has
// completed (all tiles hold the same count between launches, so a launch
// reads its starting count from its own flag).  That also keeps a tile from
// overwriting cells a neighbour still reads: a neighbour reads this tile's
// cells of the buffer being overwritten during its previous sweep, which has
// ended.  p is read from L2 (other blocks write it within the launch).  Every
// wait is bounded by ctl->bar_wait clock cycles; on time-out the block sets
// ctl->bad = 2 and returns, and the blocks waiting on it time out in turn.
template <int RB>
__global__ void __launch_bounds__(512) k_line_cycle_f32(Geom<float> g, float* A, float* B, const float* __restrict__ b,
                                                        const float* __restrict__ omega, int M, int* flags,
                                                        SolveCtl* ctl) {
  extern __shared__ __align__(16) unsigned char line_sm[];
  float* R = reinterpret_cast<float*>(line_sm);
  __shared__ int s_ok;
  const int ntx = (g.nx + 31) / 32, nty = (g.ny + RB - 1) / RB;
  const int tile = blockIdx.x, tx = tile % ntx, ty = tile / ntx;
  const int nb0 = ty * ntx + (tx == 0 ? ntx - 1 : tx - 1), nb1 = ty * ntx + (tx == ntx - 1 ? 0 : tx + 1);
  const int nb2 = (ty == 0 ? nty - 1 : ty - 1) * ntx + tx, nb3 = (ty == nty - 1 ? 0 : ty + 1) * ntx + tx;
  const int base = ld_acquire(flags + tile) + __ldcg(&ctl->wait_skew);
  const long long wait = __ldcg(&ctl->bar_wait);
  for (int m = 0; m < M; m++) {
    if (m > 0) {
      if (threadIdx.x == 0) {
        int ok = 1;
        const long long t0 = clock64();
        const int need = base + m;
        while (ok && (ld_acquire(flags + nb0) < need || ld_acquire(flags + nb1) < need ||
                      ld_acquire(flags + nb2) < need || ld_acquire(flags + nb3) < need)) {
          if (clock64() - t0 > wait) ok = 0;
          else __nanosleep(32);
        }
        s_ok = ok;
      }
      __syncthreads();
      if (!s_ok) {
        if (threadIdx.x == 0) ctl->bad = 2;
        return;
      }
    }
    line_vec_tile<float, RB, true, false>(g, (m & 1) ? B : A, b, __ldg(omega + m), (m & 1) ? A : B, tile, R);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release(flags + tile, base - __ldcg(&ctl->wait_skew) + m + 1);
    }
  }
}

// arms the inner loop of a refinement pass and clears its correction
__global__ void k_pass_begin(float* __restrict__ d, size_t n, int graph, cudaGraphConditionalHandle h_loop) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
    d[q] = 0.f;
  if (graph && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h_loop, 1u);
}

// ||b - L p||_2 reduced in FP64, then the cycle decision in the last block.
// mode 0: FP64 solve (tol * ||b||); mode 1: FP32 inner solve of the
// refinement (target max(inner_tol ||r||, tol ||b|| / 2), stop on stall).
template <typename T, int MODE>
__global__ void __launch_bounds__(kBX* kBY) k_check(Geom<T> g, const T* __restrict__ p, const T* __restrict__ b,
                                                     SolveCtl* ctl, Red red, unsigned nblocks, int graph,
                                                     cudaGraphConditionalHandle h_loop,
                                                     cudaGraphConditionalHandle h_body) {
  __shared__ double sh[32];
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  double s = 0.0;
  if (sizeof(T) == sizeof(float)) {
    // FP32 inner solve: squares and warp sums in FP32, warp sums added in FP64
    float r2 = 0.f;
    if (i < g.nx && j < g.ny) {
      T pc;
      const float r = (float)point_residual(g, p, b, i, j, k, &pc);
      r2 = r * r;
    }
    s = block_sum_f32(r2, sh);
  } else {
    if (i < g.nx && j < g.ny) {
      T pc;
      const double r = (double)point_residual(g, p, b, i, j, k, &pc);
      s = r * r;
    }
    s = block_sum(s, sh);
  }
  if (publish_partial_tree(red, nblocks, s, 0.0, false)) {
    const double tot = final_sum(red.partial, nblocks, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      const bool go = cycle_decide<MODE>(ctl, red, sqrt(tot));
      if (graph) {
        cudaGraphSetConditional(h_loop, go ? 1u : 0u);
        cudaGraphSetConditional(h_body, go ? 1u : 0u);
      }
    }
  }
}

// Refinement residual: r = b - mean(b) - L p in FP64 (neighbour-sum form,
// point_residual_sum; the reduced volume mean of b, zero when b telescopes),
// stored in FP32 for the inner solve, its norm summed from the stored
// values; decides whether another refinement pass runs.
__global__ void __launch_bounds__(kBX* kBY) k_outer(Geom<double> g, const double* __restrict__ p,
                                                     const double* __restrict__ b, float* __restrict__ r32,
                                                     SolveCtl* ctl, Red red, unsigned nblocks, int after_pass,
                                                     int graph, cudaGraphConditionalHandle h_loop) {
  __shared__ double sh[32];
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  const double bmean = __ldcg(red.sc + SC_BMEAN);
  float r2 = 0.f;
  if (i < g.nx && j < g.ny) {
    const float r = (float)(point_residual_sum(g, p, b, i, j, k) - bmean);
    r32[(k * g.ny + j) * g.nx + i] = r;
    r2 = r * r;
  }
  double s = block_sum_f32(r2, sh);
  if (publish_partial_tree(red, nblocks, s, 0.0, false)) {
    const double tot = final_sum(red.partial, nblocks, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      const bool go = pass_decide(ctl, red, sqrt(tot), after_pass);
      if (graph) cudaGraphSetConditional(h_loop, go ? 1u : 0u);
    }
  }
}

__global__ void k_addcorr(double* __restrict__ p, const float* __restrict__ d, size_t n) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
    p[q] += (double)d[q];
}

__global__ void k_difference(const double* __restrict__ a, const double* __restrict__ b, float* __restrict__ out,
                             size_t n) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
    out[q] = (float)(a[q] - b[q]);
}

__global__ void k_begin(SolveCtl* ctl, int graph, cudaGraphConditionalHandle h_loop) {
  if (graph) cudaGraphSetConditional(h_loop, 1u);
  begin_solve_state(ctl);
}

__global__ void __launch_bounds__(kBX* kBY) k_laplacian(Geom<double> g, const double* __restrict__ p,
                                                         double* __restrict__ out) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const int nx = g.nx, plane = g.nx * g.ny;
  const int ip = i == nx - 1 ? 0 : i + 1, im = i == 0 ? nx - 1 : i - 1;
  const int jp = j == g.ny - 1 ? 0 : j + 1, jm = j == 0 ? g.ny - 1 : j - 1;
  const int row = k * plane, q = row + j * nx + i;
  const double pc = p[q];
  double lap = (p[row + j * nx + ip] - 2.0 * pc + p[row + j * nx + im]) * g.idx2 +
               (p[row + jp * nx + i] - 2.0 * pc + p[row + jm * nx + i]) * g.idy2;
  if (k < g.nz - 1) lap += g.cup[k] * (p[q + plane] - pc);
  if (k > 0) lap -= g.cdn[k] * (pc - p[q - plane]);
  out[q] = lap;
}

// ||a||_2 into sc[slot]
__global__ void k_norm(const double* __restrict__ a, size_t n, int slot, Red red, unsigned nblocks) {
  __shared__ double sh[32];
  double s = 0.0;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    const double x = a[q];
    s += x * x;
  }
  s = block_sum(s, sh);
  if (publish_partial(red, nblocks, s, 0.0, false)) {
    const double tot = final_sum(red.partial, nblocks, sh);
    if (threadIdx.x == 0) {
      red.sc[slot] = sqrt(tot);
      *red.counter = 0u;
    }
  }
}

// Volume sums of a cell-centred field: sc[SC_VSUM] = sum a dz_k and
// sc[SC_VABS] = sum |a| dz_k (dx dy is common to every cell and left out);
// one 32 x 8 tile a block, one level per grid row, fixed summation order.
__global__ void k_vsum(Geom<double> g, const double* __restrict__ a, Red red, unsigned nblocks) {
  __shared__ double sh[32];
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  double s = 0.0, m = 0.0;
  if (i < g.nx && j < g.ny) {
    const double x = a[(k * g.ny + j) * g.nx + i] * g.dzv[k];
    s = x;
    m = fabs(x);
  }
  s = block_sum(s, sh);
  m = block_sum(m, sh);
  if (publish_partial(red, nblocks, s, m, true)) {
    const double ts = final_sum(red.partial, nblocks, sh);
    const double tm = final_sum(red.partial + nblocks, nblocks, sh);
    if (threadIdx.x + blockDim.x * threadIdx.y == 0) {
      red.sc[SC_VSUM] = ts;
      red.sc[SC_VABS] = tm;
      *red.counter = 0u;
    }
  }
}

// a -= sc[SC_VSUM] / sum(dz) over the cells: zero volume-weighted mean
__global__ void k_sub_vmean(size_t n, double* __restrict__ a, double inv_lz_plane, Red red) {
  const double mean = __ldcg(red.sc + SC_VSUM) * inv_lz_plane;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
    a[q] -= mean;
}

}  // namespace

// Vector kernels when the row length allows aligned vectors (nx a multiple
// of 4 in FP32, of 2 in FP64), launched as programmatic dependents; the
// one-cell-per-thread kernels otherwise.
template <typename K, typename T>
static cudaError_t launch_pdl(K kern, dim3 grid, dim3 block, cudaStream_t s, const Geom<T>& g, const T* p,
                              const T* b, T omega, T* out) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, g, p, b, omega, out);
}

// FP32 sweep variant per host thread (poisson_common.cuh numbers them)
static thread_local int t_sweep_variant = 0;
void set_sweep_variant(int v) { t_sweep_variant = v; }
int sweep_variant_count() { return kSweepVariants; }
bool sweep_variant_ok(int v, int nx, int ny, int nz) {
  if (v < 0 || v >= kSweepVariants || nx % 4 || nz % sweep_kz(v)) return false;
  if (sweep_pair(v)) return ny % sweep_by(v) == 0 && pair_smem_bytes(sweep_by(v), sweep_kz(v), nx) <= kPairSmemMax;
  return !sweep_flat(v) || ((nx / 4) * ny) % 32 == 0;
}
bool sweep_variant_is_pair(int v) { return v >= 0 && v < kSweepVariants && sweep_pair(v); }

template <int TY, int TZ>
static cudaError_t launch_pair(const Geom<float>& g, const float* p, const float* b, float om_a, float om_b,
                               float* out, cudaStream_t s) {
  const size_t smem = pair_smem_bytes(TY, TZ, g.nx);
  {
    // the kernel's shared-memory limit, raised to the device's opt-in
    // maximum once a device
    static std::atomic<unsigned> done{0u};
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (smem > (size_t)optin) return cudaErrorInvalidConfiguration;
    e = smem_limit_once(k_sweep_f32_pair<TY, TZ>, optin, done);
    if (e != cudaSuccess) return e;
  }
  const dim3 grid(g.ny / TY, g.nz / TZ), block(256);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_sweep_f32_pair<TY, TZ>, g, p, b, om_a, om_b, out);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_sweep_pair(const Geom<float>& g, const float* p, const float* b, float om_a, float om_b,
                              float* out, cudaStream_t s) {
  const int v = sweep_variant_ok(t_sweep_variant, g.nx, g.ny, g.nz) ? t_sweep_variant : -1;
  switch (v) {
    case 9: return launch_pair<8, 4>(g, p, b, om_a, om_b, out, s);
    case 10: return launch_pair<4, 4>(g, p, b, om_a, om_b, out, s);
    case 11: return launch_pair<4, 8>(g, p, b, om_a, om_b, out, s);
    default: return cudaErrorInvalidValue;
  }
}

static cudaError_t launch_sweep_cfg(const void* kern, dim3 grid, dim3 block, cudaStream_t s, void** args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelExC(&cfg, kern, args);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int KZ>
static cudaError_t launch_flat(const Geom<float>& g, const float* p, const float* b, float omega, float* out,
                               cudaStream_t s) {
  const long long units = (long long)(g.nz / KZ) * (g.nx / 4) * g.ny;
  const dim3 grid((unsigned)((units + kBX * kBY - 1) / (kBX * kBY))), block(kBX, kBY, 1);
  Geom<float> gg = g;
  void* args[] = {&gg, &p, &b, &omega, &out};
  return launch_sweep_cfg((const void*)k_sweep_f32_flat<KZ>, grid, block, s, args);
}

template <int KZ, int BY>
static cudaError_t launch_z(const Geom<float>& g, const float* p, const float* b, float omega, float* out,
                            cudaStream_t s) {
  const dim3 grid((g.nx / 4 + kBX - 1) / kBX, (g.ny + BY - 1) / BY, g.nz / KZ), block(kBX, BY, 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_sweep_f32_z<KZ, BY>, g, p, b, omega, out);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <>
cudaError_t launch_sweep<float>(const Geom<float>& g, const float* p, const float* b, float omega, float* out,
                                cudaStream_t s) {
  if (g.nx % 4 == 0) {
    const int v = sweep_variant_ok(t_sweep_variant, g.nx, g.ny, g.nz) ? t_sweep_variant : 0;
    switch (v) {
      case 6: return launch_flat<2>(g, p, b, omega, out, s);
      case 7: return launch_flat<4>(g, p, b, omega, out, s);
      case 8: return launch_flat<8>(g, p, b, omega, out, s);
      case 1: return launch_z<2, 8>(g, p, b, omega, out, s);
      case 2: return launch_z<4, 8>(g, p, b, omega, out, s);
      case 3: return launch_z<2, 4>(g, p, b, omega, out, s);
      case 4: return launch_z<4, 4>(g, p, b, omega, out, s);
      case 5: return launch_z<8, 4>(g, p, b, omega, out, s);
      default: return launch_z<1, 8>(g, p, b, omega, out, s);
    }
  }
  Launch l = plane_launch(g.nx, g.ny, g.nz);
  k_sweep_f32<<<l.grid, l.block, 0, s>>>(g, p, b, omega, out);
  return cudaGetLastError();
}
template <>
cudaError_t launch_sweep<double>(const Geom<double>& g, const double* p, const double* b, double omega, double* out,
                                 cudaStream_t s) {
  if (g.nx % 2 == 0) {
    const dim3 grid((g.nx / 2 + kBX - 1) / kBX, (g.ny + kBY - 1) / kBY, g.nz), block(kBX, kBY, 1);
    cudaError_t e = launch_pdl(k_sweep_f64_v2<true>, grid, block, s, g, p, b, omega, out);
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  Launch l = plane_launch(g.nx, g.ny, g.nz);
  k_sweep_f64<<<l.grid, l.block, 0, s>>>(g, p, b, omega, out);
  return cudaGetLastError();
}

// rows per block of the shared-memory line sweep: 4, 2 or 1 (so that the
// 32 rb columns divide the 512 threads), the most whose columns x nz values
// fit in 96 KB (two blocks an SM); 0 when one row does not fit
static int line_rows(int nz, size_t es) {
  const size_t per_row = 32 * (size_t)nz * es;
  for (int rb = 4; rb >= 1; rb /= 2)
    if (rb * per_row <= 96 * 1024) return rb;
  return 0;
}

// the shared-memory line sweeps at RB rows per block (the vector kernel when
// rows hold whole vectors); raises their shared-memory limit once a device
template <typename T, int RB>
static cudaError_t launch_line_rows(const Geom<T>& g, const T* p, const T* b, T omega, T* out, cudaStream_t s,
                                    cudaLaunchAttribute* attr) {
  static std::atomic<unsigned> done_smem{0u}, done_vec{0u};
  cudaError_t e0 = smem_limit_once(k_line_sweep_smem<T, RB>, 96 * 1024, done_smem);
  if (e0 == cudaSuccess) e0 = smem_limit_once(k_line_sweep_vec<T, RB>, 96 * 1024, done_vec);
  if (e0 != cudaSuccess) return e0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(((g.nx + 31) / 32) * ((g.ny + RB - 1) / RB)));
  cfg.blockDim = dim3(512);
  cfg.dynamicSmemBytes = (size_t)32 * RB * g.nz * sizeof(T);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = g.nx % VecOf<T>::W == 0 ? cudaLaunchKernelEx(&cfg, k_line_sweep_vec<T, RB>, g, p, b, omega, out)
                                          : cudaLaunchKernelEx(&cfg, k_line_sweep_smem<T, RB>, g, p, b, omega, out);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// levels a chunk of the register-chunked line sweep holds at most, and the
// chunks a column: columns of up to 2 x 16 x 6 = 192 levels
constexpr int kLineChunks = 32, kLineChunkLevels = 6;

bool line_chunk_ok(int nx, int nz) {
  constexpr int H = kLineChunks / 2;
  const int t = nz / 2;
  return nx % 32 == 0 && nz >= 2 && (t + H - 1) / H <= kLineChunkLevels &&
         (nz - t + H - 1) / H <= kLineChunkLevels;
}

template <typename T>
cudaError_t launch_line_sweep(const Geom<T>& g, const T* p, const T* b, T omega, T* out, cudaStream_t s,
                              int variant) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  if constexpr (sizeof(T) == 4) {
    if (variant == 1 && line_chunk_ok(g.nx, g.nz)) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)((g.nx / 32) * g.ny));
      cfg.blockDim = dim3(8 * kLineChunks);
      cfg.stream = s;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      cudaError_t e = cudaLaunchKernelEx(&cfg, k_line_sweep_chunk<kLineChunks, kLineChunkLevels>, g, p, b, omega, out);
      return e != cudaSuccess ? e : cudaGetLastError();
    }
  }
  switch (line_rows(g.nz, sizeof(T))) {
    case 4: return launch_line_rows<T, 4>(g, p, b, omega, out, s, attr);
    case 2: return launch_line_rows<T, 2>(g, p, b, omega, out, s, attr);
    case 1: return launch_line_rows<T, 1>(g, p, b, omega, out, s, attr);
    default: break;
  }
  const dim3 grid((g.nx + 127) / 128, g.ny), block(128);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_line_sweep<T>, g, p, b, omega, out);
  return e != cudaSuccess ? e : cudaGetLastError();
}
template cudaError_t launch_line_sweep<float>(const Geom<float>&, const float*, const float*, float, float*,
                                              cudaStream_t, int);
template cudaError_t launch_line_sweep<double>(const Geom<double>&, const double*, const double*, double, double*,
                                               cudaStream_t, int);

// Persistent z-line cycles (FP32, vector kernel): the rows per tile of the
// line sweep, and 0 when the grid does not take them (rows not a multiple
// of 4 cells, columns too tall for shared memory, or more tiles than can be
// resident at once)
int line_cycle_rows(const Geom<float>& g, int device) {
  if (g.nx % 4) return 0;
  const int rb = line_rows(g.nz, sizeof(float));
  if (rb == 0) return 0;
  const int tiles = ((g.nx + 31) / 32) * ((g.ny + rb - 1) / rb);
  const size_t smem = (size_t)32 * rb * g.nz * sizeof(float);
  int per_sm = 0, sms = 0;
  cudaError_t e;
  switch (rb) {
    case 4:
      e = cudaFuncSetAttribute(k_line_cycle_f32<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_line_cycle_f32<4>, 512, smem);
      break;
    case 2:
      e = cudaFuncSetAttribute(k_line_cycle_f32<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_line_cycle_f32<2>, 512, smem);
      break;
    default:
      e = cudaFuncSetAttribute(k_line_cycle_f32<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_line_cycle_f32<1>, 512, smem);
  }
  if (e != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  return tiles <= per_sm * sms ? rb : 0;
}

int line_cycle_tiles(const Geom<float>& g, int rb) { return ((g.nx + 31) / 32) * ((g.ny + rb - 1) / rb); }

cudaError_t launch_line_cycle_f32(const Geom<float>& g, int rb, float* A, float* B, const float* b,
                                  const float* omega, int M, int* flags, SolveCtl* ctl, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)line_cycle_tiles(g, rb));
  cfg.blockDim = dim3(512);
  cfg.dynamicSmemBytes = (size_t)32 * rb * g.nz * sizeof(float);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e;
  switch (rb) {
    case 4: e = cudaLaunchKernelEx(&cfg, k_line_cycle_f32<4>, g, A, B, b, omega, M, flags, ctl); break;
    case 2: e = cudaLaunchKernelEx(&cfg, k_line_cycle_f32<2>, g, A, B, b, omega, M, flags, ctl); break;
    default: e = cudaLaunchKernelEx(&cfg, k_line_cycle_f32<1>, g, A, B, b, omega, M, flags, ctl);
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

int cycle_grid_f32(int device) {
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cycle_f32, 1024, 0) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  return per_sm * sms;
}

cudaError_t launch_cycle_f32(const Geom<float>& g, float* A, float* B, const float* b, const float* omega, int M,
                             GridBar bar, SolveCtl* ctl, int nblocks, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nblocks);
  cfg.blockDim = dim3(1024);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_cycle_f32, g, A, B, b, omega, M, bar, ctl);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_pass_begin(float* d, size_t n, int graph, cudaGraphConditionalHandle h_loop, cudaStream_t s) {
  unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16);
  k_pass_begin<<<blocks ? blocks : 1, 256, 0, s>>>(d, n, graph, h_loop);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_check(const Geom<T>& g, const T* p, const T* b, int mode, SolveCtl* ctl, Red red, int graph,
                         cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_body, cudaStream_t s) {
  Launch l = plane_launch(g.nx, g.ny, g.nz);
  if (mode == 0)
    k_check<T, 0><<<l.grid, l.block, 0, s>>>(g, p, b, ctl, red, l.nblocks, graph, h_loop, h_body);
  else
    k_check<T, 1><<<l.grid, l.block, 0, s>>>(g, p, b, ctl, red, l.nblocks, graph, h_loop, h_body);
  return cudaGetLastError();
}

cudaError_t launch_outer(const Geom<double>& g, const double* p, const double* b, float* r32, SolveCtl* ctl, Red red,
                         int after_pass, int graph, cudaGraphConditionalHandle h_loop, cudaStream_t s) {
  Launch l = plane_launch(g.nx, g.ny, g.nz);
  k_outer<<<l.grid, l.block, 0, s>>>(g, p, b, r32, ctl, red, l.nblocks, after_pass, graph, h_loop);
  return cudaGetLastError();
}

cudaError_t launch_addcorr(double* p, const float* d, size_t n, cudaStream_t s) {
  unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16);
  k_addcorr<<<blocks ? blocks : 1, 256, 0, s>>>(p, d, n);
  return cudaGetLastError();
}

cudaError_t launch_difference(const double* a, const double* b, float* out, size_t n, cudaStream_t s) {
  unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16);
  k_difference<<<blocks ? blocks : 1, 256, 0, s>>>(a, b, out, n);
  return cudaGetLastError();
}

cudaError_t launch_begin(SolveCtl* ctl, int graph, cudaGraphConditionalHandle h_loop, cudaStream_t s) {
  k_begin<<<1, 1, 0, s>>>(ctl, graph, h_loop);
  return cudaGetLastError();
}

cudaError_t launch_laplacian(const Geom<double>& g, const double* p, double* out, cudaStream_t s) {
  Launch l = plane_launch(g.nx, g.ny, g.nz);
  k_laplacian<<<l.grid, l.block, 0, s>>>(g, p, out);
  return cudaGetLastError();
}

cudaError_t launch_norm(const double* a, size_t n, int slot, Red red, cudaStream_t s) {
  unsigned blocks = (unsigned)((n + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks == 0) blocks = 1;
  k_norm<<<blocks, 256, 0, s>>>(a, n, slot, red, blocks);
  return cudaGetLastError();
}

cudaError_t launch_vsum(const Geom<double>& g, const double* a, Red red, cudaStream_t s) {
  Launch l = plane_launch(g.nx, g.ny, g.nz);
  k_vsum<<<l.grid, l.block, 0, s>>>(g, a, red, l.nblocks);
  return cudaGetLastError();
}

cudaError_t launch_sub_vmean(const Geom<double>& g, double* a, double Lz, Red red, cudaStream_t s) {
  const size_t n = (size_t)g.nx * g.ny * g.nz;
  unsigned blocks = (unsigned)((n + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_sub_vmean<<<blocks, 256, 0, s>>>(n, a, 1.0 / (Lz * g.nx * g.ny), red);
  return cudaGetLastError();
}

template cudaError_t launch_check<double>(const Geom<double>&, const double*, const double*, int, SolveCtl*, Red,
                                          int, cudaGraphConditionalHandle, cudaGraphConditionalHandle, cudaStream_t);
template cudaError_t launch_check<float>(const Geom<float>&, const float*, const float*, int, SolveCtl*, Red, int,
                                         cudaGraphConditionalHandle, cudaGraphConditionalHandle, cudaStream_t);

}  // namespace stp
