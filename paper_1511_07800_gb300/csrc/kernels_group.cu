// Grouped FP32 pressure solves of the batched step (Sec. 3.4 SRJ with the
// FP64 iterative refinement of the FP32 path).
//
// A group is a set of channels that share the SRJ cycle length M.  Each
// kernel below covers the tiles of every channel of the group in one
// launch: the channels' tiles are numbered one after the other, and a block
// finds its channel by a binary search over the channels' first tiles.  The
// solve runs in lock step under the same graph loops as a single channel's
// (WHILE over refinement passes { arm; WHILE over cycles { check; IF { M
// sweeps } }; p += d; outer residual }), with per-channel flags: a channel
// whose inner loop or whose pass loop has stopped skips its tiles.  Every
// channel keeps its own schedule, reductions (in its own block order) and
// decisions (the functions of poisson_common.cuh), so it ends bitwise where
// its own solve ends.  In each deciding kernel the channel that decides
// last sets the graph conditionals: a loop runs while any channel continues.
#include <algorithm>

#include "device_util.cuh"
#include "poisson_common.cuh"
#include "stp_internal.cuh"

namespace stp {

namespace {

// channel c with off[c] <= blk < off[c+1] (off[0] = 0, off[n] = all tiles)
__device__ __forceinline__ int group_chan(const int* __restrict__ off, int n, int blk) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= blk)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Publish this block's partial at its position bl in the channel's block
// order; true in every thread of the channel's last block to arrive.
__device__ __forceinline__ bool publish_local(const Red& red, unsigned nblocks, unsigned bl, double a) {
  __shared__ bool last;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    red.partial[bl] = a;
    __threadfence();
    const unsigned t = atomicAdd(red.counter, 1u);
    last = (t == nblocks - 1);
  }
  __syncthreads();
  return last;
}

// One channel's decision enters the group's: the last of the *part
// channels taking part in this kernel sets the conditional(s) to "any
// continues", stores the number continuing in *part and counts the kernels
// the group ran.  *part is read before arriving: it changes only after the
// last arrival.
__device__ __forceinline__ void group_arrive(GState* gs, unsigned* part, bool go, long long kern_go,
                                             long long kern_stop, cudaGraphConditionalHandle h1,
                                             cudaGraphConditionalHandle h2, bool two) {
  const unsigned P = *(volatile unsigned*)part;
  if (go) atomicAdd(&gs->n_go, 1u);
  __threadfence();
  const unsigned t = atomicAdd(&gs->arrived, 1u);
  if (t + 1 == P) {
    __threadfence();
    const unsigned tot = atomicExch(&gs->n_go, 0u);
    gs->arrived = 0u;
    *part = tot;
    gs->kernels += tot ? kern_go : kern_stop;
    cudaGraphSetConditional(h1, tot ? 1u : 0u);
    if (two) cudaGraphSetConditional(h2, tot ? 1u : 0u);
  }
}

// cell of this thread in local one-level tile t of an nx x ny channel
__device__ __forceinline__ void scalar_cell(int t, int nx, int ny, int* i, int* j, int* k) {
  const int gx = (nx + kBX - 1) / kBX, gy = (ny + kBY - 1) / kBY;
  *i = (t % gx) * kBX + threadIdx.x;
  *j = ((t / gx) % gy) * kBY + threadIdx.y;
  *k = t / (gx * gy);
}

__global__ void kg_begin(Group G) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < G.n) {
    begin_solve_state(G.ch[c].ctl);
    G.pass_on[c] = 1;
    G.inner_on[c] = 0;
  }
  if (c == 0) {
    G.gs->part_pass = (unsigned)G.n;
    G.gs->part_inner = 0u;
    G.gs->arrived = 0u;
    G.gs->n_go = 0u;
    G.gs->kernels += 1;
  }
}

// refinement residual r = b - mean(b) - L p (FP64, stored FP32; as k_outer) and the pass decision
__global__ void __launch_bounds__(kBX* kBY) kg_outer(Group G, int after_pass, cudaGraphConditionalHandle h_pass) {
  __shared__ double sh[32];
  const int c = group_chan(G.soff, G.n, blockIdx.x);
  if (!G.pass_on[c]) return;
  const GChan& C = G.ch[c];
  const Geom<double>& g = C.g64;
  const int nx = g.nx, ny = g.ny;
  const int t = blockIdx.x - __ldg(G.soff + c);
  int i, j, k;
  scalar_cell(t, nx, ny, &i, &j, &k);
  const double bmean = __ldcg(C.red.sc + SC_BMEAN);
  float r2 = 0.f;
  if (i < nx && j < ny) {
    const float r = (float)(point_residual_sum(g, C.p, C.b, i, j, k) - bmean);
    C.r32[(k * ny + j) * nx + i] = r;
    r2 = r * r;
  }
  double s = block_sum_f32(r2, sh);
  const unsigned nb = (unsigned)(__ldg(G.soff + c + 1) - __ldg(G.soff + c));
  if (publish_local(C.red, nb, (unsigned)t, s)) {
    const double tot = final_sum(C.red.partial, nb, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      const bool go = pass_decide(C.ctl, C.red, sqrt(tot), after_pass);
      G.pass_on[c] = go ? 1 : 0;
      group_arrive(G.gs, &G.gs->part_pass, go, 1 + after_pass, 1 + after_pass, h_pass, h_pass, false);
    }
  }
}

// start of a refinement pass: d = 0 and the inner loop armed for every
// channel in the pass
__global__ void __launch_bounds__(kBX* kBY) kg_pass_begin(Group G, cudaGraphConditionalHandle h_loop) {
  if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
    const unsigned P = G.gs->part_pass;
    G.gs->part_inner = P;
    G.gs->kernels += 1;
    cudaGraphSetConditional(h_loop, P ? 1u : 0u);
  }
  const int c = group_chan(G.soff, G.n, blockIdx.x);
  if (!G.pass_on[c]) return;
  const GChan& C = G.ch[c];
  const int nx = C.g32.nx, ny = C.g32.ny;
  const int t = blockIdx.x - __ldg(G.soff + c);
  int i, j, k;
  scalar_cell(t, nx, ny, &i, &j, &k);
  if (i < nx && j < ny) C.d1[(k * ny + j) * nx + i] = 0.f;
  if (t == 0 && threadIdx.x == 0 && threadIdx.y == 0) G.inner_on[c] = 1;
}

// ||r - L d|| of the cycle's input (FP32 arithmetic, FP64 sum) and the
// cycle decision
__global__ void __launch_bounds__(kBX* kBY) kg_check(Group G, cudaGraphConditionalHandle h_loop,
                                                      cudaGraphConditionalHandle h_body) {
  __shared__ double sh[32];
  const int c = group_chan(G.soff, G.n, blockIdx.x);
  if (!G.inner_on[c]) return;
  const GChan& C = G.ch[c];
  const Geom<float>& g = C.g32;
  const int nx = g.nx, ny = g.ny;
  const int t = blockIdx.x - __ldg(G.soff + c);
  int i, j, k;
  scalar_cell(t, nx, ny, &i, &j, &k);
  float r2 = 0.f;
  if (i < nx && j < ny) {
    float pc;
    const float r = point_residual(g, C.d1, C.r32, i, j, k, &pc);
    r2 = r * r;
  }
  double s = block_sum_f32(r2, sh);
  const unsigned nb = (unsigned)(__ldg(G.soff + c + 1) - __ldg(G.soff + c));
  if (publish_local(C.red, nb, (unsigned)t, s)) {
    const double tot = final_sum(C.red.partial, nb, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      const bool go = cycle_decide<1>(C.ctl, C.red, sqrt(tot));
      G.inner_on[c] = go ? 1 : 0;
      group_arrive(G.gs, &G.gs->part_inner, go, 1 + G.M, 1, h_loop, h_body, true);
    }
  }
}

// sweep m of the cycle for every channel still in its inner loop
// (d1 -> d2 for even m, d2 -> d1 for odd m, the channel's own omega_m)
template <int KZ, int BY>
__global__ void __launch_bounds__(kBX* BY) kg_sweep(Group G, int m) {
  const int c = group_chan(G.voff, G.n, blockIdx.x);
  if (!G.inner_on[c]) return;  // set before the cycle began, not by the sweeps
  const GChan& C = G.ch[c];
  const int nx4 = C.g32.nx >> 2, ny = C.g32.ny;
  const int gx = (nx4 + kBX - 1) / kBX, gy = (ny + BY - 1) / BY;
  const int t = blockIdx.x - __ldg(G.voff + c);
  const float* src = (m & 1) ? C.d2 : C.d1;
  float* dst = (m & 1) ? C.d1 : C.d2;
  sweep_z_tile<KZ, BY>(C.g32, src, C.r32, __ldg(C.omega + m), dst, t % gx, (t / gx) % gy, t / (gx * gy));
}

template <int KZ>
__global__ void __launch_bounds__(kBX* kBY) kg_sweep_flat(Group G, int m) {
  const int c = group_chan(G.voff, G.n, blockIdx.x);
  if (!G.inner_on[c]) return;
  const GChan& C = G.ch[c];
  const float* src = (m & 1) ? C.d2 : C.d1;
  float* dst = (m & 1) ? C.d1 : C.d2;
  sweep_flat_tile<KZ>(C.g32, src, C.r32, __ldg(C.omega + m), dst, blockIdx.x - __ldg(G.voff + c));
}

// p += d for every channel in the pass
__global__ void __launch_bounds__(kBX* kBY) kg_addcorr(Group G) {
  const int c = group_chan(G.soff, G.n, blockIdx.x);
  if (!G.pass_on[c]) return;
  const GChan& C = G.ch[c];
  const int nx = C.g32.nx, ny = C.g32.ny;
  const int t = blockIdx.x - __ldg(G.soff + c);
  int i, j, k;
  scalar_cell(t, nx, ny, &i, &j, &k);
  if (i < nx && j < ny) {
    const size_t q = ((size_t)k * ny + j) * nx + i;
    C.p[q] += (double)C.d1[q];
  }
}

template <int KZ, int BY>
cudaError_t launch_gs(const Group& G, int m, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)G.vtiles);
  cfg.blockDim = dim3(kBX, BY, 1);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kg_sweep<KZ, BY>, G, m);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int KZ>
cudaError_t launch_gf(const Group& G, int m, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)G.vtiles);
  cfg.blockDim = dim3(kBX, kBY, 1);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kg_sweep_flat<KZ>, G, m);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

int group_scalar_tiles(int nx, int ny, int nz) { return ((nx + kBX - 1) / kBX) * ((ny + kBY - 1) / kBY) * nz; }

int group_sweep_tiles(int variant, int nx, int ny, int nz) {
  if (!sweep_variant_ok(variant, nx, ny, nz) || sweep_pair(variant)) return -1;
  const int kz = sweep_kz(variant), nx4 = nx / 4;
  if (sweep_flat(variant)) return ((nz / kz) * nx4 * ny + kBX * kBY - 1) / (kBX * kBY);
  const int by = sweep_by(variant);
  return ((nx4 + kBX - 1) / kBX) * ((ny + by - 1) / by) * (nz / kz);
}

cudaError_t launch_group_begin(const Group& G, cudaStream_t s) {
  kg_begin<<<(G.n + 127) / 128, 128, 0, s>>>(G);
  return cudaGetLastError();
}

cudaError_t launch_group_outer(const Group& G, int after_pass, cudaGraphConditionalHandle h_pass, cudaStream_t s) {
  kg_outer<<<(unsigned)G.stiles, dim3(kBX, kBY), 0, s>>>(G, after_pass, h_pass);
  return cudaGetLastError();
}

cudaError_t launch_group_pass_begin(const Group& G, cudaGraphConditionalHandle h_loop, cudaStream_t s) {
  kg_pass_begin<<<(unsigned)G.stiles, dim3(kBX, kBY), 0, s>>>(G, h_loop);
  return cudaGetLastError();
}

cudaError_t launch_group_check(const Group& G, cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_body,
                               cudaStream_t s) {
  kg_check<<<(unsigned)G.stiles, dim3(kBX, kBY), 0, s>>>(G, h_loop, h_body);
  return cudaGetLastError();
}

cudaError_t launch_group_addcorr(const Group& G, cudaStream_t s) {
  kg_addcorr<<<(unsigned)G.stiles, dim3(kBX, kBY), 0, s>>>(G);
  return cudaGetLastError();
}

cudaError_t launch_group_sweep(const Group& G, int m, cudaStream_t s) {
  switch (G.variant) {
    case 1: return launch_gs<2, 8>(G, m, s);
    case 2: return launch_gs<4, 8>(G, m, s);
    case 3: return launch_gs<2, 4>(G, m, s);
    case 4: return launch_gs<4, 4>(G, m, s);
    case 5: return launch_gs<8, 4>(G, m, s);
    case 6: return launch_gf<2>(G, m, s);
    case 7: return launch_gf<4>(G, m, s);
    case 8: return launch_gf<8>(G, m, s);
    default: return launch_gs<1, 8>(G, m, s);
  }
}

}  // namespace stp
