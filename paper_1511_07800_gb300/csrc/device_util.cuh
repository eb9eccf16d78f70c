// Device helpers shared by the kernels: indexing on the periodic x-y plane,
// the wall ghosts, and the deterministic block / grid reductions.
#pragma once

#include <cuda_runtime.h>

#include "stp_internal.cuh"

namespace stp {

constexpr int kBX = 32;  // threads along x (one warp: coalesced rows)
constexpr int kBY = 8;   // threads along y

__host__ inline Launch plane_launch(int nx, int ny, int nlev) {
  Launch l;
  l.block = dim3(kBX, kBY, 1);
  l.grid = dim3((nx + kBX - 1) / kBX, (ny + kBY - 1) / kBY, nlev);
  l.nblocks = l.grid.x * l.grid.y * l.grid.z;
  return l;
}

// Index of (i, j, k) in an x-fastest array with ny rows of nx.
__device__ __forceinline__ int at(int nx, int ny, int i, int j, int k) { return (k * ny + j) * nx + i; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum (and max) over the block; result valid in thread 0.  Fixed tree order.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  v = warp_sum(v);
  __syncthreads();
  if ((tid & 31) == 0) sh[tid >> 5] = v;
  __syncthreads();
  if (tid < 32) {
    v = (tid < (nthr >> 5)) ? sh[tid] : 0.0;
    v = warp_sum(v);
  }
  return v;
}
__device__ __forceinline__ double block_max(double v, double* sh) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  v = warp_max(v);
  __syncthreads();
  if ((tid & 31) == 0) sh[tid >> 5] = v;
  __syncthreads();
  if (tid < 32) {
    v = (tid < (nthr >> 5)) ? sh[tid] : 0.0;
    v = warp_max(v);
  }
  return v;
}

__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max_f32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum over the block of FP32 values: each warp sums its 32 values in FP32
// (relative error about 2e-6), the warp sums are added in FP64 in a fixed
// order.  Valid in thread 0.  On GB300 a per-thread FP64 warp reduction
// costs as much as a whole FP32 stencil, so the kernels whose per-cell
// values are FP32 reduce this way.
__device__ __forceinline__ double block_sum_f32(float v, double* sh) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  v = warp_sum_f32(v);
  __syncthreads();
  if ((tid & 31) == 0) sh[tid >> 5] = (double)v;
  __syncthreads();
  double d = 0.0;
  if (tid < 32) {
    d = (tid < (nthr >> 5)) ? sh[tid] : 0.0;
    d = warp_sum(d);
  }
  return d;
}
__device__ __forceinline__ double block_max_f32(float v, double* sh) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  v = warp_max_f32(v);
  __syncthreads();
  if ((tid & 31) == 0) sh[tid >> 5] = (double)v;
  __syncthreads();
  double d = 0.0;
  if (tid < 32) {
    d = (tid < (nthr >> 5)) ? sh[tid] : 0.0;
    d = warp_max(d);
  }
  return d;
}

__device__ __forceinline__ unsigned block_linear() {
  return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}

// Publish this block's partial(s); returns true in every thread of the last
// block to arrive, which then owns the final reduction.
__device__ __forceinline__ bool publish_partial(Red red, unsigned nblocks, double a, double b, bool two) {
  __shared__ bool last;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  if (tid == 0) {
    const unsigned bl = block_linear();
    red.partial[bl] = a;
    if (two) red.partial[nblocks + bl] = b;
    __threadfence();
    const unsigned t = atomicAdd(red.counter, 1u);
    last = (t == nblocks - 1);
  }
  __syncthreads();
  return last;
}

// The same with arrivals counted in two levels: blocks arrive on the
// counter of their group of 64 (red.gcount), the last of each group on
// red.counter.  With one counter, tens of thousands of blocks (one a 32 x 8
// tile and level) serialise on one address while the rest of each block
// waits at its barrier; here at most 64 arrivals meet on any counter.  The
// partials and the order of the final sum are unchanged.
__device__ __forceinline__ bool publish_partial_tree(Red red, unsigned nblocks, double a, double b, bool two) {
  __shared__ bool last;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  if (tid == 0) {
    const unsigned bl = block_linear();
    red.partial[bl] = a;
    if (two) red.partial[nblocks + bl] = b;
    __threadfence();
    constexpr unsigned G = 64;
    const unsigned ng = (nblocks + G - 1) / G;
    bool l = false;
    if (ng <= 1) {
      l = atomicAdd(red.counter, 1u) == nblocks - 1;
    } else {
      const unsigned g = bl / G, gs = min(G, nblocks - g * G);
      if (atomicAdd(red.gcount + g, 1u) == gs - 1) {
        red.gcount[g] = 0u;  // every block of the group has arrived
        __threadfence();
        l = atomicAdd(red.counter, 1u) == ng - 1;
      }
    }
    if (l) __threadfence();
    last = l;
  }
  __syncthreads();
  return last;
}

// In the last block: sum of partial[0..n) in a fixed order (strided per
// thread, then the block tree).  Valid in thread 0.
__device__ __forceinline__ double final_sum(const double* part, unsigned n, double* sh) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  double s = 0.0;
  for (unsigned q = tid; q < n; q += nthr) s += __ldcg(part + q);
  return block_sum(s, sh);
}
__device__ __forceinline__ double final_max(const double* part, unsigned n, double* sh) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  double s = 0.0;
  for (unsigned q = tid; q < n; q += nthr) s = fmax(s, __ldcg(part + q));
  return block_max(s, sh);
}

__device__ __forceinline__ int flag_read(const int* f) { return __ldcg(f); }

}  // namespace stp
