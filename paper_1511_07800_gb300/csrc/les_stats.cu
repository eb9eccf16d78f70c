// Statistics of the LES (Sec. 6): plane averages of the velocity moments per
// level and streamwise two-point correlations, accumulated on the device
// between steps.  Velocities are taken at the cell centres (the mean of the
// two faces of each component), so that products are of co-located values.
// Sums are FP64, in a fixed order (one block per level, one per x shift),
// so repeated runs give the same bits.
#include "device_util.cuh"
#include "stp_internal.cuh"

namespace stp {

namespace {

// plane sums of uc, vc, wc, uc^2, vc^2, wc^2, uc vc, uc wc, vc wc at level
// blockIdx.x, added to mom[m * nz + k]
template <typename T>
__global__ void __launch_bounds__(256) k_plane_moments(int nx, int ny, int nz, const T* __restrict__ u,
                                                       const T* __restrict__ v, const T* __restrict__ w,
                                                       double* __restrict__ mom) {
  __shared__ double sh[32];
  const int k = blockIdx.x;
  const size_t plane = (size_t)nx * ny, base = (size_t)k * plane;
  double s[kStatMoments];
#pragma unroll
  for (int m = 0; m < kStatMoments; m++) s[m] = 0.0;
  for (size_t q = threadIdx.x; q < plane; q += blockDim.x) {
    const int i = (int)(q % nx), j = (int)(q / nx);
    const int ip = i == nx - 1 ? 0 : i + 1, jp = j == ny - 1 ? 0 : j + 1;
    const double uc = 0.5 * ((double)u[base + (size_t)j * nx + i] + (double)u[base + (size_t)j * nx + ip]);
    const double vc = 0.5 * ((double)v[base + (size_t)j * nx + i] + (double)v[base + (size_t)jp * nx + i]);
    const double wc = 0.5 * ((double)w[base + q] + (double)w[base + plane + q]);
    s[0] += uc;
    s[1] += vc;
    s[2] += wc;
    s[3] += uc * uc;
    s[4] += vc * vc;
    s[5] += wc * wc;
    s[6] += uc * vc;
    s[7] += uc * wc;
    s[8] += vc * wc;
  }
#pragma unroll
  for (int m = 0; m < kStatMoments; m++) {
    const double t = block_sum(s[m], sh);
    if (threadIdx.x == 0) mom[m * nz + k] += t;
    __syncthreads();
  }
}

// streamwise products at level kc: corr[c * nx + d] += sum_{i, j} q_c(i + d, j) q_c(i, j)
// for q = u (x faces), v (y faces), wc (centre); one block per shift d
template <typename T>
__global__ void __launch_bounds__(256) k_corr_x(int nx, int ny, int kc, const T* __restrict__ u,
                                                const T* __restrict__ v, const T* __restrict__ w,
                                                double* __restrict__ corr) {
  __shared__ double sh[32];
  const int d = blockIdx.x;
  const size_t plane = (size_t)nx * ny, base = (size_t)kc * plane;
  double su = 0.0, sv = 0.0, sw = 0.0;
  for (size_t q = threadIdx.x; q < plane; q += blockDim.x) {
    const int i = (int)(q % nx), j = (int)(q / nx);
    const int id = i + d < nx ? i + d : i + d - nx;
    const size_t a = base + (size_t)j * nx + i, b = base + (size_t)j * nx + id;
    su += (double)u[b] * (double)u[a];
    sv += (double)v[b] * (double)v[a];
    const double wa = 0.5 * ((double)w[a] + (double)w[a + plane]), wb = 0.5 * ((double)w[b] + (double)w[b + plane]);
    sw += wb * wa;
  }
  const double tu = block_sum(su, sh);
  if (threadIdx.x == 0) corr[0 * nx + d] += tu;
  __syncthreads();
  const double tv = block_sum(sv, sh);
  if (threadIdx.x == 0) corr[1 * nx + d] += tv;
  __syncthreads();
  const double tw = block_sum(sw, sh);
  if (threadIdx.x == 0) corr[2 * nx + d] += tw;
}

}  // namespace

template <typename T>
cudaError_t launch_les_stats(int nx, int ny, int nz, int kc, const T* u, const T* v, const T* w, double* mom,
                             double* corr, cudaStream_t s) {
  k_plane_moments<T><<<nz, 256, 0, s>>>(nx, ny, nz, u, v, w, mom);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_corr_x<T><<<nx, 256, 0, s>>>(nx, ny, kc, u, v, w, corr);
  return cudaGetLastError();
}
template cudaError_t launch_les_stats<float>(int, int, int, int, const float*, const float*, const float*, double*,
                                             double*, cudaStream_t);
template cudaError_t launch_les_stats<double>(int, int, int, int, const double*, const double*, const double*,
                                              double*, double*, cudaStream_t);

}  // namespace stp
