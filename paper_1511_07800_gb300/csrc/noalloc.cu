// Pressure-equation residual norm without any device allocation.
//
// A variant of the solve's residual-check kernel whose scratch memory (the
// z couplings, one partial sum per block, the arrival counter and the
// result) lives in one file-scope device array instead of buffers that
// stp_init allocates.  It serves callers that hold their own device buffers
// for p and b but may not allocate: for example a host program that has
// handed all device memory to its own pool allocator, or a time-critical
// loop that cannot accept the device-wide synchronisation that cudaMalloc
// and cudaFree can cause.
//
// The array is a host-side stand-in in host code: its device address is
// obtained once per device with cudaGetSymbolAddress (the first call on a
// device does this set-up).  With CUDA's lazy module loading (the default
// since CUDA 12.2) that first call can also be what loads this library's
// device code on the device, and with it the array: that one-time load is
// a device allocation made by the CUDA runtime, not by this call.  A caller
// that must not see it at all can load the module eagerly
// (CUDA_MODULE_LOADING=EAGER) or make one call during its set-up.  Every
// call shares the array, which keeps the last call's contents; the arrival
// counter is cleared at the start of each call.  Calls whose work overlaps
// on the GPU (different streams, or several host threads) race on the
// array and must be serialised by the caller.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "device_util.cuh"
#include "stp_internal.cuh"

namespace stp {

// limits of the shared scratch array
constexpr int kNoallocMaxNz = 4096;
constexpr unsigned kNoallocMaxBlocks = 65536;

struct NoallocScratch {
  double cup[kNoallocMaxNz];
  double cdn[kNoallocMaxNz];
  double partial[kNoallocMaxBlocks];
  double result[8];
  unsigned counter[8];
  int flag[8];
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

namespace {

std::mutex g_setup_mutex;
NoallocScratch* g_scratch_addr[256] = {};

__global__ void __launch_bounds__(kBX* kBY) k_residual_noalloc(int nx, int ny, int nz, double idx2, double idy2,
                                                                const double* __restrict__ p,
                                                                const double* __restrict__ b,
                                                                double* __restrict__ r_out, NoallocScratch* sc,
                                                                unsigned nblocks) {
  __shared__ double sh[32];
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  double s = 0.0;
  if (i < nx && j < ny) {
    const int plane = nx * ny;
    const int ip = i == nx - 1 ? 0 : i + 1, im = i == 0 ? nx - 1 : i - 1;
    const int jp = j == ny - 1 ? 0 : j + 1, jm = j == 0 ? ny - 1 : j - 1;
    const int row = k * plane, q = row + j * nx + i;
    const double pc = p[q];
    double lap = idx2 * ((p[row + j * nx + ip] - pc) + (p[row + j * nx + im] - pc)) +
                 idy2 * ((p[row + jp * nx + i] - pc) + (p[row + jm * nx + i] - pc));
    if (k < nz - 1) lap += sc->cup[k] * (p[q + plane] - pc);
    if (k > 0) lap += sc->cdn[k] * (p[q - plane] - pc);
    const double r = b[q] - lap;
    if (r_out) r_out[q] = r;
    s = r * r;
  }
  s = block_sum(s, sh);
  Red red{sc->partial, sc->counter, sc->result, sc->flag};
  if (publish_partial(red, nblocks, s, 0.0, false)) {
    const double tot = final_sum(sc->partial, nblocks, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      sc->result[0] = sqrt(tot);
      sc->counter[0] = 0u;
    }
  }
}

}  // namespace

// defined in api.cu: z couplings of the Poisson operator for a channel, and
// the message stp_last_error(NULL) returns
void poisson_couplings(const stp_config& c, std::vector<double>& cup, std::vector<double>& cdn);
void set_thread_error(const std::string& msg);

namespace {
int noalloc_fail(int code, const std::string& m) {
  set_thread_error(m);
  return code;
}
}  // namespace

}  // namespace stp

using namespace stp;

extern "C" int stp_poisson_residual_noalloc(int nx, int ny, int nz, double Lx, double Ly, double Lz, double stretch,
                                            const double* p, const double* b, double* r_out, double* norm_out,
                                            void* stream) {
  if (!p || !b || !norm_out) return noalloc_fail(STP_EINVAL, "p, b and norm_out are required");
  if (nx < 3 || ny < 3 || nz < 2) return noalloc_fail(STP_EINVAL, "need nx, ny >= 3 and nz >= 2");
  if (!(Lx > 0 && Ly > 0 && Lz > 0) || !(stretch >= 0))
    return noalloc_fail(STP_EINVAL, "box lengths must be positive and stretch >= 0");
  if (nz > kNoallocMaxNz)
    return noalloc_fail(STP_EINVAL, "nz exceeds the scratch limit of " + std::to_string(kNoallocMaxNz));
  const Launch l = plane_launch(nx, ny, nz);
  if ((double)l.grid.x * l.grid.y * l.grid.z > (double)kNoallocMaxBlocks)
    return noalloc_fail(STP_EINVAL, "grid too large for the scratch array: ceil(nx/32)*ceil(ny/8)*nz must be <= " +
                                        std::to_string(kNoallocMaxBlocks));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(STP_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 256) return noalloc_fail(STP_EINVAL, "device ordinal out of range");
  NoallocScratch* sc = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* addr = nullptr;
      e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
      if (e != cudaSuccess)
        return noalloc_fail(STP_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = (NoallocScratch*)addr;
    }
    sc = g_scratch_addr[dev];
  }
  stp_config c;
  stp_config_defaults(&c);
  c.nx = nx;
  c.ny = ny;
  c.nz = nz;
  c.Lx = Lx;
  c.Ly = Ly;
  c.Lz = Lz;
  c.stretch = stretch;
  std::vector<double> cup, cdn;
  poisson_couplings(c, cup, cdn);
  cudaStream_t st = (cudaStream_t)stream;
  e = cudaMemcpyAsync(sc->cup, cup.data(), sizeof(double) * nz, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sc->cdn, cdn.data(), sizeof(double) * nz, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc->counter, 0, sizeof(sc->counter), st);
  if (e != cudaSuccess) return noalloc_fail(STP_ECUDA, std::string("scratch set-up: ") + cudaGetErrorString(e));
  const double dx = Lx / nx, dy = Ly / ny;
  k_residual_noalloc<<<l.grid, l.block, 0, st>>>(nx, ny, nz, 1.0 / (dx * dx), 1.0 / (dy * dy), p, b, r_out, sc,
                                                 l.nblocks);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(norm_out, sc->result, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return noalloc_fail(STP_ECUDA, std::string("residual kernel: ") + cudaGetErrorString(e));
  return STP_OK;
}
