// 3-D U-Net for the learned pressure guess: forward, backward and Adam, all
// in hand-written kernels.  BF16 weights and activations, FP32 accumulation
// on the tensor cores (tcgen05 with TMEM accumulators for the 3x3x3
// convolutions of the larger levels, mma.sync m16n8k16 for the rest), FP32
// master weights, gradients and optimiser state.
//
// Network (channels-last [voxel][channel], voxel = ((n*D + z)*H + y)*W + x):
//   encoder level l = 1..4 (16, 32, 64, 128 channels): two 3x3x3 conv+ReLU,
//     then a 2x2x2 mean pool (not after level 4)
//   decoder level l = 3, 2, 1: input = concat(upsample2(deeper), skip e_l),
//     two 3x3x3 conv+ReLU
//   output: 1x1x1 conv of the 16 channels, linear
// Convolutions are periodic in x and y and zero-padded in z.  The skip of
// level l is written straight into the channel slice of the decoder's
// concat buffer, so no copy is needed.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <string>
#include <vector>

#include "device_util.cuh"
#include "stp_internal.cuh"

namespace stp {
namespace nn {

typedef __nv_bfloat16 bf16;

struct Dims {
  int n, d, h, w;
  __host__ __device__ long long vox() const { return (long long)n * d * h * w; }
};

__device__ __forceinline__ void mma16816(float* c, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ unsigned ld_u32(const bf16* p) { return *reinterpret_cast<const unsigned*>(p); }

__device__ __forceinline__ unsigned pack2(bf16 lo, bf16 hi) {
  return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

// source voxel of v shifted by tap t (periodic y, x; -1 outside the walls)
// voxel index (below 2^31, checked at creation) as sample and coordinates,
// in 32-bit arithmetic
struct Coord {
  int n, z, y, x;
};
__device__ __forceinline__ Coord coord_of(const Dims& dm, unsigned v) {
  Coord c;
  c.x = (int)(v % (unsigned)dm.w);
  v /= (unsigned)dm.w;
  c.y = (int)(v % (unsigned)dm.h);
  v /= (unsigned)dm.h;
  c.z = (int)(v % (unsigned)dm.d);
  c.n = (int)(v / (unsigned)dm.d);
  return c;
}
__device__ __forceinline__ long long voxel_at(const Dims& dm, int n, int z, int y, int x) {
  return ((long long)(n * dm.d + z) * dm.h + y) * dm.w + x;
}

// source voxel of tap t = (kz*3 + ky)*3 + kx at c: periodic in x and y,
// -1 outside the walls in z
__device__ __forceinline__ long long tap_from(const Dims& dm, const Coord& c, int t) {
  const int z2 = c.z + t / 9 - 1;
  if (z2 < 0 || z2 >= dm.d) return -1;
  int y2 = c.y + (t / 3) % 3 - 1;
  int x2 = c.x + t % 3 - 1;
  y2 = y2 < 0 ? y2 + dm.h : (y2 >= dm.h ? y2 - dm.h : y2);
  x2 = x2 < 0 ? x2 + dm.w : (x2 >= dm.w ? x2 - dm.w : x2);
  return voxel_at(dm, c.n, z2, y2, x2);
}

// ---------------------------------------------------------------------------
// 3x3x3 convolution as an implicit GEMM on the tensor cores:
//   y[v][o] = b[o] + sum_{t, c} wt[t][o][c] x[v + off(t)][c]
// M = voxels, N = output channels, K = 27 taps x input channels.  A warp
// computes 32 voxels x 8*NT channels; a block has 4 warps (128 voxels).
// Options: ReLU; multiply by (mask > 0) (the derivative of the ReLU that
// produced this layer's input, used when the kernel runs the backward data
// pass with transposed weights); no bias when bias is NULL.
// ---------------------------------------------------------------------------
template <int NT>
__global__ void __launch_bounds__(128) k_conv3(Dims dm, const bf16* __restrict__ x, int ldx, int cin,
                                               const bf16* __restrict__ wt, const float* __restrict__ bias, int cout,
                                               bf16* __restrict__ y, int ldy, int relu, const bf16* __restrict__ mask,
                                               int ldm) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const long long V = dm.vox();
  const long long vb = ((long long)blockIdx.x * 4 + warp) * 32;
  const int cob = blockIdx.y * NT * 8;
  float acc[2][NT][4];
#pragma unroll
  for (int m = 0; m < 2; m++)
#pragma unroll
    for (int n = 0; n < NT; n++) acc[m][n][0] = acc[m][n][1] = acc[m][n][2] = acc[m][n][3] = 0.f;
  long long vrow[4];
  Coord crow[4];
#pragma unroll
  for (int r = 0; r < 4; r++) {
    vrow[r] = vb + (r >> 1) * 16 + g + (r & 1) * 8;
    crow[r] = coord_of(dm, (unsigned)(vrow[r] < V ? vrow[r] : 0));
  }
  const int kc = cin >> 4;
  for (int t = 0; t < 27; t++) {
    long long src[4];
#pragma unroll
    for (int r = 0; r < 4; r++) src[r] = vrow[r] < V ? tap_from(dm, crow[r], t) : -1;
    for (int c = 0; c < kc; c++) {
      unsigned a[2][4];
#pragma unroll
      for (int m = 0; m < 2; m++) {
        const long long s0 = src[2 * m], s1 = src[2 * m + 1];
        const int col = c * 16 + 2 * q;
        a[m][0] = s0 >= 0 ? ld_u32(x + s0 * ldx + col) : 0u;
        a[m][1] = s1 >= 0 ? ld_u32(x + s1 * ldx + col) : 0u;
        a[m][2] = s0 >= 0 ? ld_u32(x + s0 * ldx + col + 8) : 0u;
        a[m][3] = s1 >= 0 ? ld_u32(x + s1 * ldx + col + 8) : 0u;
      }
#pragma unroll
      for (int n = 0; n < NT; n++) {
        const int co = cob + n * 8 + g;
        unsigned b[2] = {0u, 0u};
        if (co < cout) {
          const bf16* wp = wt + ((long long)t * cout + co) * cin + c * 16 + 2 * q;
          b[0] = ld_u32(wp);
          b[1] = ld_u32(wp + 8);
        }
        mma16816(acc[0][n], a[0], b);
        mma16816(acc[1][n], a[1], b);
      }
    }
  }
#pragma unroll
  for (int m = 0; m < 2; m++)
#pragma unroll
    for (int n = 0; n < NT; n++) {
      const int co = cob + n * 8 + 2 * q;
      if (co >= cout) continue;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const long long v = vrow[2 * m + h];
        if (v >= V) continue;
        float v0 = acc[m][n][2 * h], v1 = acc[m][n][2 * h + 1];
        if (bias) {
          v0 += bias[co];
          v1 += bias[co + 1];
        }
        if (relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        if (mask) {
          const bf16* mp = mask + v * ldm + co;
          if (!(__bfloat162float(mp[0]) > 0.f)) v0 = 0.f;
          if (!(__bfloat162float(mp[1]) > 0.f)) v1 = 0.f;
        }
        *reinterpret_cast<unsigned*>(y + v * ldy + co) = pack2(__float2bfloat16(v0), __float2bfloat16(v1));
      }
    }
}

// ---------------------------------------------------------------------------
// The same convolution on the fifth-generation tensor cores (tcgen05, TMEM
// accumulator), for layers whose level has w % 8 == 0 and h % 16 == 0 and
// channel counts that are multiples of 16.
//
// A block computes zt planes of 128 voxels, 8 (x) x 16 (y) at zt
// consecutive z, for all cout channels: per plane M = 128, N = cout,
// K = 27 taps x cin, the zt accumulators side by side in tensor memory.  The
// input is staged once per group of up to 64 channels as a halo of
// 10 x 18 x (zt + 2) voxels (periodic in x and y, zeros outside the walls)
// in the K-major core-matrix layout without swizzle: 8-channel chunk j of
// halo voxel (hx, hy, hz) is 16 bytes at j CHUNK + ((hz HY + hy) HX + hx) 16,
// CHUNK = 16 HX HY (zt + 2).  The A operand of tap (dz, dy, dx) for plane p
// is then the descriptor whose start is the halo voxel (1+dx, 1+dy, p+dz):
// its 8-row core matrices are 8 consecutive x (16 bytes apart), the next 8
// rows are the next y (SBO = 16 HX bytes), the next 8 channels the next
// chunk (LBO = one chunk of the halo).  So the 27 taps need no data
// movement.  The weights of a tap (cout x group channels, the same layout
// with LBO = 128, SBO = 16 x group chunks) are either all resident (every
// tap of a group loaded at once, then all the group's MMAs back to back,
// one commit and one wait) or, when they do not fit, stream through a ring
// of three stages, a stage refilled once the MMAs that read it have
// completed (tcgen05.commit to that stage's mbarrier).  One thread issues
// the MMAs and one thread polls each barrier while the others wait at the
// block barrier.  Every wait is bounded; on a time-out the block sets *err,
// skips the rest, and still frees its tensor memory.
// ---------------------------------------------------------------------------
constexpr int TC_TX = 8, TC_TY = 16, TC_HX = 10, TC_HY = 18;
constexpr int TC_PLANE = TC_HX * TC_HY * 16;  // bytes of one halo plane of one 8-channel chunk
constexpr int TC_CG = 64;                     // channels per halo group
constexpr int TC_STAGES = 3;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16(uint32_t dst, const void* src, bool fill) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(fill ? 16 : 0)
               : "memory");
}

// shared-memory matrix descriptor: no swizzle, K-major core matrices
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: BF16 A and B, FP32 D, both K-major
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// bounded wait for phase `parity` of an mbarrier (about one second of
// clock), polled with a short sleep between tries
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > 2000000000LL) return false;
    __nanosleep(64);
  }
}

__global__ void __launch_bounds__(128) k_conv3_tc(Dims dm, const bf16* __restrict__ x, int ldx, int cin,
                                                  const bf16* __restrict__ wt, const float* __restrict__ bias,
                                                  int cout, bf16* __restrict__ y, int ldy, int relu,
                                                  const bf16* __restrict__ mask, int ldm, int resident, int zt,
                                                  const bf16* __restrict__ wimg, int* err) {
  extern __shared__ __align__(1024) uint8_t tsm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cgmax = cin < TC_CG ? cin : TC_CG;  // channels of the widest group
  const int stage_bytes = cout * cgmax * 2;     // one tap's weights of one group
  const int hz_n = zt + 2;                      // halo planes
  const int chunk = TC_PLANE * hz_n;            // bytes of one 8-channel chunk of the halo
  uint8_t* halo = tsm;
  uint8_t* wst = tsm + (cgmax / 8) * chunk;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(wst + (resident ? 27 : TC_STAGES) * stage_bytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + TC_STAGES + 1);  // mbar[TC_STAGES]: the bulk weight copy
  volatile int* sfail = reinterpret_cast<volatile int*>(tslot + 1);
  // block -> tile
  const int nxt = dm.w / TC_TX, nyt = dm.h / TC_TY;
  long long b = blockIdx.x;
  const int xt = (int)(b % nxt);
  b /= nxt;
  const int yt = (int)(b % nyt);
  b /= nyt;
  const int nzt = dm.d / zt;
  const int z0 = (int)(b % nzt) * zt;
  const long long nn = b / nzt;
  const int x0 = xt * TC_TX, y0 = yt * TC_TY;
  if (tid == 0) {
    for (int s = 0; s <= TC_STAGES; s++) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(mbar + s)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *sfail = 0;
  }
  int ncols = 32;
  while (ncols < zt * cout) ncols <<= 1;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const int ngroups = (cin + TC_CG - 1) / TC_CG;
  const int Q = ngroups * 27;
  const uint32_t idesc = tc_idesc(128, cout);
  // streaming: one tap's weights of channel group g into a ring stage
  auto load_w = [&](int q) {
    const int g = q / 27, t = q % 27;
    const int c0 = g * TC_CG, nch = min(TC_CG, cin - c0) / 8;
    const uint32_t base = su32(wst + (q % TC_STAGES) * stage_bytes);
    for (int o = tid; o < cout; o += 128) {
      const bf16* src = wt + ((long long)t * cout + o) * cin + c0;
      const uint32_t dst = base + (o / 8) * (nch * 128) + (o % 8) * 16;
      for (int j = 0; j < nch; j++) cp16(dst + j * 128, src + 8 * j, true);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // resident: every tap's weights of group g, (tap, row) pairs spread over the block
  auto load_w_all = [&](int g) {
    const int c0 = g * TC_CG, nch = min(TC_CG, cin - c0) / 8;
    const uint32_t base = su32(wst);
    for (int i = tid; i < 27 * cout; i += 128) {
      const int t = i / cout, o = i - t * cout;
      const bf16* src = wt + ((long long)t * cout + o) * cin + c0;
      const uint32_t dst = base + t * stage_bytes + (o / 8) * (nch * 128) + (o % 8) * 16;
      for (int j = 0; j < nch; j++) cp16(dst + j * 128, src + 8 * j, true);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // halo of group g: one voxel per thread, its chunks inner
  auto load_halo = [&](int g) {
    const int c0 = g * TC_CG, nch = min(TC_CG, cin - c0) / 8;
    const uint32_t base = su32(halo);
    for (int i = tid; i < TC_HX * TC_HY * hz_n; i += 128) {
      const int hx = i % TC_HX, hy = (i / TC_HX) % TC_HY, hz = i / (TC_HX * TC_HY);
      int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
      const int gz = z0 - 1 + hz;
      gx = gx < 0 ? gx + dm.w : (gx >= dm.w ? gx - dm.w : gx);
      gy = gy < 0 ? gy + dm.h : (gy >= dm.h ? gy - dm.h : gy);
      const bool in = gz >= 0 && gz < dm.d;
      const long long v = ((nn * dm.d + (in ? gz : 0)) * dm.h + gy) * dm.w + gx;
      const bf16* src = x + v * ldx + c0;
      const uint32_t dst = base + i * 16;  // chunk 0 of voxel (hx, hy, hz); chunk j is `chunk` further
      for (int j = 0; j < nch; j++) cp16(dst + j * chunk, src + 8 * j, in);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // the MMAs of step q (group q / 27, tap q % 27) for every plane, with that
  // tap's weights at b0; plane p accumulates in columns [p cout, (p+1) cout)
  auto issue_tap = [&](int q, uint32_t b0) {
    const int g = q / 27, t = q % 27;
    const int c0 = g * TC_CG, nch = min(TC_CG, cin - c0) / 8;
    const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;  // halo offsets 0..2 (shift + 1)
    const uint32_t a0 = su32(halo) + ((dz * TC_HY + dy) * TC_HX + dx) * 16;
    for (int pl = 0; pl < zt; pl++) {
      for (int kk = 0; kk < nch / 2; kk++) {
        const uint64_t ad = tc_desc(a0 + pl * TC_PLANE + 2 * kk * chunk, chunk, TC_HX * 16);
        const uint64_t bd = tc_desc(b0 + 2 * kk * 128, 128, nch * 128);
        const uint32_t acc = (q > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + (uint32_t)(pl * cout)),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
    }
  };
  auto commit = [&](int stage) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     su32(mbar + stage))
                 : "memory");
  };
  // one thread polls the barrier, the others wait at __syncthreads (no issue
  // slots spent spinning); false on a time-out
  auto block_wait = [&](int stage, uint32_t parity) {
    if (tid == 0 && !tc_wait(su32(mbar + stage), parity)) *sfail = 1;
    __syncthreads();
    return *sfail == 0;
  };
  bool ok = true;
  if (resident) {
    for (int g = 0; g < ngroups && ok; g++) {
      if (wimg) {
        // the group's 27 taps, pre-arranged in this layout, as one bulk copy
        if (tid == 0) {
          const uint32_t bytes = 27u * (uint32_t)stage_bytes;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(mbar + TC_STAGES)),
                       "r"(bytes)
                       : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(wst)),
              "l"(wimg + (size_t)g * 27 * (stage_bytes / 2)), "r"(bytes), "r"(su32(mbar + TC_STAGES))
              : "memory");
        }
        load_halo(g);
      } else {
        load_halo(g);
        load_w_all(g);
      }
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (wimg && !block_wait(TC_STAGES, g & 1)) {
        ok = false;
        break;
      }
      if (tid == 0) {
        for (int t = 0; t < 27; t++) issue_tap(g * 27 + t, su32(wst + t * stage_bytes));
        commit(0);
      }
      if (g + 1 < ngroups && !block_wait(0, g & 1)) ok = false;  // the next group overwrites halo and weights
    }
  } else {
    load_halo(0);
    load_w(0);
    if (Q > 1) load_w(1);
    for (int q = 0; q < Q; q++) {
      const int g = q / 27, t = q % 27;
      if (t == 0 && g > 0) {
        // the previous group's MMAs read the halo: wait for the last of them
        if (!block_wait((q - 1) % TC_STAGES, ((q - 1) / TC_STAGES) & 1)) {
          ok = false;
          break;
        }
        load_halo(g);
      }
      // this step's weights (and a new halo) have landed; the next step's may be in flight
      if (t == 0 || q + 1 >= Q)
        asm volatile("cp.async.wait_group 0;" ::: "memory");
      else
        asm volatile("cp.async.wait_group 1;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        issue_tap(q, su32(wst + (q % TC_STAGES) * stage_bytes));
        commit(q % TC_STAGES);
      }
      // refill the stage that step q-1 used with step q+2's weights
      if (q + 2 < Q) {
        if (q >= 1 && !block_wait((q - 1) % TC_STAGES, ((q - 1) / TC_STAGES) & 1)) {
          ok = false;
          break;
        }
        load_w(q + 2);
      }
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  // all MMAs done: the last commit covers every earlier one
  __syncthreads();
  const bool done = ok && *sfail == 0 &&
                    (resident ? block_wait(0, (ngroups - 1) & 1)
                              : block_wait((Q - 1) % TC_STAGES, ((Q - 1) / TC_STAGES) & 1));
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!done) {
    if (tid == 0) atomicExch(err, 1);
  } else {
    const int r = warp * 32 + lane;  // TMEM lane = output row
    for (int pl = 0; pl < zt; pl++) {
      const long long v = ((nn * dm.d + z0 + pl) * dm.h + y0 + r / 8) * dm.w + x0 + (r % 8);
      for (int c = 0; c < cout; c += 16) {
        uint32_t a[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]),
              "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15])
            : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(pl * cout + c)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        uint32_t o[8];
#pragma unroll
        for (int h = 0; h < 8; h++) {
          float v0 = __uint_as_float(a[2 * h]), v1 = __uint_as_float(a[2 * h + 1]);
          const int co = c + 2 * h;
          if (bias) {
            v0 += bias[co];
            v1 += bias[co + 1];
          }
          if (relu) {
            v0 = fmaxf(v0, 0.f);
            v1 = fmaxf(v1, 0.f);
          }
          if (mask) {
            const bf16* mp = mask + v * ldm + co;
            if (!(__bfloat162float(mp[0]) > 0.f)) v0 = 0.f;
            if (!(__bfloat162float(mp[1]) > 0.f)) v1 = 0.f;
          }
          o[h] = pack2(__float2bfloat16(v0), __float2bfloat16(v1));
        }
        uint4* yp = reinterpret_cast<uint4*>(y + v * ldy + c);
        yp[0] = make_uint4(o[0], o[1], o[2], o[3]);
        yp[1] = make_uint4(o[4], o[5], o[6], o[7]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// First layer: 1 input channel (FP32 input rounded to BF16) -> 16 channels, ReLU.
__global__ void k_conv_in(Dims dm, const float* __restrict__ x, const float* __restrict__ w /*[16][27]*/,
                          const float* __restrict__ bias, bf16* __restrict__ y, int ldy) {
  __shared__ float ws[16 * 27 + 16];
  for (int i = threadIdx.x; i < 16 * 27; i += blockDim.x) ws[i] = __bfloat162float(__float2bfloat16(w[i]));
  for (int i = threadIdx.x; i < 16; i += blockDim.x) ws[16 * 27 + i] = bias[i];
  __syncthreads();
  const long long V = dm.vox();
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    float acc[16];
#pragma unroll
    for (int o = 0; o < 16; o++) acc[o] = ws[16 * 27 + o];
    // the taps in order, one z plane of 9 at a time: its 9 inputs are loaded
    // together, then multiplied in; planes outside the walls add nothing
    const Coord cv = coord_of(dm, (unsigned)v);
    for (int kz = 0; kz < 3; kz++) {
      if (tap_from(dm, cv, kz * 9) < 0) continue;
      float xt[9];
#pragma unroll
      for (int u = 0; u < 9; u++) xt[u] = __bfloat162float(__float2bfloat16(x[tap_from(dm, cv, kz * 9 + u)]));
#pragma unroll
      for (int u = 0; u < 9; u++)
#pragma unroll
        for (int o = 0; o < 16; o++) acc[o] = fmaf(ws[o * 27 + kz * 9 + u], xt[u], acc[o]);
    }
#pragma unroll
    for (int o = 0; o < 16; o += 2)
      *reinterpret_cast<unsigned*>(y + v * ldy + o) =
          pack2(__float2bfloat16(fmaxf(acc[o], 0.f)), __float2bfloat16(fmaxf(acc[o + 1], 0.f)));
  }
}

// Output layer: 1x1x1, 16 channels -> 1, linear, FP32 output.
__global__ void k_conv_out(long long V, const bf16* __restrict__ x, int ldx, const float* __restrict__ w,
                           const float* __restrict__ bias, float* __restrict__ y) {
  float ws[16];
#pragma unroll
  for (int c = 0; c < 16; c++) ws[c] = __bfloat162float(__float2bfloat16(w[c]));
  const float b = bias[0];
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    float s = b;
#pragma unroll
    for (int c = 0; c < 16; c++) s = fmaf(ws[c], __bfloat162float(x[v * ldx + c]), s);
    y[v] = s;
  }
}

// Backward of the output layer: g_d1[v][c] = gy[v] w[c] (d1 > 0);
// dW[c] += sum_v gy[v] d1[v][c], db += sum_v gy[v].
__global__ void k_conv_out_bwd(long long V, const float* __restrict__ gy, const bf16* __restrict__ d1, int ldx,
                               const float* __restrict__ w, bf16* __restrict__ gd, int ldg, float* __restrict__ gw,
                               float* __restrict__ gb) {
  __shared__ float red[17][33];
  float ws[16], acc[17];
#pragma unroll
  for (int c = 0; c < 16; c++) {
    ws[c] = __bfloat162float(__float2bfloat16(w[c]));
    acc[c] = 0.f;
  }
  acc[16] = 0.f;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    const float g = gy[v];
    acc[16] += g;
#pragma unroll
    for (int c = 0; c < 16; c += 2) {
      const float a0 = __bfloat162float(d1[v * ldx + c]), a1 = __bfloat162float(d1[v * ldx + c + 1]);
      acc[c] += g * a0;
      acc[c + 1] += g * a1;
      *reinterpret_cast<unsigned*>(gd + v * ldg + c) =
          pack2(__float2bfloat16(a0 > 0.f ? g * ws[c] : 0.f), __float2bfloat16(a1 > 0.f ? g * ws[c + 1] : 0.f));
    }
  }
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 17; c++) {
    float s = acc[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[c][wp] = s;
  }
  __syncthreads();
  if (threadIdx.x < 17) {
    float s = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += red[threadIdx.x][i];
    if (threadIdx.x < 16)
      atomicAdd(gw + threadIdx.x, s);
    else
      atomicAdd(gb, s);
  }
}

// ---------------------------------------------------------------------------
// Weight gradient of a 3x3x3 layer on the tensor cores:
//   gw[o][c][t] += sum_v gz[v][o] x[v + off(t)][c],   gb[o] += sum_v gz[v][o]
// GEMM with M = output channels (16 per warp), N = input channels (32 per
// warp, 4 n-tiles), K = voxels.  Block = 4 warps over consecutive voxel
// chunks of one (tap, o-tile, c-tile); partial sums are reduced in shared
// memory and added to the FP32 gradient with atomics.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_wgrad3(Dims dm, const bf16* __restrict__ x, int ldx, int cin,
                                                const bf16* __restrict__ gz, int ldg, int cout,
                                                float* __restrict__ gw, float* __restrict__ gb, long long vchunk) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const int ct = (cin + 31) / 32;
  int idx = blockIdx.x;
  const int t = idx % 27;
  idx /= 27;
  const int cti = idx % ct;
  const int oti = idx / ct;
  const int ob = oti * 16, cb = cti * 32;
  const long long V = dm.vox();
  const long long v0 = (long long)blockIdx.y * vchunk;
  const long long v1 = V < v0 + vchunk ? V : v0 + vchunk;
  float acc[4][4];
#pragma unroll
  for (int n = 0; n < 4; n++) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
  const bf16 zero = __float2bfloat16(0.f);
  for (long long vs = v0 + warp * 16; vs < v1; vs += 64) {
    // the four voxels of this thread in the chunk: k = 2q, 2q+1, 2q+8, 2q+9
    long long vk[4] = {vs + 2 * q, vs + 2 * q + 1, vs + 2 * q + 8, vs + 2 * q + 9};
    long long sk[4];
    bf16 gzv[2][4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
      const bool ok = vk[i] < v1;
      sk[i] = ok ? tap_from(dm, coord_of(dm, (unsigned)vk[i]), t) : -1;
      gzv[0][i] = ok ? gz[vk[i] * ldg + ob + g] : zero;
      gzv[1][i] = ok ? gz[vk[i] * ldg + ob + g + 8] : zero;
    }
    unsigned a[4];
    a[0] = pack2(gzv[0][0], gzv[0][1]);
    a[1] = pack2(gzv[1][0], gzv[1][1]);
    a[2] = pack2(gzv[0][2], gzv[0][3]);
    a[3] = pack2(gzv[1][2], gzv[1][3]);
#pragma unroll
    for (int n = 0; n < 4; n++) {
      const int c = cb + n * 8 + g;
      bf16 xv[4];
#pragma unroll
      for (int i = 0; i < 4; i++) xv[i] = (c < cin && sk[i] >= 0) ? x[sk[i] * ldx + c] : zero;
      unsigned b[2] = {pack2(xv[0], xv[1]), pack2(xv[2], xv[3])};
      mma16816(acc[n], a, b);
    }
  }
  __shared__ float red[4][16][33];
#pragma unroll
  for (int n = 0; n < 4; n++) {
    red[warp][g][n * 8 + 2 * q] = acc[n][0];
    red[warp][g][n * 8 + 2 * q + 1] = acc[n][1];
    red[warp][g + 8][n * 8 + 2 * q] = acc[n][2];
    red[warp][g + 8][n * 8 + 2 * q + 1] = acc[n][3];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 16 * 32; e += 128) {
    const int o = e / 32, c = e % 32;
    if (cb + c >= cin) continue;
    const float s = red[0][o][c] + red[1][o][c] + red[2][o][c] + red[3][o][c];
    atomicAdd(gw + ((long long)(ob + o) * cin + cb + c) * 27 + t, s);
  }
  (void)gb;
}

// bias gradient: gb[o] += sum_v gz[v][o]
__global__ void k_bias_grad(long long V, const bf16* __restrict__ gz, int ldg, int cout, float* __restrict__ gb) {
  const int o = blockIdx.y * blockDim.x + threadIdx.x;
  if (o >= cout) return;
  float s = 0.f;
  for (long long v = blockIdx.x; v < V; v += gridDim.x) s += __bfloat162float(gz[v * ldg + o]);
  atomicAdd(gb + o, s);
}

// first-layer weight gradient: gw[o][0][t] += sum_v gz[v][o] x[v + off(t)];
// one tap per blockIdx.y
__global__ void k_wgrad_in(Dims dm, const float* __restrict__ x, const bf16* __restrict__ gz, int ldg,
                           float* __restrict__ gw) {
  __shared__ float red[16];
  if (threadIdx.x < 16) red[threadIdx.x] = 0.f;
  __syncthreads();
  const int t = blockIdx.y;
  float acc[16];
#pragma unroll
  for (int o = 0; o < 16; o++) acc[o] = 0.f;
  const long long V = dm.vox();
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    const long long s = tap_from(dm, coord_of(dm, (unsigned)v), t);
    if (s < 0) continue;
    const float xv = __bfloat162float(__float2bfloat16(x[s]));
#pragma unroll
    for (int o = 0; o < 16; o++) acc[o] = fmaf(__bfloat162float(gz[v * ldg + o]), xv, acc[o]);
  }
#pragma unroll
  for (int o = 0; o < 16; o++) {
    float s = acc[o];
    for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
    if ((threadIdx.x & 31) == 0) atomicAdd(&red[o], s);
  }
  __syncthreads();
  if (threadIdx.x < 16) atomicAdd(gw + threadIdx.x * 27 + t, red[threadIdx.x]);
}

// ---------------------------------------------------------------------------
// pooling, upsampling and the gradient plumbing between levels
// ---------------------------------------------------------------------------
// Pooling and upsampling move 16-byte channel vectors (c a multiple of 8,
// leading dimensions multiples of 8, so every vector is aligned), in 32-bit
// index arithmetic.  The kernels that reduce 8 fine voxels into a coarse
// one take one 8-channel vector a thread (blockIdx.y); those that write the
// fine level take one voxel a thread, all its channels (whole rows of
// stores).
__device__ __forceinline__ void unpack8(const uint4& u, float* f) {
  const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int i = 0; i < 4; i++) {
    f[2 * i] = __bfloat162float(__ushort_as_bfloat16((unsigned short)(w[i] & 0xFFFFu)));
    f[2 * i + 1] = __bfloat162float(__ushort_as_bfloat16((unsigned short)(w[i] >> 16)));
  }
}
__device__ __forceinline__ uint4 pack8(const float* f) {
  return make_uint4(pack2(__float2bfloat16(f[0]), __float2bfloat16(f[1])),
                    pack2(__float2bfloat16(f[2]), __float2bfloat16(f[3])),
                    pack2(__float2bfloat16(f[4]), __float2bfloat16(f[5])),
                    pack2(__float2bfloat16(f[6]), __float2bfloat16(f[7])));
}
__device__ __forceinline__ uint4 ld16(const bf16* p) { return *reinterpret_cast<const uint4*>(p); }
__device__ __forceinline__ void st16(bf16* p, const uint4& u) { *reinterpret_cast<uint4*>(p) = u; }

// out (coarse) = mean of the 2x2x2 fine block (summed in block order); fine dims dm
__global__ void k_pool(Dims dm, const bf16* __restrict__ x, int ldx, int c, bf16* __restrict__ y, int ldy) {
  const Dims cd{dm.n, dm.d / 2, dm.h / 2, dm.w / 2};
  const unsigned V = (unsigned)cd.vox();
  if ((int)blockIdx.y * 8 >= c) return;
  for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
    const Coord q = coord_of(cd, v);
    long long f[8];
#pragma unroll
    for (int k = 0; k < 8; k++)
      f[k] = voxel_at(dm, q.n, 2 * q.z + (k >> 2), 2 * q.y + ((k >> 1) & 1), 2 * q.x + (k & 1));
    const int ch = blockIdx.y * 8;
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, e[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
      unpack8(ld16(x + f[k] * ldx + ch), e);
#pragma unroll
      for (int i = 0; i < 8; i++) s[i] += e[i];
    }
#pragma unroll
    for (int i = 0; i < 8; i++) s[i] *= 0.125f;
    st16(y + (long long)v * ldy + ch, pack8(s));
  }
}

// fine = coarse value (nearest); coarse dims cd
__global__ void k_upsample(Dims cd, const bf16* __restrict__ x, int ldx, int c, bf16* __restrict__ y, int ldy) {
  const Dims fd{cd.n, cd.d * 2, cd.h * 2, cd.w * 2};
  const unsigned V = (unsigned)fd.vox();
  for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
    const Coord q = coord_of(fd, v);
    const long long cv = voxel_at(cd, q.n, q.z / 2, q.y / 2, q.x / 2);
    for (int ch = 0; ch < c; ch += 8) st16(y + (long long)v * ldy + ch, ld16(x + cv * ldx + ch));
  }
}

// coarse gradient of an upsample = sum over the fine block (in block
// order), times (act > 0)
__global__ void k_upsample_bwd_mask(Dims cd, const bf16* __restrict__ gf, int ldg, int c, const bf16* __restrict__ act,
                                    int lda, bf16* __restrict__ out, int ldo) {
  const Dims fd{cd.n, cd.d * 2, cd.h * 2, cd.w * 2};
  const unsigned V = (unsigned)cd.vox();
  if ((int)blockIdx.y * 8 >= c) return;
  for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
    const Coord q = coord_of(cd, v);
    long long f[8];
#pragma unroll
    for (int k = 0; k < 8; k++)
      f[k] = voxel_at(fd, q.n, 2 * q.z + (k >> 2), 2 * q.y + ((k >> 1) & 1), 2 * q.x + (k & 1));
    const int ch = blockIdx.y * 8;
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, e[8], a[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
      unpack8(ld16(gf + f[k] * ldg + ch), e);
#pragma unroll
      for (int i = 0; i < 8; i++) s[i] += e[i];
    }
    unpack8(ld16(act + (long long)v * lda + ch), a);
#pragma unroll
    for (int i = 0; i < 8; i++) s[i] = a[i] > 0.f ? s[i] : 0.f;
    st16(out + (long long)v * ldo + ch, pack8(s));
  }
}

// fine gradient of a level's output: pool backward (coarse / 8) plus the skip
// gradient, times (act > 0); fine dims fd
__global__ void k_pool_bwd_add_mask(Dims fd, const bf16* __restrict__ gc, int ldc, const bf16* __restrict__ gskip,
                                    int lds, int c, const bf16* __restrict__ act, int lda, bf16* __restrict__ out,
                                    int ldo) {
  const Dims cd{fd.n, fd.d / 2, fd.h / 2, fd.w / 2};
  const unsigned V = (unsigned)fd.vox();
  for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
    const Coord q = coord_of(fd, v);
    const long long cv = voxel_at(cd, q.n, q.z / 2, q.y / 2, q.x / 2);
    for (int ch = 0; ch < c; ch += 8) {
      float g[8], k[8], a[8], s[8];
      unpack8(ld16(gc + cv * ldc + ch), g);
      unpack8(ld16(gskip + (long long)v * lds + ch), k);
      unpack8(ld16(act + (long long)v * lda + ch), a);
#pragma unroll
      for (int i = 0; i < 8; i++) {
        const float t = 0.125f * g[i] + k[i];
        s[i] = a[i] > 0.f ? t : 0.f;
      }
      st16(out + (long long)v * ldo + ch, pack8(s));
    }
  }
}

// weights: master W[o][c][t] (FP32) -> wt[t][o][c] (BF16) and, for the
// backward data pass, wtt[26-t][c][o] (BF16)
__global__ void k_pack_weights(const float* __restrict__ w, int cout, int cin, bf16* __restrict__ wt,
                               bf16* __restrict__ wtt) {
  const long long total = (long long)cout * cin * 27;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(e % 27);
    const long long oc = e / 27;
    const int c = (int)(oc % cin), o = (int)(oc / cin);
    const bf16 v = __float2bfloat16(w[e]);
    wt[((long long)t * cout + o) * cin + c] = v;
    if (wtt) wtt[((long long)(26 - t) * cin + c) * cout + o] = v;
  }
}

// wt [t][cout][cin] (BF16) -> the resident weights of k_conv3_tc exactly as
// its shared memory holds them, so that a block loads a channel group's 27
// taps with one bulk copy: for group g (64 channels), tap t, output o and
// 8-channel chunk j, 16 bytes at g 27 S + t S + (o/8)(nch 128) + (o%8) 16 +
// j 128, with S = 2 cout min(cin, 64) bytes a tap and nch the group's chunks
__global__ void k_pack_image(const bf16* __restrict__ wt, int cin, int cout, bf16* __restrict__ img) {
  const int cg = cin < TC_CG ? cin : TC_CG, ngroups = (cin + TC_CG - 1) / TC_CG;
  const long long S = 2LL * cout * cg;
  const long long total = (long long)ngroups * 27 * cout * (cg / 8);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % (cg / 8));
    long long r = e / (cg / 8);
    const int o = (int)(r % cout);
    r /= cout;
    const int t = (int)(r % 27);
    const int g = (int)(r / 27);
    const int c0 = g * TC_CG, nch = min(TC_CG, cin - c0) / 8;
    if (j >= nch) continue;
    const long long off = g * 27 * S + t * S + (o / 8) * (nch * 128) + (o % 8) * 16 + j * 128;
    *reinterpret_cast<uint4*>(reinterpret_cast<char*>(img) + off) =
        *reinterpret_cast<const uint4*>(wt + ((long long)t * cout + o) * cin + c0 + 8 * j);
  }
}

// mean((y - t)^2) (per-block partials, summed with atomics) and gy = 2(y - t)/n
__global__ void k_mse(long long n, const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ gy,
                      float* __restrict__ loss) {
  float s = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    s += d * d;
    gy[i] = 2.f * d / (float)n;
  }
  for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s / (float)n);
}

__global__ void k_adam(long long n, float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// per-sample sums of squares: s2[i] += sum over sample i of r^2 (blockIdx.y = sample)
__global__ void k_sample_sumsq(long long Vs, const float* __restrict__ r, float* __restrict__ s2) {
  const float* rs = r + (long long)blockIdx.y * Vs;
  float s = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Vs; i += (long long)gridDim.x * blockDim.x)
    s += rs[i] * rs[i];
  for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
  if ((threadIdx.x & 31) == 0) atomicAdd(s2 + blockIdx.y, s);
}

// x = r / s_i and t = dp / s_i with s_i = RMS of sample i's r (0 if r = 0)
__global__ void k_scale_pairs(long long Vs, int nb, const float* __restrict__ r, const float* __restrict__ dp,
                              const float* __restrict__ s2, float kscale, float* __restrict__ x, float* __restrict__ t) {
  const long long total = Vs * nb;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const float rms = sqrtf(s2[e / Vs] / (float)Vs);
    const float inv = rms > 0.f ? 1.f / rms : 0.f;
    x[e] = r[e] * inv;
    if (t) t[e] = dp[e] * inv * kscale;
  }
}

// guess in the solver: x = r / s (s = ||r||_2 / sqrt(V), ||r|| read on the device)
__global__ void k_guess_in(long long V, const float* __restrict__ r, const double* __restrict__ norm,
                           float* __restrict__ x) {
  const double s = __ldcg(norm) / sqrt((double)V);
  const float inv = s > 0.0 ? (float)(1.0 / s) : 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x)
    x[i] = r[i] * inv;
}

// d = s * y / kscale
__global__ void k_guess_out(long long V, const float* __restrict__ y, const double* __restrict__ norm, float kscale,
                            float* __restrict__ d) {
  const float s = (float)(__ldcg(norm) / sqrt((double)V)) / kscale;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x)
    d[i] = s * y[i];
}

// FP32 -> BF16 (round to nearest even) and back, for the single-layer checks
__global__ void k_to_bf16(long long n, const float* __restrict__ a, bf16* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}
__global__ void k_from_bf16(long long n, const bf16* __restrict__ a, float* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = __bfloat162float(a[i]);
}

}  // namespace nn
}  // namespace stp

// ===========================================================================
// the network object and its C ABI
// ===========================================================================
using namespace stp;
using namespace stp::nn;

namespace {

const int kCh[4] = {16, 32, 64, 128};

struct Layer {
  int cin, cout, taps;
  long long woff, boff;  // offsets of W and b in the flat parameter vector
  bf16 *wt = nullptr, *wtt = nullptr;
  // wt and wtt in the shared-memory order of k_conv3_tc's resident weights
  // (null where that convolution does not run with resident weights)
  bf16 *img = nullptr, *timg = nullptr;
};

int blocks_for(long long n, int threads = 256) {
  long long b = (n + threads - 1) / threads;
  return (int)std::max<long long>(1, std::min<long long>(b, 152LL * 32));
}

}  // namespace

struct stp_unet {
  Dims dm[4];  // level dims (batch included), level 0 = full resolution
  int nmax;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::vector<Layer> L;  // 15 layers in parameter order
  long long np = 0;
  float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  long long adam_step = 0;
  // activations (BF16, channels-last)
  bf16 *ha[4] = {}, *e4 = nullptr, *u[3] = {}, *q[3] = {}, *hd[3] = {}, *d[3] = {};
  // gradients of activations
  bf16 *ga[4] = {}, *gb[4] = {}, *gu[3] = {};
  float *y = nullptr, *gy = nullptr, *loss = nullptr, *h_loss = nullptr;
  float *xin = nullptr, *tin = nullptr, *snorm = nullptr;  // normalised pairs, per-sample norms
  int guess_kernels = 0;                                   // kernels launched by one guess
  float out_scale = 1.f;                                   // the network predicts out_scale * dp / s
  int* d_err = nullptr;                                    // set by a tensor-core kernel whose wait timed out
  bool use_tc = true;                                      // tcgen05 convolutions where the shapes allow
  int tc_planes = 0;                                       // planes a tcgen05 block computes (0: by layer shape)
  int mma_nt = 0;                                          // mma.sync 8-channel tiles a block (0: by grid size)
  std::vector<void*> allocs;
  std::string err;
};

namespace {

int ufail(stp_unet* n, int code, const std::string& m) {
  if (n) n->err = m;
  return code;
}

#define UTRY(n, call)                                                                                  \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess) return ufail(n, STP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// after a synchronisation: did a tensor-core convolution give up waiting?
int check_tc_timeout(stp_unet* n) {
  int e = 0;
  UTRY(n, cudaMemcpy(&e, n->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) return ufail(n, STP_ETIMEOUT, "a tensor-core convolution timed out waiting for its MMAs");
  return STP_OK;
}

template <typename T>
int ualloc(stp_unet* n, T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * std::max<size_t>(count, 1));
  if (e != cudaSuccess) return ufail(n, STP_ENOMEM, "cudaMalloc failed in the network");
  n->allocs.push_back(*p);
  return STP_OK;
}

// concat widths: decoder level l (0..2) input = kCh[l+1] + kCh[l]
int cu_width(int l) { return kCh[l + 1] + kCh[l]; }

// shared memory of k_conv3_tc with zt planes a block: the halo of the
// widest channel group, then the weights (all 27 taps of a group when
// resident, else three stages)
size_t conv3_tc_smem(int cin, int cout, bool resident, int zt) {
  const int cg = std::min(cin, TC_CG);
  return (size_t)(cg / 8) * TC_PLANE * (zt + 2) + (size_t)(resident ? 27 : TC_STAGES) * cout * cg * 2 + 64;
}
constexpr size_t kTcSmemMax = 200 * 1024;

bool conv3_tc_ok(const stp_unet* n, const Dims& dm, int ldx, int cin, int cout, int ldy) {
  return n->use_tc && dm.w % TC_TX == 0 && dm.h % TC_TY == 0 && cin % 16 == 0 && cout % 16 == 0 && cout <= 256 &&
         ldx % 8 == 0 && ldy % 8 == 0 && conv3_tc_smem(cin, cout, false, 1) <= kTcSmemMax;
}

// planes a block of k_conv3_tc computes (measured on GB300 over the
// network's layer shapes): 4 when the block stays within 64 KB of shared
// memory (four blocks an SM) and the layer still has 1024 blocks; else 2
// when it fits and leaves 512 blocks; else 1.  Always a divisor of the depth,
// accumulators within 128 tensor-memory columns, and resident weights.  A
// forced count (STP_UNET_TC_PLANES: 1, 2 or 4) is halved until it is valid.
int conv3_tc_planes(const stp_unet* n, const Dims& dm, int cin, int cout, bool resident) {
  if (!resident) return 1;
  const long long tiles = dm.vox() / (TC_TX * TC_TY);
  auto fits = [&](int zt, size_t smem_max, long long min_blocks) {
    return dm.d % zt == 0 && zt * cout <= 128 && conv3_tc_smem(cin, cout, true, zt) <= smem_max &&
           tiles / zt >= min_blocks;
  };
  if (n->tc_planes == 1 || n->tc_planes == 2 || n->tc_planes == 4) {
    for (int zt = n->tc_planes; zt > 1; zt /= 2)
      if (fits(zt, kTcSmemMax, 1)) return zt;
    return 1;
  }
  if (fits(4, 64 * 1024, 1024)) return 4;
  if (fits(2, kTcSmemMax, 512)) return 2;
  return 1;
}

// launch a 3x3x3 convolution (forward form): tcgen05 where the shapes allow, else mma.sync
int conv3(stp_unet* n, const Dims& dm, const bf16* x, int ldx, int cin, const bf16* wt, const bf16* wimg,
          const float* bias, int cout, bf16* y, int ldy, int relu, const bf16* mask, int ldm) {
  const long long V = dm.vox();
  if (conv3_tc_ok(n, dm, ldx, cin, cout, ldy)) {
    static std::atomic<unsigned> done{0u};
    UTRY(n, smem_limit_once(k_conv3_tc, (int)kTcSmemMax, done));
    const bool resident = conv3_tc_smem(cin, cout, true, 1) <= kTcSmemMax;
    const int zt = conv3_tc_planes(n, dm, cin, cout, resident);
    const unsigned blocks = (unsigned)(V / (TC_TX * TC_TY * zt));
    k_conv3_tc<<<blocks, 128, conv3_tc_smem(cin, cout, resident, zt), n->st>>>(
        dm, x, ldx, cin, wt, bias, cout, y, ldy, relu, mask, ldm, resident ? 1 : 0, zt, resident ? wimg : nullptr,
        n->d_err);
    UTRY(n, cudaGetLastError());
    return STP_OK;
  }
  // output channels a block: 64, 32, 16 or 8, the widest that still gives two
  // blocks an SM (small levels have few 128-voxel rows); each output sees the
  // same sequence of MMAs whichever width computes it (STP_UNET_MMA_NT =
  // 8, 4, 2 or 1 forces a width where the channel count allows it)
  const unsigned gx = (unsigned)((V + 127) / 128);
  const long long enough = 2LL * 152;
  int nt = n->mma_nt;
  if (nt != 8 && nt != 4 && nt != 2 && nt != 1) {
    nt = 1;
    for (int c = 8; c > 1; c /= 2)
      if (cout % (8 * c) == 0 && (long long)gx * (cout / (8 * c)) >= enough) {
        nt = c;
        break;
      }
    if (nt == 1 && (long long)gx * ((cout + 15) / 16) >= enough) nt = 2;
  }
  if (nt == 8 && cout % 64) nt = 4;
  if (nt == 4 && cout % 32) nt = 2;
  switch (nt) {
    case 8:
      k_conv3<8><<<dim3(gx, cout / 64), 128, 0, n->st>>>(dm, x, ldx, cin, wt, bias, cout, y, ldy, relu, mask, ldm);
      break;
    case 4:
      k_conv3<4><<<dim3(gx, cout / 32), 128, 0, n->st>>>(dm, x, ldx, cin, wt, bias, cout, y, ldy, relu, mask, ldm);
      break;
    case 2:
      k_conv3<2><<<dim3(gx, (cout + 15) / 16), 128, 0, n->st>>>(dm, x, ldx, cin, wt, bias, cout, y, ldy, relu, mask,
                                                                 ldm);
      break;
    default:
      k_conv3<1><<<dim3(gx, (cout + 7) / 8), 128, 0, n->st>>>(dm, x, ldx, cin, wt, bias, cout, y, ldy, relu, mask,
                                                               ldm);
  }
  UTRY(n, cudaGetLastError());
  return STP_OK;
}

int wgrad3(stp_unet* n, const Dims& dm, const bf16* x, int ldx, int cin, const bf16* gz, int ldg, int cout,
           const Layer& ly) {
  const long long V = dm.vox();
  const int tiles = 27 * ((cin + 31) / 32) * (cout / 16);
  long long splits = std::max<long long>(1, std::min<long long>((152LL * 16) / tiles + 1, (V + 63) / 64));
  long long chunk = (V + splits - 1) / splits;
  chunk = ((chunk + 63) / 64) * 64;
  splits = (V + chunk - 1) / chunk;
  k_wgrad3<<<dim3(tiles, (unsigned)splits), 128, 0, n->st>>>(dm, x, ldx, cin, gz, ldg, cout, n->grad + ly.woff,
                                                             nullptr, chunk);
  UTRY(n, cudaGetLastError());
  const int bx = (int)std::min<long long>(V, 1024);
  k_bias_grad<<<dim3(bx, (cout + 127) / 128), 128, 0, n->st>>>(V, gz, ldg, cout, n->grad + ly.boff);
  UTRY(n, cudaGetLastError());
  return STP_OK;
}

int pack_all(stp_unet* n) {
  for (size_t i = 0; i < n->L.size(); i++) {
    Layer& ly = n->L[i];
    if (ly.taps != 27 || ly.cin == 1) continue;
    const long long tot = (long long)ly.cout * ly.cin * 27;
    k_pack_weights<<<blocks_for(tot), 256, 0, n->st>>>(n->theta + ly.woff, ly.cout, ly.cin, ly.wt, ly.wtt);
    UTRY(n, cudaGetLastError());
    if (ly.img) k_pack_image<<<blocks_for(tot / 8), 256, 0, n->st>>>(ly.wt, ly.cin, ly.cout, ly.img);
    if (ly.timg) k_pack_image<<<blocks_for(tot / 8), 256, 0, n->st>>>(ly.wtt, ly.cout, ly.cin, ly.timg);
    UTRY(n, cudaGetLastError());
  }
  return STP_OK;
}

// forward of nb samples; x [nb][D][H][W] FP32 on the device
int forward(stp_unet* n, const float* x, int nb) {
  Dims dm[4];
  for (int l = 0; l < 4; l++) dm[l] = Dims{nb, n->dm[l].d, n->dm[l].h, n->dm[l].w};
  int rc;
  // encoder
  const Layer* P = n->L.data();
  // level 1: input layer, second conv writes e1 into u[0][:, 32:48]
  k_conv_in<<<blocks_for(dm[0].vox()), 256, 0, n->st>>>(dm[0], x, n->theta + P[0].woff, n->theta + P[0].boff, n->ha[0],
                                                         16);
  UTRY(n, cudaGetLastError());
  const bf16* in = nullptr;
  int ldin = 0;
  for (int l = 0; l < 4; l++) {
    const int c = kCh[l];
    const Layer& la = P[2 * l];
    const Layer& lb = P[2 * l + 1];
    if (l > 0) {
      if ((rc = conv3(n, dm[l], in, ldin, la.cin, la.wt, la.img, n->theta + la.boff, c, n->ha[l], c, 1, nullptr, 0))) return rc;
    }
    bf16* e = l < 3 ? n->u[l] + kCh[l + 1] : n->e4;
    const int lde = l < 3 ? cu_width(l) : c;
    if ((rc = conv3(n, dm[l], n->ha[l], c, c, lb.wt, lb.img, n->theta + lb.boff, c, e, lde, 1, nullptr, 0))) return rc;
    if (l < 3) {
      k_pool<<<dim3(blocks_for(dm[l + 1].vox()), c / 8), 256, 0, n->st>>>(dm[l], e, lde, c, n->q[l], c);
      UTRY(n, cudaGetLastError());
      in = n->q[l];
      ldin = c;
    }
  }
  // decoder
  const bf16* deeper = n->e4;
  int cdeep = kCh[3];
  for (int l = 2; l >= 0; l--) {
    const int c = kCh[l], cw = cu_width(l);
    k_upsample<<<blocks_for(dm[l].vox()), 256, 0, n->st>>>(dm[l + 1], deeper, cdeep, cdeep, n->u[l], cw);
    UTRY(n, cudaGetLastError());
    const Layer& la = P[8 + 2 * (2 - l)];
    const Layer& lb = P[9 + 2 * (2 - l)];
    if ((rc = conv3(n, dm[l], n->u[l], cw, cw, la.wt, la.img, n->theta + la.boff, c, n->hd[l], c, 1, nullptr, 0))) return rc;
    if ((rc = conv3(n, dm[l], n->hd[l], c, c, lb.wt, lb.img, n->theta + lb.boff, c, n->d[l], c, 1, nullptr, 0))) return rc;
    deeper = n->d[l];
    cdeep = c;
  }
  const Layer& lo = P[14];
  k_conv_out<<<blocks_for(dm[0].vox()), 256, 0, n->st>>>(dm[0].vox(), n->d[0], 16, n->theta + lo.woff,
                                                          n->theta + lo.boff, n->y);
  UTRY(n, cudaGetLastError());
  return STP_OK;
}

// backward from gy (FP32 [V0]) into n->grad (zeroed here)
int backward(stp_unet* n, const float* x, int nb) {
  Dims dm[4];
  for (int l = 0; l < 4; l++) dm[l] = Dims{nb, n->dm[l].d, n->dm[l].h, n->dm[l].w};
  const Layer* P = n->L.data();
  int rc;
  UTRY(n, cudaMemsetAsync(n->grad, 0, sizeof(float) * n->np, n->st));
  // output layer -> gradient of the pre-activation of d1 (ga[0])
  const Layer& lo = P[14];
  k_conv_out_bwd<<<blocks_for(dm[0].vox()), 256, 0, n->st>>>(dm[0].vox(), n->gy, n->d[0], 16, n->theta + lo.woff,
                                                              n->ga[0], 16, n->grad + lo.woff, n->grad + lo.boff);
  UTRY(n, cudaGetLastError());
  // decoder, level 0 up to 2; ga[l] holds the gradient of d_l's pre-activation
  for (int l = 0; l <= 2; l++) {
    const int c = kCh[l], cw = cu_width(l);
    const Layer& la = P[8 + 2 * (2 - l)];
    const Layer& lb = P[9 + 2 * (2 - l)];
    // conv b: input hd[l], gradient ga[l]
    if ((rc = wgrad3(n, dm[l], n->hd[l], c, c, n->ga[l], c, c, lb))) return rc;
    if ((rc = conv3(n, dm[l], n->ga[l], c, c, lb.wtt, lb.timg, nullptr, c, n->gb[l], c, 0, n->hd[l], c))) return rc;
    // conv a: input u[l], gradient gb[l]
    if ((rc = wgrad3(n, dm[l], n->u[l], cw, cw, n->gb[l], c, c, la))) return rc;
    if ((rc = conv3(n, dm[l], n->gb[l], c, c, la.wtt, la.timg, nullptr, cw, n->gu[l], cw, 0, nullptr, 0))) return rc;
    // upsample part -> gradient of the deeper level's output pre-activation
    const int cd = kCh[l + 1];
    const bf16* act = l < 2 ? n->d[l + 1] : n->e4;
    bf16* out = l < 2 ? n->ga[l + 1] : n->ga[3];
    k_upsample_bwd_mask<<<dim3(blocks_for(dm[l + 1].vox()), cd / 8), 256, 0, n->st>>>(dm[l + 1], n->gu[l], cw, cd, act, cd, out,
                                                                              cd);
    UTRY(n, cudaGetLastError());
  }
  // encoder, level 3 down to 0.  Buffers at level l: gz (gradient of e_l's
  // pre-activation), gha (of ha_l's), gq (of q_{l-1}, handed to level l-1).
  //   l = 3: gz = ga[3] (from the decoder), gha = gb[3], gq = ga[3]
  //   l < 3: gz = gb[l], gha = ga[l], gq = gb[l]
  // each is overwritten only after its last reader has run.
  const bf16* gq_in = nullptr;
  for (int l = 3; l >= 0; l--) {
    const int c = kCh[l];
    const Layer& la = P[2 * l];
    const Layer& lb = P[2 * l + 1];
    bf16* gz = l == 3 ? n->ga[3] : n->gb[l];
    if (l < 3) {
      // gz = (pool backward of the gradient of q_l + skip gradient) * (e_l > 0)
      const bf16* e = n->u[l] + kCh[l + 1];
      k_pool_bwd_add_mask<<<blocks_for(dm[l].vox()), 256, 0, n->st>>>(dm[l], gq_in, c, n->gu[l] + kCh[l + 1],
                                                                            cu_width(l), c, e, cu_width(l), gz, c);
      UTRY(n, cudaGetLastError());
    }
    // conv b: input ha[l]
    if ((rc = wgrad3(n, dm[l], n->ha[l], c, c, gz, c, c, lb))) return rc;
    bf16* gha = l == 3 ? n->gb[3] : n->ga[l];
    if ((rc = conv3(n, dm[l], gz, c, c, lb.wtt, lb.timg, nullptr, c, gha, c, 0, n->ha[l], c))) return rc;
    if (l > 0) {
      // conv a: input q[l-1]
      const int cp = kCh[l - 1];
      if ((rc = wgrad3(n, dm[l], n->q[l - 1], cp, cp, gha, c, c, la))) return rc;
      bf16* gq = l == 3 ? n->ga[3] : n->gb[l];
      if ((rc = conv3(n, dm[l], gha, c, c, la.wtt, la.timg, nullptr, cp, gq, cp, 0, nullptr, 0))) return rc;
      gq_in = gq;
    } else {
      // conv a of level 1: the network input (1 channel)
      k_wgrad_in<<<dim3((unsigned)std::min<long long>(152 * 2, (dm[0].vox() + 255) / 256), 27), 256, 0, n->st>>>(
          dm[0], x, gha, c, n->grad + la.woff);
      UTRY(n, cudaGetLastError());
      const int bx = (int)std::min<long long>(dm[0].vox(), 1024);
      k_bias_grad<<<dim3(bx, 1), 128, 0, n->st>>>(dm[0].vox(), gha, c, c, n->grad + la.boff);
      UTRY(n, cudaGetLastError());
    }
  }
  return STP_OK;
}

int check_n(stp_unet* n, int nb) {
  if (nb < 1 || nb > n->nmax) return ufail(n, STP_EINVAL, "batch size out of range");
  return STP_OK;
}

}  // namespace

namespace stp {

bool unet_matches(const stp_unet* n, int nz, int ny, int nx) {
  return n && n->dm[0].d == nz && n->dm[0].h == ny && n->dm[0].w == nx;
}

// d = s U(r / s) for one sample on stream st, s = norm / sqrt(V) with the
// norm read on the device; launches only (no synchronisation), so it can be
// captured into a graph.  Returns the number of kernels through *kernels.
int unet_guess(stp_unet* n, const float* r, const double* norm, float* d, cudaStream_t st, int* kernels) {
  cudaStream_t keep = n->st;
  n->st = st;
  const long long V = n->dm[0].vox() / n->nmax;
  int rc = STP_OK;
  k_guess_in<<<blocks_for(V), 256, 0, st>>>(V, r, norm, n->xin);
  if (cudaGetLastError() != cudaSuccess) rc = STP_ECUDA;
  if (rc == STP_OK) rc = forward(n, n->xin, 1);
  if (rc == STP_OK) {
    k_guess_out<<<blocks_for(V), 256, 0, st>>>(V, n->y, norm, n->out_scale, d);
    if (cudaGetLastError() != cudaSuccess) rc = STP_ECUDA;
  }
  n->st = keep;
  // scale in and out + the forward pass: input layer, 7 further encoder
  // convolutions, 3 pools, 3 upsamplings, 6 decoder convolutions, output layer
  if (kernels) *kernels = 2 + 21;
  return rc;
}

}  // namespace stp

extern "C" {

long long stp_unet_param_count(void) {
  long long np = 0;
  int cin = 1;
  for (int l = 0; l < 4; l++) {
    np += 27LL * cin * kCh[l] + kCh[l] + 27LL * kCh[l] * kCh[l] + kCh[l];
    cin = kCh[l];
  }
  for (int l = 2; l >= 0; l--) np += 27LL * cu_width(l) * kCh[l] + kCh[l] + 27LL * kCh[l] * kCh[l] + kCh[l];
  return np + 16 + 1;
}

int stp_unet_create(int nmax, int nz, int ny, int nx, void* stream, stp_unet** out) {
  if (!out) return STP_EINVAL;
  *out = nullptr;
  if (nmax < 1 || nz < 8 || ny < 8 || nx < 8 || nz % 8 || ny % 8 || nx % 8) return STP_EINVAL;
  if ((double)nmax * nz * ny * nx > 2147483647.0) return STP_EINVAL;  // voxel indices are 32-bit
  stp_unet* n = new stp_unet();
  n->nmax = nmax;
  for (int l = 0; l < 4; l++) n->dm[l] = Dims{nmax, nz >> l, ny >> l, nx >> l};
  if (stream) {
    n->st = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&n->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete n;
      return STP_ECUDA;
    }
    n->own_stream = true;
  }
  // layers in parameter order
  long long q = 0;
  auto add = [&](int ci, int co, int taps) {
    Layer ly;
    ly.cin = ci;
    ly.cout = co;
    ly.taps = taps;
    ly.woff = q;
    q += (long long)co * ci * taps;
    ly.boff = q;
    q += co;
    n->L.push_back(ly);
  };
  int cin = 1;
  for (int l = 0; l < 4; l++) {
    add(cin, kCh[l], 27);
    add(kCh[l], kCh[l], 27);
    cin = kCh[l];
  }
  for (int l = 2; l >= 0; l--) {
    add(cu_width(l), kCh[l], 27);
    add(kCh[l], kCh[l], 27);
  }
  add(16, 1, 1);
  n->np = q;
  int rc = STP_OK;
  auto A = [&](auto** p, size_t count) {
    if (rc == STP_OK) rc = ualloc(n, p, count);
  };
  A(&n->theta, n->np);
  A(&n->grad, n->np);
  A(&n->m, n->np);
  A(&n->v, n->np);
  // elements of the resident-weight image of a convolution cin -> cout, 0
  // where k_conv3_tc would stream its weights (or not run at all)
  auto image_elems = [](int ci, int co) -> size_t {
    if (ci % 16 || co % 16 || co > 256 || conv3_tc_smem(ci, co, true, 1) > kTcSmemMax) return 0;
    return (size_t)((ci + TC_CG - 1) / TC_CG) * 27 * co * std::min(ci, TC_CG);
  };
  for (Layer& ly : n->L) {
    if (ly.taps == 27 && ly.cin > 1) {
      A(&ly.wt, (size_t)ly.cout * ly.cin * 27);
      A(&ly.wtt, (size_t)ly.cout * ly.cin * 27);
      if (const size_t e = image_elems(ly.cin, ly.cout)) A(&ly.img, e);
      if (const size_t e = image_elems(ly.cout, ly.cin)) A(&ly.timg, e);
    }
  }
  const long long V[4] = {n->dm[0].vox(), n->dm[1].vox(), n->dm[2].vox(), n->dm[3].vox()};
  for (int l = 0; l < 4; l++) {
    A(&n->ha[l], (size_t)V[l] * kCh[l]);
    A(&n->ga[l], (size_t)V[l] * kCh[l]);
    A(&n->gb[l], (size_t)V[l] * kCh[l]);
  }
  A(&n->e4, (size_t)V[3] * kCh[3]);
  for (int l = 0; l < 3; l++) {
    A(&n->u[l], (size_t)V[l] * cu_width(l));
    A(&n->gu[l], (size_t)V[l] * cu_width(l));
    A(&n->q[l], (size_t)V[l + 1] * kCh[l]);
    A(&n->hd[l], (size_t)V[l] * kCh[l]);
    A(&n->d[l], (size_t)V[l] * kCh[l]);
  }
  A(&n->y, (size_t)V[0]);
  A(&n->xin, (size_t)V[0]);
  A(&n->tin, (size_t)V[0]);
  A(&n->snorm, (size_t)nmax);
  A(&n->gy, (size_t)V[0]);
  A(&n->loss, 1);
  A(&n->d_err, 1);
  if (const char* e = std::getenv("STP_UNET_TC")) n->use_tc = std::atoi(e) != 0;
  if (const char* e = std::getenv("STP_UNET_TC_PLANES")) n->tc_planes = std::atoi(e);
  if (const char* e = std::getenv("STP_UNET_MMA_NT")) n->mma_nt = std::atoi(e);
  if (rc == STP_OK && cudaMallocHost((void**)&n->h_loss, sizeof(float)) != cudaSuccess) rc = STP_ENOMEM;
  if (rc == STP_OK) {
    cudaMemsetAsync(n->theta, 0, sizeof(float) * n->np, n->st);
    cudaMemsetAsync(n->m, 0, sizeof(float) * n->np, n->st);
    cudaMemsetAsync(n->v, 0, sizeof(float) * n->np, n->st);
    cudaMemsetAsync(n->d_err, 0, sizeof(int), n->st);
    if (cudaStreamSynchronize(n->st) != cudaSuccess) rc = STP_ECUDA;
  }
  if (rc != STP_OK) {
    stp_unet_destroy(n);
    return rc;
  }
  *out = n;
  return STP_OK;
}

void stp_unet_destroy(stp_unet* n) {
  if (!n) return;
  if (n->st) cudaStreamSynchronize(n->st);
  for (void* p : n->allocs) cudaFree(p);
  if (n->h_loss) cudaFreeHost(n->h_loss);
  if (n->own_stream && n->st) cudaStreamDestroy(n->st);
  delete n;
}

const char* stp_unet_last_error(const stp_unet* n) { return n ? n->err.c_str() : ""; }

int stp_unet_set_params(stp_unet* n, const float* theta, int where) {
  if (!n || !theta) return STP_EINVAL;
  UTRY(n, cudaMemcpyAsync(n->theta, theta, sizeof(float) * n->np,
                          where == STP_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, n->st));
  UTRY(n, cudaMemsetAsync(n->m, 0, sizeof(float) * n->np, n->st));
  UTRY(n, cudaMemsetAsync(n->v, 0, sizeof(float) * n->np, n->st));
  n->adam_step = 0;
  int rc = pack_all(n);
  if (rc) return rc;
  UTRY(n, cudaStreamSynchronize(n->st));
  return STP_OK;
}

int stp_unet_get_params(stp_unet* n, float* theta, int where) {
  if (!n || !theta) return STP_EINVAL;
  UTRY(n, cudaMemcpyAsync(theta, n->theta, sizeof(float) * n->np,
                          where == STP_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, n->st));
  UTRY(n, cudaStreamSynchronize(n->st));
  return STP_OK;
}

int stp_unet_forward(stp_unet* n, const float* x, float* y, int nb) {
  if (!n || !x || !y) return STP_EINVAL;
  if (int rc = check_n(n, nb)) return rc;
  int rc = forward(n, x, nb);
  if (rc) return rc;
  UTRY(n, cudaMemcpyAsync(y, n->y, sizeof(float) * n->dm[0].vox() / n->nmax * nb, cudaMemcpyDeviceToDevice, n->st));
  UTRY(n, cudaStreamSynchronize(n->st));
  return check_tc_timeout(n);
}

int stp_unet_gradient(stp_unet* n, const float* x, const float* target, int nb, float* grad, float* loss) {
  if (!n || !x || !target) return STP_EINVAL;
  if (int rc = check_n(n, nb)) return rc;
  int rc = forward(n, x, nb);
  if (rc) return rc;
  const long long V = n->dm[0].vox() / n->nmax * nb;
  UTRY(n, cudaMemsetAsync(n->loss, 0, sizeof(float), n->st));
  k_mse<<<blocks_for(V), 256, 0, n->st>>>(V, n->y, target, n->gy, n->loss);
  UTRY(n, cudaGetLastError());
  if ((rc = backward(n, x, nb))) return rc;
  if (grad) UTRY(n, cudaMemcpyAsync(grad, n->grad, sizeof(float) * n->np, cudaMemcpyDeviceToDevice, n->st));
  UTRY(n, cudaMemcpyAsync(n->h_loss, n->loss, sizeof(float), cudaMemcpyDeviceToHost, n->st));
  UTRY(n, cudaStreamSynchronize(n->st));
  if (loss) *loss = *n->h_loss;
  return check_tc_timeout(n);
}

int stp_unet_train_step(stp_unet* n, const float* x, const float* target, int nb, float lr, float* loss) {
  int rc = stp_unet_gradient(n, x, target, nb, nullptr, loss);
  if (rc) return rc;
  n->adam_step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)n->adam_step), c2 = 1.f - std::pow(b2, (float)n->adam_step);
  k_adam<<<blocks_for(n->np), 256, 0, n->st>>>(n->np, n->theta, n->grad, n->m, n->v, lr, b1, b2, 1e-8f, c1, c2);
  UTRY(n, cudaGetLastError());
  if ((rc = pack_all(n))) return rc;
  UTRY(n, cudaStreamSynchronize(n->st));
  return STP_OK;
}

int stp_unet_layer(stp_unet* n, int layer, int mode, const float* a, const float* b, float* out, int nb) {
  if (!n || !a || !out) return STP_EINVAL;
  if (int rc = check_n(n, nb)) return rc;
  if (layer < 0 || layer > 13) return ufail(n, STP_EINVAL, "layer must be 0..13 (the 3x3x3 convolutions)");
  if (mode < 0 || mode > 2 || (mode == 1 && layer == 0)) return ufail(n, STP_EINVAL, "bad mode for this layer");
  if (mode == 2 && !b) return ufail(n, STP_EINVAL, "the weight gradient needs gz");
  const Layer& ly = n->L[layer];
  const int lev = layer < 8 ? layer / 2 : 2 - (layer - 8) / 2;
  const Dims dm{nb, n->dm[lev].d, n->dm[lev].h, n->dm[lev].w};
  const long long V = dm.vox();
  const int ci = ly.cin, co = ly.cout;
  // temporaries: BF16 copies of the inputs and the BF16 output
  bf16 *xa = nullptr, *xb = nullptr, *y = nullptr;
  std::vector<void*> tmp;
  auto talloc = [&](bf16** p, long long count) -> int {
    if (cudaMalloc((void**)p, sizeof(bf16) * std::max<long long>(count, 1)) != cudaSuccess) return STP_ENOMEM;
    tmp.push_back(*p);
    return STP_OK;
  };
  auto done = [&](int rc) {
    cudaStreamSynchronize(n->st);
    for (void* p : tmp) cudaFree(p);
    return rc;
  };
  int rc = STP_OK;
  if (mode == 0) {
    if (layer == 0) {
      if ((rc = talloc(&y, V * co))) return done(ufail(n, rc, "cudaMalloc failed"));
      k_conv_in<<<blocks_for(V), 256, 0, n->st>>>(dm, a, n->theta + ly.woff, n->theta + ly.boff, y, co);
      if (cudaGetLastError() != cudaSuccess) return done(ufail(n, STP_ECUDA, "k_conv_in launch failed"));
    } else {
      if ((rc = talloc(&xa, V * ci)) || (rc = talloc(&y, V * co))) return done(ufail(n, rc, "cudaMalloc failed"));
      k_to_bf16<<<blocks_for(V * ci), 256, 0, n->st>>>(V * ci, a, xa);
      if ((rc = conv3(n, dm, xa, ci, ci, ly.wt, ly.img, n->theta + ly.boff, co, y, co, 1, nullptr, 0)))
        return done(rc);
    }
    k_from_bf16<<<blocks_for(V * co), 256, 0, n->st>>>(V * co, y, out);
  } else if (mode == 1) {
    if ((rc = talloc(&xa, V * co)) || (rc = talloc(&y, V * ci)) || (b && (rc = talloc(&xb, V * ci))))
      return done(ufail(n, rc, "cudaMalloc failed"));
    k_to_bf16<<<blocks_for(V * co), 256, 0, n->st>>>(V * co, a, xa);
    if (b) k_to_bf16<<<blocks_for(V * ci), 256, 0, n->st>>>(V * ci, b, xb);
    if ((rc = conv3(n, dm, xa, co, co, ly.wtt, ly.timg, nullptr, ci, y, ci, 0, xb, xb ? ci : 0))) return done(rc);
    k_from_bf16<<<blocks_for(V * ci), 256, 0, n->st>>>(V * ci, y, out);
  } else {
    UTRY(n, cudaMemsetAsync(n->grad + ly.woff, 0, sizeof(float) * ((long long)co * ci * 27 + co), n->st));
    if ((rc = talloc(&xb, V * co))) return done(ufail(n, rc, "cudaMalloc failed"));
    k_to_bf16<<<blocks_for(V * co), 256, 0, n->st>>>(V * co, b, xb);
    if (layer == 0) {
      k_wgrad_in<<<dim3((unsigned)std::min<long long>(152 * 2, (V + 255) / 256), 27), 256, 0, n->st>>>(
          dm, a, xb, co, n->grad + ly.woff);
      const int bx = (int)std::min<long long>(V, 1024);
      k_bias_grad<<<dim3(bx, 1), 128, 0, n->st>>>(V, xb, co, co, n->grad + ly.boff);
    } else {
      if ((rc = talloc(&xa, V * ci))) return done(ufail(n, rc, "cudaMalloc failed"));
      k_to_bf16<<<blocks_for(V * ci), 256, 0, n->st>>>(V * ci, a, xa);
      if ((rc = wgrad3(n, dm, xa, ci, ci, xb, co, co, ly))) return done(rc);
    }
    UTRY(n, cudaMemcpyAsync(out, n->grad + ly.woff, sizeof(float) * ((long long)co * ci * 27 + co),
                            cudaMemcpyDeviceToDevice, n->st));
  }
  if (cudaGetLastError() != cudaSuccess) return done(ufail(n, STP_ECUDA, "a layer-check kernel failed to launch"));
  if (cudaStreamSynchronize(n->st) != cudaSuccess) return done(ufail(n, STP_ECUDA, "layer check failed"));
  return done(check_tc_timeout(n));
}

int stp_unet_set_output_scale(stp_unet* n, float k) {
  if (!n || !(k > 0.f)) return STP_EINVAL;
  n->out_scale = k;
  return STP_OK;
}

int stp_unet_train_pairs(stp_unet* n, const float* r, const float* dp, int nb, float lr, float* loss) {
  if (!n || !r || !dp) return STP_EINVAL;
  if (int rc = check_n(n, nb)) return rc;
  const long long Vs = n->dm[0].vox() / n->nmax;
  UTRY(n, cudaMemsetAsync(n->snorm, 0, sizeof(float) * nb, n->st));
  k_sample_sumsq<<<dim3((unsigned)std::min<long long>(256, (Vs + 255) / 256), nb), 256, 0, n->st>>>(Vs, r, n->snorm);
  UTRY(n, cudaGetLastError());
  k_scale_pairs<<<blocks_for(Vs * nb), 256, 0, n->st>>>(Vs, nb, r, dp, n->snorm, n->out_scale, n->xin, n->tin);
  UTRY(n, cudaGetLastError());
  return stp_unet_train_step(n, n->xin, n->tin, nb, lr, loss);
}

int stp_unet_eval_pairs(stp_unet* n, const float* r, const float* dp, int nb, float* loss) {
  if (!n || !r || !dp) return STP_EINVAL;
  if (int rc = check_n(n, nb)) return rc;
  const long long Vs = n->dm[0].vox() / n->nmax;
  UTRY(n, cudaMemsetAsync(n->snorm, 0, sizeof(float) * nb, n->st));
  k_sample_sumsq<<<dim3((unsigned)std::min<long long>(256, (Vs + 255) / 256), nb), 256, 0, n->st>>>(Vs, r, n->snorm);
  UTRY(n, cudaGetLastError());
  k_scale_pairs<<<blocks_for(Vs * nb), 256, 0, n->st>>>(Vs, nb, r, dp, n->snorm, n->out_scale, n->xin, n->tin);
  UTRY(n, cudaGetLastError());
  int rc = forward(n, n->xin, nb);
  if (rc) return rc;
  UTRY(n, cudaMemsetAsync(n->loss, 0, sizeof(float), n->st));
  k_mse<<<blocks_for(Vs * nb), 256, 0, n->st>>>(Vs * nb, n->y, n->tin, n->gy, n->loss);
  UTRY(n, cudaGetLastError());
  UTRY(n, cudaMemcpyAsync(n->h_loss, n->loss, sizeof(float), cudaMemcpyDeviceToHost, n->st));
  UTRY(n, cudaStreamSynchronize(n->st));
  if (loss) *loss = *n->h_loss;
  return check_tc_timeout(n);
}

}  // extern "C"
