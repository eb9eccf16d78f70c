// Host side of the C ABI (include/stp.h): handle, device buffers, metrics,
// the SRJ schedule, and the drivers of the projection step and of the
// pressure solve.  Every kernel lives in kernels_step.cu / kernels_poisson.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "stp_internal.cuh"

using namespace stp;

namespace {

thread_local std::string g_init_error;

// stp_poisson_solve: |sum rhs dV| above this fraction of sum |rhs| dV is a
// right-hand side without a solution (round-off of an exactly telescoping
// divergence stays many orders below it)
constexpr double kMeanTol = 1e-9;

}  // namespace

struct stp_handle {
  stp_config cfg{};
  int prec = 0;
  int dev = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int nx = 0, ny = 0, nz = 0;
  size_t nc = 0, nw = 0, nplane = 0;
  size_t esz = 8;

  double* m64 = nullptr;
  float* m32 = nullptr;
  Geom<double> g64{};
  Geom<float> g32{};

  void *u = nullptr, *v = nullptr, *w = nullptr;
  void *ru = nullptr, *rv = nullptr, *rw = nullptr;
  void *tu = nullptr, *tv = nullptr, *tw = nullptr;
  void *Nu[3] = {}, *Nv[3] = {}, *Nw[3] = {};
  void* nu = nullptr;
  double* b = nullptr;
  double *p = nullptr, *p2 = nullptr;
  float *d1 = nullptr, *d2 = nullptr, *r32 = nullptr;
  double* stage = nullptr;
  // the fields before the current step, restored when the step diverges
  void *bu = nullptr, *bv = nullptr, *bw = nullptr;
  double* bp = nullptr;
  void* cn_scr = nullptr;  // z-line Crank-Nicolson: the columns' 1/pivots, or (c', d') pairs of tall columns

  Red red{};
  double* h_sc = nullptr;  // pinned copies of red.sc and red.flag
  int* h_flag = nullptr;

  std::vector<double> omega;
  int cn_sweeps = 0;
  int nhist = 0;
  long long step = 0;
  double last_dpdx = 0.0;
  std::vector<void*> allocs;
  std::string err;
  // accounting of the current API call
  long long launches = 0;     // kernels launched directly from the host
  long long solve_sweeps = 0;
  double solve_ms = 0.0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int* d_step = nullptr;       // steps since the fields were set (device copy)
  // device-steered pressure solve
  cudaStream_t cap = nullptr;  // private stream used only for graph capture
  SolveCtl* ctl = nullptr;
  SolveCtl* h_ctl = nullptr;   // pinned
  cudaGraph_t solve_graph = nullptr;
  cudaGraphExec_t solve_exec = nullptr;
  bool host_solve = false;     // STP_HOST_SOLVE=1: drive the solve from the host
  int cycle_blocks = 0;        // >0: FP32 cycles run as one persistent cooperative kernel
  int line_rb = 0;             // >0: FP32 z-line cycles run as one persistent kernel (tile rows)
  int line_variant = 0;        // FP32 z-line sweep kernel: 1 register-chunked columns, 0 shared-memory lock step
  int* line_flags = nullptr;   // its per-tile sweep counters
  int sweep_variant = -1;      // FP32 sweep kernel variant chosen by the autotuner (-1: not yet)
  float sweep_us = 0.f;        // its measured time per sweep
  float* d_omega32 = nullptr;  // the schedule on the device (FP32)
  GridBar bar{};
  // learned guess and training-pair harvest
  stp_unet* net = nullptr;
  int learned_mode = 0;        // 0: guess once per solve; 1: at every refinement pass / SRJ cycle
  int guess_kernels = 0;
  float *hr = nullptr, *hdp = nullptr;  // caller buffers for harvested pairs
  double* p_prev = nullptr;
  // LES statistics (stp_stats_*)
  double* st_mom = nullptr;   // [kStatMoments][nz] plane sums
  double* st_corr = nullptr;  // [3][nx] two-point product sums
  int st_kc = 0;
  long long st_n = 0;
};

namespace {

// true for the launch_* wrappers (each launches exactly one kernel)
constexpr bool is_launch(const char* s) {
  while (*s == ' ' || *s == '(') s++;
  return s[0] == 'l' && s[1] == 'a' && s[2] == 'u' && s[3] == 'n' && s[4] == 'c' && s[5] == 'h' && s[6] == '_';
}

int fail(stp_handle* h, int code, const std::string& msg) {
  if (h)
    h->err = msg;
  else
    g_init_error = msg;
  return code;
}

#define CUDA_TRY(h, call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (is_launch(#call)) h->launches++;                                                   \
    if (e_ != cudaSuccess)                                                                 \
      return fail(h, e_ == cudaErrorMemoryAllocation ? STP_ENOMEM : STP_ECUDA,             \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                     \
  } while (0)

int dalloc(stp_handle* h, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(h, STP_ENOMEM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes: " +
                                   cudaGetErrorString(e));
  }
  h->allocs.push_back(*p);
  return STP_OK;
}

// ---------------------------------------------------------------------------
// z grid and metrics (FP64 on the host)
// ---------------------------------------------------------------------------
struct ZGrid {
  std::vector<double> zf, zc, dz, hz, dzf;
};

ZGrid make_z(const stp_config& c) {
  ZGrid z;
  const int nz = c.nz;
  z.zf.resize(nz + 1);
  for (int k = 0; k <= nz; k++) {
    const double s = (double)k / nz;
    z.zf[k] = c.stretch > 0 ? 0.5 * c.Lz * (1.0 + std::tanh(c.stretch * (2.0 * s - 1.0)) / std::tanh(c.stretch))
                            : c.Lz * s;
  }
  z.zf[0] = 0.0;
  z.zf[nz] = c.Lz;
  z.dz.resize(nz);
  z.zc.resize(nz);
  for (int k = 0; k < nz; k++) {
    z.dz[k] = z.zf[k + 1] - z.zf[k];
    z.zc[k] = 0.5 * (z.zf[k] + z.zf[k + 1]);
  }
  z.hz.assign(nz + 1, 0.0);
  z.hz[0] = z.zc[0] - z.zf[0];
  z.hz[nz] = z.zf[nz] - z.zc[nz - 1];
  for (int k = 1; k < nz; k++) z.hz[k] = z.zc[k] - z.zc[k - 1];
  z.dzf.assign(nz + 1, 0.0);
  z.dzf[0] = z.dz[0];
  z.dzf[nz] = z.dz[nz - 1];
  for (int k = 1; k < nz; k++) z.dzf[k] = z.hz[k];
  return z;
}

// Poisson couplings in z: cup_k to k+1, cdn_k to k-1 (zero through the walls)
void poisson_z(const stp_config& c, const ZGrid& z, std::vector<double>& cup, std::vector<double>& cdn) {
  const int nz = c.nz;
  cup.assign(nz, 0.0);
  cdn.assign(nz, 0.0);
  for (int k = 0; k < nz; k++) {
    if (k < nz - 1) cup[k] = 1.0 / (z.hz[k + 1] * z.dz[k]);
    if (k > 0) cdn[k] = 1.0 / (z.hz[k] * z.dz[k]);
  }
}

// ---------------------------------------------------------------------------
// SRJ schedule (Sec. 3.4).  Eigenvalues mu of D^-1(-L) separate into Fourier
// modes in x, y and, for each x-y eigenvalue a, a symmetric generalized
// tridiagonal problem in z:  W(a - L_z) phi = mu W S phi, W = diag(dz).
// Its eigenvalues come from Sturm-sequence bisection.
// ---------------------------------------------------------------------------
struct Tridiag {
  std::vector<double> d, e;  // diagonal, off-diagonal of B^-1/2 A B^-1/2
};

Tridiag z_problem(const stp_config& c, const ZGrid& z, double a) {
  const int nz = c.nz;
  std::vector<double> cup, cdn;
  poisson_z(c, z, cup, cdn);
  const double dx = c.Lx / c.nx, dy = c.Ly / c.ny;
  Tridiag t;
  t.d.resize(nz);
  t.e.assign(nz > 1 ? nz - 1 : 0, 0.0);
  std::vector<double> B(nz);
  for (int k = 0; k < nz; k++) {
    const double S = 2.0 / (dx * dx) + 2.0 / (dy * dy) + cup[k] + cdn[k];
    B[k] = z.dz[k] * S;
    t.d[k] = z.dz[k] * (a + cup[k] + cdn[k]) / B[k];
  }
  for (int k = 0; k + 1 < nz; k++) t.e[k] = (-1.0 / z.hz[k + 1]) / std::sqrt(B[k] * B[k + 1]);
  return t;
}

// number of eigenvalues < x
int sturm_count(const Tridiag& t, double x) {
  int cnt = 0;
  double q = 1.0;
  for (size_t k = 0; k < t.d.size(); k++) {
    const double e2 = k ? t.e[k - 1] * t.e[k - 1] : 0.0;
    q = (t.d[k] - x) - (k ? e2 / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0) cnt++;
  }
  return cnt;
}

// m-th smallest eigenvalue (0-based)
double tri_eig(const Tridiag& t, int m) {
  double lo = 1e300, hi = -1e300;
  const size_t n = t.d.size();
  for (size_t k = 0; k < n; k++) {
    const double r = (k ? std::fabs(t.e[k - 1]) : 0.0) + (k + 1 < n ? std::fabs(t.e[k]) : 0.0);
    lo = std::min(lo, t.d[k] - r);
    hi = std::max(hi, t.d[k] + r);
  }
  for (int it = 0; it < 400 && hi - lo > 1e-17 * std::max(1.0, std::fabs(hi)); it++) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count(t, mid) > m)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}

void jacobi_bounds(const stp_config& c, double* mn, double* mx) {
  const ZGrid z = make_z(c);
  const double dx = c.Lx / c.nx, dy = c.Ly / c.ny;
  const double pi = 3.14159265358979323846;
  auto lx = [&](int m) { return 4.0 / (dx * dx) * std::pow(std::sin(pi * m / c.nx), 2); };
  auto ly = [&](int n) { return 4.0 / (dy * dy) * std::pow(std::sin(pi * n / c.ny), 2); };
  double lo = c.nz > 1 ? tri_eig(z_problem(c, z, 0.0), 1) : 1e300;
  if (c.nx > 1) lo = std::min(lo, tri_eig(z_problem(c, z, lx(1)), 0));
  if (c.ny > 1) lo = std::min(lo, tri_eig(z_problem(c, z, ly(1)), 0));
  *mn = lo;
  *mx = tri_eig(z_problem(c, z, lx(c.nx / 2) + ly(c.ny / 2)), c.nz - 1);
}

// z-line Jacobi: A = -L_z + dxy I shares its eigenvectors with -L (the
// Kronecker sum of -L_z and the periodic x-y operator), so the eigenvalues of
// A^-1(-L) are (tau + lam)/(tau + dxy): tau of -L_z (W(-L_z) phi = tau W phi,
// W = diag(dz), Sturm bisection), lam of the x-y operator.  The extremes over
// all pairs but the constant mode are at tau in {0, tau_1, tau_max} and lam in
// {0, lam_1, lam_max}.
void line_bounds(const stp_config& c, double* mn, double* mx) {
  const ZGrid z = make_z(c);
  const int nz = c.nz;
  std::vector<double> cup, cdn;
  poisson_z(c, z, cup, cdn);
  Tridiag t;
  t.d.resize(nz);
  t.e.assign(nz > 1 ? nz - 1 : 0, 0.0);
  for (int k = 0; k < nz; k++) t.d[k] = cup[k] + cdn[k];
  for (int k = 0; k + 1 < nz; k++) t.e[k] = (-1.0 / z.hz[k + 1]) / std::sqrt(z.dz[k] * z.dz[k + 1]);
  const double dx = c.Lx / c.nx, dy = c.Ly / c.ny;
  const double pi = 3.14159265358979323846;
  const double dxy = 2.0 / (dx * dx) + 2.0 / (dy * dy);
  const double lam1 = std::min(4.0 / (dx * dx) * std::pow(std::sin(pi / c.nx), 2),
                               4.0 / (dy * dy) * std::pow(std::sin(pi / c.ny), 2));
  const double lmax = 4.0 / (dx * dx) * std::pow(std::sin(pi * (c.nx / 2) / c.nx), 2) +
                      4.0 / (dy * dy) * std::pow(std::sin(pi * (c.ny / 2) / c.ny), 2);
  const double tau1 = nz > 1 ? tri_eig(t, 1) : 1e300, tmax = tri_eig(t, nz - 1);
  *mn = std::min(lam1 / dxy, nz > 1 ? tau1 / (tau1 + dxy) : 1e300);
  *mx = std::max(lmax / dxy, (tmax + lmax) / (tmax + dxy));
}

void solve_bounds(const stp_config& c, double* mn, double* mx) {
  if (c.zline)
    line_bounds(c, mn, mx);
  else
    jacobi_bounds(c, mn, mx);
}

double cycle_factor(double mn, double mx, int M) {
  const double x0 = (mx + mn) / (mx - mn);
  return 1.0 / std::cosh(M * std::acosh(x0));
}

// odd numbers 1..2M-1 in the recursive mirror-pair order (M a power of two)
std::vector<int> mirror_order(int M) {
  std::vector<int> th{1};
  for (int m = 1; m < M; m *= 2) {
    std::vector<int> nx;
    nx.reserve(2 * th.size());
    for (int t : th) {
      nx.push_back(t);
      nx.push_back(4 * m - t);
    }
    th.swap(nx);
  }
  return th;
}

std::vector<double> chebyshev(double mn, double mx, int M) {
  const double pi = 3.14159265358979323846;
  const double mid = 0.5 * (mx + mn), half = 0.5 * (mx - mn);
  std::vector<double> om;
  for (int t : mirror_order(M)) om.push_back(1.0 / (mid + half * std::cos(t * pi / (2.0 * M))));
  return om;
}

bool pow2(int m) { return m >= 1 && (m & (m - 1)) == 0; }

int auto_cycle(double mn, double mx) {
  int M = 2;
  while (M < 1024 && cycle_factor(mn, mx, M) > 0.01) M *= 2;
  return M;
}

// Crank-Nicolson Jacobi sweeps to the storage precision: the smallest count
// whose contraction reaches 1e-12 with FP64 fields, 2^-24 with FP32 fields
// (more sweeps cannot change what FP32 stores).  Point Jacobi contracts by
// hS/(1+hS) a sweep with S the largest diagonal weight; z-line Jacobi by the
// same bound with S the x-y coupling weights alone (the column matrix is an
// M-matrix whose row sums are at least 1 + h S_xy).  nu_T is bounded by 4 nu
// with LES.
int auto_cn_sweeps(const stp_config& c, const ZGrid& z) {
  const double dx = c.Lx / c.nx, dy = c.Ly / c.ny;
  double smax = 0.0;
  for (int k = 0; k < c.nz; k++) {
    const double sz = 2.0 / (z.dzf[k] * z.dz[k]) + 2.0 / (z.dzf[k + 1] * z.dz[k]);
    smax = std::max(smax, 4.0 / (dx * dx) + 4.0 / (dy * dy) + (c.cn_zline ? 0.0 : sz));
  }
  if (c.cn_zline) smax = 2.0 / (dx * dx) + 2.0 / (dy * dy);
  const double nu = c.nu * (c.les ? 4.0 : 1.0);
  const double hs = 0.5 * c.dt * nu * smax;
  const double rho = hs / (1.0 + hs);
  if (rho <= 0) return 1;
  const double target = c.precision == STP_FP32_REFINE ? std::ldexp(1.0, -24) : 1e-12;
  int k = (int)std::ceil(std::log(target) / std::log(rho));
  return std::max(c.cn_zline ? 1 : 2, std::min(k, 200));
}

int validate(const stp_config* c, std::string* why) {
  if (!c) return *why = "config is NULL", STP_EINVAL;
  if (c->nx < 3 || c->ny < 3 || c->nz < 2) return *why = "need nx, ny >= 3 and nz >= 2", STP_EINVAL;
  if ((double)c->nx * c->ny * (c->nz + 1) > 2.0e9) return *why = "grid too large (cells must fit a 31-bit index)", STP_EINVAL;
  if (!(c->Lx > 0 && c->Ly > 0 && c->Lz > 0)) return *why = "box lengths must be positive", STP_EINVAL;
  if (!(c->nu >= 0) || !(c->dt > 0)) return *why = "need nu >= 0 and dt > 0", STP_EINVAL;
  if (c->precision != STP_FP64 && c->precision != STP_FP32_REFINE) return *why = "unknown precision", STP_EINVAL;
  if (c->forcing != 0 && c->forcing != 1) return *why = "forcing must be 0 or 1", STP_EINVAL;
  if (c->stretch < 0) return *why = "stretch must be >= 0", STP_EINVAL;
  if (!(c->ptol >= 0) || c->pmaxit < 0 || c->cn_sweeps < 0) return *why = "bad solver limits", STP_EINVAL;
  if (c->srj_m < 0 || c->srj_m > 4096) return *why = "srj_m out of range", STP_EINVAL;
  if (c->srj_omega && c->srj_m <= 0) return *why = "srj_omega given without srj_m", STP_EINVAL;
  if (c->srj_m % 2) return *why = "the SRJ cycle length must be even", STP_EINVAL;
  if (c->zline != 0 && c->zline != 1) return *why = "zline must be 0 or 1", STP_EINVAL;
  if (c->cn_zline != 0 && c->cn_zline != 1) return *why = "cn_zline must be 0 or 1", STP_EINVAL;
  if (c->cn_zline && c->ny > 65535) return *why = "z-line Crank-Nicolson needs ny <= 65535 (one grid row a block row)", STP_EINVAL;
  if (!c->srj_omega && c->srj_m > 0 && !pow2(c->srj_m)) return *why = "library schedules need srj_m a power of two", STP_EINVAL;
  if (c->les && !(c->cs >= 0 && c->vd_a > 0 && c->re_tau > 0)) return *why = "bad LES constants", STP_EINVAL;
  return STP_OK;
}

template <typename T>
Geom<T> geom_from(const stp_handle* h, T* pack) {
  const int nz = h->nz, L = nz + 1;
  const double dx = h->cfg.Lx / h->nx, dy = h->cfg.Ly / h->ny;
  Geom<T> g;
  g.nx = h->nx;
  g.ny = h->ny;
  g.nz = nz;
  g.idx = (T)(1.0 / dx);
  g.idy = (T)(1.0 / dy);
  g.idx2 = (T)(1.0 / (dx * dx));
  g.idy2 = (T)(1.0 / (dy * dy));
  g.hidx = (T)(0.5 / dx);
  g.hidy = (T)(0.5 / dy);
  g.idxdy = (T)(1.0 / (dx * dy));
  g.idz = pack + 0 * L;
  g.ihz = pack + 1 * L;
  g.idzf = pack + 2 * L;
  g.i2dzc = pack + 3 * L;
  g.idzw = pack + 4 * L;
  g.cup = pack + 5 * L;
  g.cdn = pack + 6 * L;
  g.iS = pack + 7 * L;
  g.S = pack + 8 * L;
  g.lm2 = pack + 9 * L;
  g.dzv = pack + 10 * L;
  g.li = pack + 11 * L;
  g.lu = pack + 12 * L;
  g.tli = pack + 13 * L;
  g.tlf = pack + 14 * L;
  g.tlb = pack + 15 * L;
  // the packed level coefficients follow the kMetricArrays arrays (offset
  // 64 L bytes: 16-byte aligned)
  if constexpr (sizeof(T) == sizeof(float)) g.lz4 = reinterpret_cast<const float4*>(pack + kMetricArrays * L);
  else g.lz4 = nullptr;
  return g;
}

std::vector<double> metric_pack(const stp_config& c) {
  const int nz = c.nz, L = nz + 1;
  const ZGrid z = make_z(c);
  std::vector<double> cup, cdn;
  poisson_z(c, z, cup, cdn);
  const double dx = c.Lx / c.nx, dy = c.Ly / c.ny;
  std::vector<double> m((size_t)kMetricArrays * L, 0.0);
  for (int k = 0; k < nz; k++) {
    m[0 * L + k] = 1.0 / z.dz[k];
    const double up = (k < nz - 1) ? z.hz[k + 1] : z.dz[nz - 1];
    const double dn = (k > 0) ? z.hz[k] : z.dz[0];
    m[3 * L + k] = 1.0 / (up + dn);
    m[5 * L + k] = cup[k];
    m[6 * L + k] = cdn[k];
    const double S = 2.0 / (dx * dx) + 2.0 / (dy * dy) + cup[k] + cdn[k];
    m[7 * L + k] = 1.0 / S;
    m[8 * L + k] = S;
    const double delta = 2.0 * std::cbrt(dx * dy * z.dz[k]);
    const double d = std::min(z.zc[k], c.Lz - z.zc[k]);
    const double dplus = d * c.re_tau / (0.5 * c.Lz);
    const double phi = c.les ? 1.0 - std::exp(-dplus / c.vd_a) : 0.0;
    const double lm = c.cs * delta * phi;
    m[9 * L + k] = lm * lm;
    m[10 * L + k] = z.dz[k];
  }
  // z-line Thomas pivots of A = -L_z + dxy I: diagonal D_k = dxy + cup + cdn,
  // off-diagonals -cup (k+1) and -cdn (k-1).  One-sided (from the bottom
  // wall): m_k = D_k - cdn_k cup_{k-1}/m_{k-1}.  Twisted: those top-down
  // pivots for k < t, bottom-up pivots m'_k = D_k - cup_k cdn_{k+1}/m'_{k+1}
  // for k > t, and gamma_t = D_t - cdn_t cup_{t-1}/m_{t-1} -
  // cup_t cdn_{t+1}/m'_{t+1} at the twist level t = nz/2.
  {
    const double dxy = 2.0 / (dx * dx) + 2.0 / (dy * dy);
    const int t = nz / 2;
    std::vector<double> mt(nz), mb(nz);
    for (int k = 0; k < nz; k++) {
      mt[k] = dxy + cup[k] + cdn[k];
      if (k > 0) mt[k] -= cdn[k] * cup[k - 1] / mt[k - 1];
      m[11 * L + k] = 1.0 / mt[k];
      m[12 * L + k] = cup[k] / mt[k];
    }
    for (int k = nz - 1; k >= 0; k--) {
      mb[k] = dxy + cup[k] + cdn[k];
      if (k < nz - 1) mb[k] -= cup[k] * cdn[k + 1] / mb[k + 1];
    }
    for (int k = 0; k < nz; k++) {
      if (k < t) {
        m[13 * L + k] = 1.0 / mt[k];
        m[14 * L + k] = cdn[k] / mt[k];
        m[15 * L + k] = cup[k] / mt[k];
      } else if (k > t) {
        m[13 * L + k] = 1.0 / mb[k];
        m[14 * L + k] = cup[k] / mb[k];
        m[15 * L + k] = cdn[k] / mb[k];
      } else {
        double gam = dxy + cup[k] + cdn[k];
        if (k > 0) gam -= cdn[k] * cup[k - 1] / mt[k - 1];
        if (k < nz - 1) gam -= cup[k] * cdn[k + 1] / mb[k + 1];
        m[13 * L + k] = 1.0 / gam;
        m[14 * L + k] = cdn[k] / gam;
        m[15 * L + k] = cup[k] / gam;
      }
    }
  }
  for (int k = 0; k <= nz; k++) {
    m[1 * L + k] = (k >= 1 && k < nz) ? 1.0 / z.hz[k] : 0.0;
    m[2 * L + k] = 1.0 / z.dzf[k];
    m[4 * L + k] = (k >= 1 && k < nz) ? 1.0 / (z.dz[k] + z.dz[k - 1]) : 0.0;
  }
  return m;
}

int sync_scalars(stp_handle* h) {
  CUDA_TRY(h, cudaMemcpyAsync(h->h_sc, h->red.sc, sizeof(double) * SC_COUNT, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(h->h_flag, h->red.flag, sizeof(int) * FL_COUNT, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return STP_OK;
}

// ---------------------------------------------------------------------------
// Pressure solves (Sec. 3.4) as CUDA graphs steered from the device.
//   FP64: begin -> WHILE(loop) { check -> IF(body) { M sweeps } }
//   FP32: begin -> outer -> WHILE(pass) { d = 0 -> WHILE(loop) { check ->
//         IF(body) { M sweeps } } -> p += d -> outer }
// As in the oracle, each cycle first measures ||b - L p|| of its input and
// either stops (that input is the answer) or runs its M sweeps.  With M
// even the answer is always back in the first buffer, so the graphs are
// built once per handle.  On entry sc[SC_BNORM] = ||b||.
// ---------------------------------------------------------------------------
struct SolveOut {
  int sweeps = 0, passes = 0, converged = 0, bad = 0;
  double rel = 0.0;
  long long kernels = 0, tot_sweeps = 0;
  int nonconv = 0;
};

cudaGraphNode_t leaf_node(cudaGraph_t g) {
  size_t n = 0;
  cudaGraphGetNodes(g, nullptr, &n);
  std::vector<cudaGraphNode_t> v(n);
  cudaGraphGetNodes(g, v.data(), &n);
  for (cudaGraphNode_t x : v) {
    size_t d = 0;
    cudaGraphNodeGetDependentNodes(x, nullptr, nullptr, &d);
    if (d == 0) return x;
  }
  return nullptr;
}

// WHILE or IF node after `dep` in graph g; returns its body graph
int add_conditional(stp_handle* h, cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle hc,
                    cudaGraphConditionalNodeType type, cudaGraph_t* body, cudaGraphNode_t* node) {
  cudaGraphNodeParams prm = {};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = hc;
  prm.conditional.type = type;
  prm.conditional.size = 1;
  CUDA_TRY(h, cudaGraphAddNode(node, g, dep ? &dep : nullptr, nullptr, dep ? 1 : 0, &prm));
  *body = prm.conditional.phGraph_out[0];
  return STP_OK;
}

int begin_capture(stp_handle* h, cudaGraph_t g, cudaGraphNode_t dep) {
  CUDA_TRY(h, cudaStreamBeginCaptureToGraph(h->cap, g, dep ? &dep : nullptr, nullptr, dep ? 1 : 0,
                                            cudaStreamCaptureModeRelaxed));
  return STP_OK;
}
int end_capture(stp_handle* h, cudaGraph_t g) {
  cudaGraph_t out = g;
  CUDA_TRY(h, cudaStreamEndCapture(h->cap, &out));
  return STP_OK;
}

// FP32 cycles run as pair launches (two sweeps each) with the tuned variant
bool uses_pairs(const stp_handle* h) {
  return h->prec == STP_FP32_REFINE && h->cycle_blocks == 0 && !h->cfg.zline && sweep_variant_is_pair(h->sweep_variant) &&
         h->omega.size() % 4 == 0;
}

// the cycle: check -> IF { M sweeps }, inside the WHILE body `wb`
template <typename T>
int build_cycle(stp_handle* h, const Geom<T>& g, cudaGraph_t wb, cudaGraphConditionalHandle h_loop, T* A, T* B,
                const T* rhs, int mode) {
  cudaGraphConditionalHandle h_body;
  CUDA_TRY(h, cudaGraphConditionalHandleCreate(&h_body, wb, 0, cudaGraphCondAssignDefault));
  int rc;
  if ((rc = begin_capture(h, wb, nullptr))) return rc;
  CUDA_TRY(h, launch_check<T>(g, A, rhs, mode, h->ctl, h->red, 1, h_loop, h_body, h->cap));
  if ((rc = end_capture(h, wb))) return rc;
  cudaGraph_t ib;
  cudaGraphNode_t ifn;
  if ((rc = add_conditional(h, wb, leaf_node(wb), h_body, cudaGraphCondTypeIf, &ib, &ifn))) return rc;
  if ((rc = begin_capture(h, ib, nullptr))) return rc;
  const int M = (int)h->omega.size();
  if (sizeof(T) == sizeof(double) && h->net && h->learned_mode == 1) {
    // learned preconditioner in an FP64 solve: before every cycle's sweeps,
    // r = b - L p and p += s U(r / s)
    CUDA_TRY(h, launch_outer(h->g64, h->p, h->b, h->r32, h->ctl, h->red, 0, 0, 0, h->cap));
    if ((rc = unet_guess(h->net, h->r32, h->red.sc + SC_INNER_REF, h->d1, h->cap, &h->guess_kernels)))
      return fail(h, rc, "learned preconditioner: " + std::string(stp_unet_last_error(h->net)));
    CUDA_TRY(h, launch_addcorr(h->p, h->d1, h->nc, h->cap));
  }
  if (sizeof(T) == sizeof(float) && h->cycle_blocks > 0) {
    // the whole cycle in one persistent kernel
    CUDA_TRY(h, launch_cycle_f32(h->g32, (float*)A, (float*)B, (const float*)rhs, h->d_omega32, M, h->bar, h->ctl,
                                 h->cycle_blocks, h->cap));
    return end_capture(h, ib);
  }
  if (h->cfg.zline) {
    if (sizeof(T) == sizeof(float) && h->line_rb > 0) {
      CUDA_TRY(h, launch_line_cycle_f32(h->g32, h->line_rb, (float*)A, (float*)B, (const float*)rhs, h->d_omega32, M,
                                        h->line_flags, h->ctl, h->cap));
      return end_capture(h, ib);
    }
    for (int m = 0; m < M; m++)
      CUDA_TRY(h, launch_line_sweep<T>(g, (m % 2 == 0) ? A : B, rhs, (T)h->omega[m], (m % 2 == 0) ? B : A, h->cap,
                                       h->line_variant));
    return end_capture(h, ib);
  }
  if (sizeof(T) == sizeof(float) && uses_pairs(h)) {
    // two sweeps per launch: A -> B, B -> A, ... (M / 2 even: ends in A)
    for (int m = 0; m < M; m += 2) {
      const float* src = (const float*)((m % 4 == 0) ? A : B);
      float* dst = (float*)((m % 4 == 0) ? B : A);
      CUDA_TRY(h, launch_sweep_pair(h->g32, src, (const float*)rhs, (float)h->omega[m], (float)h->omega[m + 1], dst,
                                    h->cap));
    }
    return end_capture(h, ib);
  }
  for (int m = 0; m < M; m++) {
    const T* src = (m % 2 == 0) ? A : B;
    T* dst = (m % 2 == 0) ? B : A;
    CUDA_TRY(h, launch_sweep<T>(g, src, rhs, (T)h->omega[m], dst, h->cap));
  }
  return end_capture(h, ib);
}

// Time of one sweep of the FP32 variant currently set on this host thread,
// as the solve runs it: 20 sweeps (10 launches of a pair variant) captured
// into a graph (programmatic dependent launches between them), best of
// three launches after a warm-up launch, CUDA events on the handle's stream.
int time_sweeps(stp_handle* h, bool pair, float* us) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t x = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeRelaxed);
  const bool capturing = e == cudaSuccess;
  if (pair) {
    for (int w = 0; w < 10 && e == cudaSuccess; w++)
      e = launch_sweep_pair(h->g32, (w & 1) ? h->d2 : h->d1, h->r32, 1.0f, 1.0f, (w & 1) ? h->d1 : h->d2, h->cap);
  } else {
    for (int w = 0; w < 20 && e == cudaSuccess; w++)
      e = launch_sweep<float>(h->g32, (w & 1) ? h->d2 : h->d1, h->r32, 1.0f, (w & 1) ? h->d1 : h->d2, h->cap);
  }
  if (capturing) {
    const cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
  float best = 1e30f;
  for (int r = 0; r < 4 && e == cudaSuccess; r++) {
    float ms = 0.f;
    e = cudaEventRecord(h->ev0, h->st);
    if (e == cudaSuccess) e = cudaGraphLaunch(x, h->st);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev1, h->st);
    if (e == cudaSuccess) e = cudaEventSynchronize(h->ev1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    if (e == cudaSuccess && r > 0 && ms < best) best = ms;
  }
  if (x) cudaGraphExecDestroy(x);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(h, STP_ECUDA, std::string("sweep autotuner: ") + cudaGetErrorString(e));
  *us = best * 1e3f / 20.f;
  return STP_OK;
}

// Pick among timed variants: the lowest-numbered one within 2 % of the
// fastest (timing noise then does not flip the choice between near-equal
// tiles from run to run).
int pick_variant(const std::vector<std::pair<int, float>>& timed, float* us) {
  float best = 1e30f;
  for (const auto& t : timed) best = std::min(best, t.second);
  for (const auto& t : timed)
    if (t.second <= 1.02f * best) {
      *us = t.second;
      return t.first;
    }
  *us = 0.f;
  return 0;
}

// Autotuner of the FP32 sweep kernel: times every variant valid for this
// grid (time_sweeps, on the handle's own scratch buffers) and keeps the
// choice of pick_variant; cached per (device, nx, ny, nz).
// STP_SWEEP_VARIANT=<v> forces a variant.  All variants compute the same values.
int tune_sweep(stp_handle* h) {
  if (h->sweep_variant >= 0) return STP_OK;
  h->sweep_variant = 0;
  if (h->prec != STP_FP32_REFINE || h->nx % 4 || h->cfg.zline) return STP_OK;
  if (const char* env = std::getenv("STP_SWEEP_VARIANT")) {
    const int v = std::atoi(env);
    if (sweep_variant_ok(v, h->nx, h->ny, h->nz)) h->sweep_variant = v;
    return STP_OK;
  }
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int>, std::pair<int, float>> cache;
  const auto key = std::make_tuple(h->dev, h->nx, h->ny, h->nz);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      h->sweep_variant = it->second.first;
      h->sweep_us = it->second.second;
      return STP_OK;
    }
  }
  CUDA_TRY(h, cudaMemsetAsync(h->d1, 0, sizeof(float) * h->nc, h->st));
  CUDA_TRY(h, cudaMemsetAsync(h->r32, 0, sizeof(float) * h->nc, h->st));
  std::vector<std::pair<int, float>> timed;
  for (int v = 0; v < sweep_variant_count(); v++) {
    if (!sweep_variant_ok(v, h->nx, h->ny, h->nz)) continue;
    const bool pair = sweep_variant_is_pair(v);
    if (pair && (h->omega.size() % 4 != 0 || h->cycle_blocks > 0)) continue;
    set_sweep_variant(v);
    float us = 0.f;
    if (int rc = time_sweeps(h, pair, &us)) {
      if (!pair) return rc;
      cudaGetLastError();  // a pair tile this device cannot launch: not a candidate
      h->err.clear();
      continue;
    }
    timed.emplace_back(v, us);
  }
  const int bv = pick_variant(timed, &h->sweep_us);
  h->sweep_variant = bv;
  if (const char* lg = std::getenv("STP_TUNE_LOG")) {
    if (std::atoi(lg)) {
      std::fprintf(stderr, "stp: FP32 sweep tiles at %dx%dx%d (us per sweep):", h->nx, h->ny, h->nz);
      for (const auto& t : timed) std::fprintf(stderr, " %d=%.3f", t.first, t.second);
      std::fprintf(stderr, " -> %d\n", bv);
    }
  }
  std::lock_guard<std::mutex> lock(mu);
  cache[key] = std::make_pair(bv, h->sweep_us);
  return STP_OK;
}

// end the capture on h->cap, returning the node the capture ended on
int end_capture_tail(stp_handle* h, cudaGraph_t g, cudaGraphNode_t* tail) {
  cudaStreamCaptureStatus st;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CUDA_TRY(h, cudaStreamGetCaptureInfo(h->cap, &st, nullptr, nullptr, &deps, nullptr, &nd));
  *tail = nd ? deps[nd - 1] : nullptr;
  return end_capture(h, g);
}

// Append the pressure solve of h to graph G after node dep (nullptr: a
// root); *last receives its final node.  Conditional handles are created on
// G and armed explicitly every time the solve runs, so the solve can also sit
// inside another WHILE body (the batched step).
int append_solve(stp_handle* h, cudaGraph_t G, cudaGraphNode_t dep, cudaGraphNode_t* last) {
  if (int rc = tune_sweep(h)) return rc;
  set_sweep_variant(h->sweep_variant);
  int rc;
  cudaGraph_t wb, pb;
  cudaGraphNode_t wn, pn, tail;
  if (h->prec == STP_FP64) {
    cudaGraphConditionalHandle h_loop;
    CUDA_TRY(h, cudaGraphConditionalHandleCreate(&h_loop, G, 1, cudaGraphCondAssignDefault));
    if ((rc = begin_capture(h, G, dep))) return rc;
    CUDA_TRY(h, launch_begin(h->ctl, 1, h_loop, h->cap));
    if (h->net && h->learned_mode == 0) {
      // learned guess: r = b - L p (FP32), p += s U(r / s)
      CUDA_TRY(h, launch_outer(h->g64, h->p, h->b, h->r32, h->ctl, h->red, 0, 0, 0, h->cap));
      if ((rc = unet_guess(h->net, h->r32, h->red.sc + SC_INNER_REF, h->d1, h->cap, &h->guess_kernels)))
        return fail(h, rc, "learned guess: " + std::string(stp_unet_last_error(h->net)));
      CUDA_TRY(h, launch_addcorr(h->p, h->d1, h->nc, h->cap));
    }
    if ((rc = end_capture_tail(h, G, &tail))) return rc;
    if ((rc = add_conditional(h, G, tail, h_loop, cudaGraphCondTypeWhile, &wb, &wn))) return rc;
    if ((rc = build_cycle<double>(h, h->g64, wb, h_loop, h->p, h->p2, h->b, 0))) return rc;
    *last = wn;
  } else {
    cudaGraphConditionalHandle h_pass, h_loop;
    CUDA_TRY(h, cudaGraphConditionalHandleCreate(&h_pass, G, 0, cudaGraphCondAssignDefault));
    if ((rc = begin_capture(h, G, dep))) return rc;
    CUDA_TRY(h, launch_begin(h->ctl, 0, 0, h->cap));
    CUDA_TRY(h, launch_outer(h->g64, h->p, h->b, h->r32, h->ctl, h->red, 0, 1, h_pass, h->cap));
    if (h->net && h->learned_mode == 0) {
      // learned guess at the start of the solve: p += s U(r / s), then the
      // residual of the new p decides the first pass
      if ((rc = unet_guess(h->net, h->r32, h->red.sc + SC_INNER_REF, h->d1, h->cap, &h->guess_kernels)))
        return fail(h, rc, "learned guess: " + std::string(stp_unet_last_error(h->net)));
      CUDA_TRY(h, launch_addcorr(h->p, h->d1, h->nc, h->cap));
      CUDA_TRY(h, launch_outer(h->g64, h->p, h->b, h->r32, h->ctl, h->red, 0, 1, h_pass, h->cap));
    }
    if ((rc = end_capture_tail(h, G, &tail))) return rc;
    if ((rc = add_conditional(h, G, tail, h_pass, cudaGraphCondTypeWhile, &pb, &pn))) return rc;
    // pass body: d = 0, arm the loop -> WHILE(loop){cycle} -> p += d -> outer
    // residual.  The loop handle is set explicitly each pass: a handle's
    // default value is applied only when the top-level graph launches.
    CUDA_TRY(h, cudaGraphConditionalHandleCreate(&h_loop, pb, 1, 0));
    if ((rc = begin_capture(h, pb, nullptr))) return rc;
    CUDA_TRY(h, launch_pass_begin(h->d1, h->nc, 1, h_loop, h->cap));
    if (h->net && h->learned_mode == 1) {
      // learned preconditioner: every pass starts its inner solve of
      // L d = r from d = s U(r / s) instead of zero
      if ((rc = unet_guess(h->net, h->r32, h->red.sc + SC_INNER_REF, h->d1, h->cap, &h->guess_kernels)))
        return fail(h, rc, "learned preconditioner: " + std::string(stp_unet_last_error(h->net)));
    }
    if ((rc = end_capture(h, pb))) return rc;
    if ((rc = add_conditional(h, pb, leaf_node(pb), h_loop, cudaGraphCondTypeWhile, &wb, &wn))) return rc;
    if ((rc = build_cycle<float>(h, h->g32, wb, h_loop, h->d1, h->d2, h->r32, 1))) return rc;
    if ((rc = begin_capture(h, pb, wn))) return rc;
    CUDA_TRY(h, launch_addcorr(h->p, h->d1, h->nc, h->cap));
    CUDA_TRY(h, launch_outer(h->g64, h->p, h->b, h->r32, h->ctl, h->red, 1, 1, h_pass, h->cap));
    if ((rc = end_capture(h, pb))) return rc;
    *last = pn;
  }
  return STP_OK;
}

int build_solve_graph(stp_handle* h) {
  if (h->solve_exec) return STP_OK;
  cudaGraph_t G;
  CUDA_TRY(h, cudaGraphCreate(&G, 0));
  h->solve_graph = G;
  cudaGraphNode_t last;
  if (int rc = append_solve(h, G, nullptr, &last)) return rc;
  CUDA_TRY(h, cudaGraphInstantiate(&h->solve_exec, G, 0));
  return STP_OK;
}

// write the solve parameters and clear the totals (once per API call)
int arm_solves(stp_handle* h, double tol, int maxit) {
  if (int rc = tune_sweep(h)) return rc;
  SolveCtl c = {};
  c.tol = tol;
  c.inner_tol = h->cfg.inner_tol > 0 ? h->cfg.inner_tol : 1e-3;
  c.max_sweeps = maxit;
  c.max_passes = 64;
  c.M = (int)h->omega.size();
  c.kpc = (h->cycle_blocks > 0 || h->line_rb > 0) ? 1 : uses_pairs(h) ? c.M / 2 : c.M;
  c.bar_wait = 2000000000LL;
  if (const char* e = std::getenv("STP_BARRIER_WAIT")) {
    const long long w = std::atoll(e);
    if (w > 0) c.bar_wait = w;
  }
  if (const char* e = std::getenv("STP_WAIT_SKEW")) c.wait_skew = std::max(0, std::atoi(e));
  *h->h_ctl = c;
  CUDA_TRY(h, cudaMemcpyAsync(h->ctl, h->h_ctl, sizeof(SolveCtl), cudaMemcpyHostToDevice, h->st));
  // the persistent cycle's barrier state starts clean on every call, also
  // after a wait that timed out (count, generation, error flag)
  CUDA_TRY(h, cudaMemsetAsync(h->bar.count, 0, sizeof(unsigned) * 4, h->st));
  if (h->line_rb > 0)
    CUDA_TRY(h, cudaMemsetAsync(h->line_flags, 0, sizeof(int) * line_cycle_tiles(h->g32, h->line_rb), h->st));
  return STP_OK;
}

// The same solve driven from the host: the check kernels write their
// decision to ctl->go and the host reads it once per cycle.  Used when the
// environment sets STP_HOST_SOLVE=1 at stp_init (profilers cannot see the
// kernels inside graphs with conditional nodes).
int read_go(stp_handle* h, int* go) {
  CUDA_TRY(h, cudaMemcpyAsync(&h->h_ctl->go, &h->ctl->go, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  *go = h->h_ctl->go;
  return STP_OK;
}

template <typename T>
int host_cycles(stp_handle* h, const Geom<T>& g, T* A, T* B, const T* rhs, int mode) {
  const int M = (int)h->omega.size();
  for (;;) {
    CUDA_TRY(h, launch_check<T>(g, A, rhs, mode, h->ctl, h->red, 0, 0, 0, h->st));
    int go = 0, rc = read_go(h, &go);
    if (rc) return rc;
    if (!go) return STP_OK;
    if (sizeof(T) == sizeof(double) && h->net && h->learned_mode == 1) {
      CUDA_TRY(h, launch_outer(h->g64, h->p, h->b, h->r32, h->ctl, h->red, 0, 0, 0, h->st));
      rc = unet_guess(h->net, h->r32, h->red.sc + SC_INNER_REF, h->d1, h->st, &h->guess_kernels);
      if (rc) return fail(h, rc, "learned preconditioner failed");
      CUDA_TRY(h, launch_addcorr(h->p, h->d1, h->nc, h->st));
    }
    if (sizeof(T) == sizeof(float) && h->cycle_blocks > 0) {
      CUDA_TRY(h, launch_cycle_f32(h->g32, (float*)A, (float*)B, (const float*)rhs, h->d_omega32, M, h->bar, h->ctl,
                                   h->cycle_blocks, h->st));
      continue;
    }
    if (h->cfg.zline) {
      if (sizeof(T) == sizeof(float) && h->line_rb > 0) {
        CUDA_TRY(h, launch_line_cycle_f32(h->g32, h->line_rb, (float*)A, (float*)B, (const float*)rhs, h->d_omega32,
                                          M, h->line_flags, h->ctl, h->st));
        continue;
      }
      for (int m = 0; m < M; m++)
        CUDA_TRY(h, launch_line_sweep<T>(g, (m % 2 == 0) ? A : B, rhs, (T)h->omega[m], (m % 2 == 0) ? B : A,
                                         h->st, h->line_variant));
      continue;
    }
    if (sizeof(T) == sizeof(float) && uses_pairs(h)) {
      for (int m = 0; m < M; m += 2)
        CUDA_TRY(h, launch_sweep_pair(h->g32, (const float*)((m % 4 == 0) ? A : B), (const float*)rhs,
                                      (float)h->omega[m], (float)h->omega[m + 1], (float*)((m % 4 == 0) ? B : A),
                                      h->st));
      continue;
    }
    for (int m = 0; m < M; m++)
      CUDA_TRY(h, launch_sweep<T>(g, (m % 2 == 0) ? A : B, rhs, (T)h->omega[m], (m % 2 == 0) ? B : A, h->st));
  }
}

int host_solve(stp_handle* h) {
  if (int rc = tune_sweep(h)) return rc;
  set_sweep_variant(h->sweep_variant);
  CUDA_TRY(h, launch_begin(h->ctl, 0, 0, h->st));
  if (h->prec == STP_FP64) {
    if (h->net && h->learned_mode == 0) {
      CUDA_TRY(h, launch_outer(h->g64, h->p, h->b, h->r32, h->ctl, h->red, 0, 0, 0, h->st));
      int rc = unet_guess(h->net, h->r32, h->red.sc + SC_INNER_REF, h->d1, h->st, &h->guess_kernels);
      if (rc) return fail(h, rc, "learned guess failed");
      CUDA_TRY(h, launch_addcorr(h->p, h->d1, h->nc, h->st));
    }
    return host_cycles<double>(h, h->g64, h->p, h->p2, h->b, 0);
  }
  CUDA_TRY(h, launch_outer(h->g64, h->p, h->b, h->r32, h->ctl, h->red, 0, 0, 0, h->st));
  if (h->net && h->learned_mode == 0) {
    int rc = unet_guess(h->net, h->r32, h->red.sc + SC_INNER_REF, h->d1, h->st, &h->guess_kernels);
    if (rc) return fail(h, rc, "learned guess failed");
    CUDA_TRY(h, launch_addcorr(h->p, h->d1, h->nc, h->st));
    CUDA_TRY(h, launch_outer(h->g64, h->p, h->b, h->r32, h->ctl, h->red, 0, 0, 0, h->st));
  }
  for (;;) {
    int go = 0, rc = read_go(h, &go);
    if (rc) return rc;
    if (!go) return STP_OK;
    CUDA_TRY(h, launch_pass_begin(h->d1, h->nc, 0, 0, h->st));
    if (h->net && h->learned_mode == 1) {
      rc = unet_guess(h->net, h->r32, h->red.sc + SC_INNER_REF, h->d1, h->st, &h->guess_kernels);
      if (rc) return fail(h, rc, "learned preconditioner failed");
    }
    if ((rc = host_cycles<float>(h, h->g32, h->d1, h->d2, h->r32, 1))) return rc;
    CUDA_TRY(h, launch_addcorr(h->p, h->d1, h->nc, h->st));
    CUDA_TRY(h, launch_outer(h->g64, h->p, h->b, h->r32, h->ctl, h->red, 1, 0, 0, h->st));
  }
}

// training pairs: r = b - L p_prev before the solve, dp = p - p_prev after
int harvest_before(stp_handle* h) {
  if (!h->hr) return STP_OK;
  CUDA_TRY(h, cudaMemcpyAsync(h->p_prev, h->p, sizeof(double) * h->nc, cudaMemcpyDeviceToDevice, h->st));
  CUDA_TRY(h, launch_outer(h->g64, h->p, h->b, h->hr, h->ctl, h->red, 0, 0, 0, h->st));
  return STP_OK;
}
int harvest_after(stp_handle* h) {
  if (!h->hr) return STP_OK;
  CUDA_TRY(h, launch_difference(h->p, h->p_prev, h->hdp, h->nc, h->st));
  return STP_OK;
}

// one solve on the stream, bracketed by events
int launch_solve(stp_handle* h) {
  if (h->host_solve) {
    CUDA_TRY(h, cudaEventRecord(h->ev0, h->st));
    int rc = host_solve(h);
    if (rc) return rc;
    CUDA_TRY(h, cudaEventRecord(h->ev1, h->st));
    return STP_OK;
  }
  int rc = build_solve_graph(h);
  if (rc) return rc;
  CUDA_TRY(h, cudaEventRecord(h->ev0, h->st));
  CUDA_TRY(h, cudaGraphLaunch(h->solve_exec, h->st));
  CUDA_TRY(h, cudaEventRecord(h->ev1, h->st));
  return STP_OK;
}

// after a sync: elapsed time of the last solve and its counters
int finish_solve(stp_handle* h, SolveOut* o) {
  float ms = 0.f;
  CUDA_TRY(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
  CUDA_TRY(h, cudaMemcpy(h->h_ctl, h->ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost));
  const SolveCtl& c = *h->h_ctl;
  o->sweeps = c.sweeps;
  o->passes = c.passes;
  o->converged = c.converged;
  o->bad = c.bad;
  o->kernels = c.tot_kernels + c.kernels;
  // the learned guess runs once per solve: its kernels, the outer residual
  // before it, the correction and (FP32) the residual after it
  if (h->net && h->learned_mode == 0) o->kernels += (long long)c.solves * (h->guess_kernels + 3);
  // preconditioner: the network once per pass (FP32), or residual, network
  // and correction once per cycle (FP64); the last solve's counts
  if (h->net && h->learned_mode == 1)
    o->kernels += h->prec == STP_FP64 ? (long long)(c.sweeps / std::max(1, c.M)) * (h->guess_kernels + 2)
                                      : (long long)c.passes * h->guess_kernels;
  o->tot_sweeps = c.tot_sweeps + c.sweeps;
  o->nonconv = c.nonconv + (c.converged ? 0 : 1);
  const double nb = h->h_sc[SC_BNORM];
  o->rel = nb > 0 ? c.res / nb : c.res;
  h->solve_ms += ms;
  h->solve_sweeps += c.sweeps;
  return STP_OK;
}

// ---------------------------------------------------------------------------
// one projection step (Sec. 3.1).  Every pointer is fixed across steps (the
// Adams-Bashforth slot and coefficients come from the device step counter,
// and the Crank-Nicolson ping-pong always ends in the u buffer), so the
// launches of a step can be captured once into a graph.
// ---------------------------------------------------------------------------
// velocity part up to the Poisson right-hand side, on stream s
template <typename T>
int step_pre(stp_handle* h, const Geom<T>& g, cudaStream_t s) {
  const stp_config& c = h->cfg;
  T *u = (T*)h->u, *v = (T*)h->v, *w = (T*)h->w;
  T* nu = (T*)h->nu;
  const T nu0 = (T)c.nu;
  if (c.les) CUDA_TRY(h, launch_viscosity<T>(g, u, v, w, nu0, nu, s));
  const T fx = (T)(c.forcing == 0 ? c.fx : 0.0);
  Hist<T> H;
  for (int l = 0; l < 3; l++) {
    H.u[l] = (T*)h->Nu[l];
    H.v[l] = (T*)h->Nv[l];
    H.w[l] = (T*)h->Nw[l];
  }
  H.step = h->d_step;
  CUDA_TRY(h, launch_momentum<T>(g, c.les != 0, u, v, w, nu, nu0, fx, H, (T)c.dt, (T*)h->ru, (T*)h->rv, (T*)h->rw, s));
  // Crank-Nicolson Jacobi sweeps from the rhs, alternating between the t and
  // u buffers so that the last sweep writes u (u^n is no longer needed)
  void* R[3] = {h->ru, h->rv, h->rw};
  void* U[3] = {h->u, h->v, h->w};
  void* Tb[3] = {h->tu, h->tv, h->tw};
  void** cur = R;
  const int n = h->cn_sweeps;
  // z-line sweeps: the columns' pivots once per step (nu_T is fixed within
  // it), then every sweep in level chunks; columns too tall for the chunks
  // eliminate column by column with the scratch array
  const T* piv = nullptr;
  if (c.cn_zline && n > 0 && cn_chunk_ok(h->nz)) {
    CUDA_TRY(h, launch_cn_pivots<T>(g, c.les != 0, nu, nu0, (T)(0.5 * c.dt), (T*)h->cn_scr, s));
    piv = (const T*)h->cn_scr;
  }
  for (int k = 0; k < n; k++) {
    void** out = ((n - 1 - k) % 2 == 0) ? U : Tb;
    if (c.cn_zline)
      CUDA_TRY(h, launch_cn_line<T>(g, c.les != 0, nu, nu0, (T)(0.5 * c.dt), (const T*)h->ru, (const T*)h->rv,
                                    (const T*)h->rw, (const T*)cur[0], (const T*)cur[1], (const T*)cur[2],
                                    (T*)out[0], (T*)out[1], (T*)out[2], h->cn_scr, piv, s));
    else
      CUDA_TRY(h, launch_cn_sweep<T>(g, c.les != 0, nu, nu0, (T)(0.5 * c.dt), (const T*)h->ru, (const T*)h->rv,
                                     (const T*)h->rw, (const T*)cur[0], (const T*)cur[1], (const T*)cur[2],
                                     (T*)out[0], (T*)out[1], (T*)out[2], s));
    cur = out;
  }
  if (n == 0) {
    CUDA_TRY(h, cudaMemcpyAsync(h->u, h->ru, h->esz * h->nc, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(h, cudaMemcpyAsync(h->v, h->rv, h->esz * h->nc, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(h, cudaMemcpyAsync(h->w, h->rw, h->esz * h->nw, cudaMemcpyDeviceToDevice, s));
  }
  // b = D u* / dt
  CUDA_TRY(h, launch_divergence_rhs<T>(g, u, v, w, 1.0 / c.dt, h->b, h->red, c.Lz, s));
  return STP_OK;
}

// projection, wall conditions, flux fix-up and the step counter, on stream s
template <typename T>
int step_post(stp_handle* h, const Geom<T>& g, cudaStream_t s) {
  const stp_config& c = h->cfg;
  T *u = (T*)h->u, *v = (T*)h->v, *w = (T*)h->w;
  const double inv_vol = 1.0 / ((double)h->nx * h->ny * c.Lz);
  CUDA_TRY(h, launch_correct_impl<T>(g, h->p, c.dt, u, v, w, h->g64.ihz, h->g64.dzv, inv_vol, h->red, s));
  if (c.forcing == 1) CUDA_TRY(h, launch_flux_shift<T>(g, u, c.ubulk, h->red, s));
  CUDA_TRY(h, launch_step_end(h->d_step, s));
  return STP_OK;
}

template <typename T>
int step_impl(stp_handle* h, const Geom<T>& g) {
  int rc = step_pre<T>(h, g, h->st);
  if (rc) return rc;
  if ((rc = harvest_before(h))) return rc;
  if ((rc = launch_solve(h))) return rc;
  if ((rc = harvest_after(h))) return rc;
  if ((rc = step_post<T>(h, g, h->st))) return rc;
  h->step++;
  if (h->nhist < 3) h->nhist++;
  return STP_OK;
}

// copy a double field (host or device) into a T device field
template <typename T>
int put_field(stp_handle* h, T* dst, const double* src, size_t n, int where) {
  const cudaMemcpyKind kind = where == STP_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (sizeof(T) == sizeof(double)) {
    CUDA_TRY(h, cudaMemcpyAsync(dst, src, n * sizeof(double), kind, h->st));
  } else {
    CUDA_TRY(h, cudaMemcpyAsync(h->stage, src, n * sizeof(double), kind, h->st));
    CUDA_TRY(h, (launch_convert<float, double>((float*)dst, h->stage, n, h->st)));
  }
  return STP_OK;
}

template <typename T>
int get_field(stp_handle* h, double* dst, const T* src, size_t n, int where) {
  const cudaMemcpyKind kind = where == STP_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (sizeof(T) == sizeof(double)) {
    CUDA_TRY(h, cudaMemcpyAsync(dst, src, n * sizeof(double), kind, h->st));
  } else {
    CUDA_TRY(h, (launch_convert<double, float>(h->stage, (const float*)src, n, h->st)));
    CUDA_TRY(h, cudaMemcpyAsync(dst, h->stage, n * sizeof(double), kind, h->st));
  }
  return STP_OK;
}

int put_any(stp_handle* h, void* dst, const double* src, size_t n, int where) {
  return h->prec == STP_FP64 ? put_field<double>(h, (double*)dst, src, n, where)
                             : put_field<float>(h, (float*)dst, src, n, where);
}
int get_any(stp_handle* h, double* dst, const void* src, size_t n, int where) {
  return h->prec == STP_FP64 ? get_field<double>(h, dst, (const double*)src, n, where)
                             : get_field<float>(h, dst, (const float*)src, n, where);
}

int fill_const(stp_handle* h, double* dst, double val, size_t n, int where) {
  std::vector<double> tmp(n, val);
  if (where == STP_HOST) {
    std::copy(tmp.begin(), tmp.end(), dst);
    return STP_OK;
  }
  CUDA_TRY(h, cudaMemcpyAsync(dst, tmp.data(), n * sizeof(double), cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return STP_OK;
}

int check_where(stp_handle* h, int where) {
  if (where != STP_HOST && where != STP_DEVICE) return fail(h, STP_EINVAL, "where must be STP_HOST or STP_DEVICE");
  return STP_OK;
}

}  // namespace

// State buffer: a header of four doubles (format tag, history depth, step
// counter, cells), then u, v, w, p and the two latest history levels of
// u, v, w.  Fields are kept in the handle's precision: an FP64 handle
// stores doubles (tag 1511.07800); an FP32 handle stores its FP32 fields
// as raw floats, each array padded to a whole number of doubles, and p in
// FP64 (tag 1511.07832): about half the bytes that widening them would take.
namespace {
constexpr double kStateTag64 = 1511.07800, kStateTag32 = 1511.07832;
long long state_words(const stp_handle* h, long long n) {  // doubles holding n field values
  return h->prec == STP_FP64 ? n : (n + 1) / 2;
}
// copy n field values between the device array f and the buffer section q
int state_get(stp_handle* h, double* q, const void* f, long long n) {
  if (h->prec == STP_FP64) return get_any(h, q, f, (size_t)n, STP_HOST);
  CUDA_TRY(h, cudaMemcpyAsync(q, f, sizeof(float) * n, cudaMemcpyDeviceToHost, h->st));
  return STP_OK;
}
int state_put(stp_handle* h, void* f, const double* q, long long n) {
  if (h->prec == STP_FP64) return put_any(h, f, q, (size_t)n, STP_HOST);
  CUDA_TRY(h, cudaMemcpyAsync(f, q, sizeof(float) * n, cudaMemcpyHostToDevice, h->st));
  return STP_OK;
}
}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void stp_config_defaults(stp_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->nx = c->ny = c->nz = 32;
  c->Lx = 2.0 * 3.14159265358979323846;
  c->Ly = 3.14159265358979323846;
  c->Lz = 2.0;
  c->nu = 1.0;
  c->dt = 1e-3;
  c->cs = 0.1;
  c->vd_a = 25.0;
  c->re_tau = 180.0;
  c->precision = STP_FP64;
  c->ptol = 1e-8;
  c->pmaxit = 200000;
  c->inner_tol = 1e-3;
}

const char* stp_last_error(const stp_handle* h) { return h ? h->err.c_str() : g_init_error.c_str(); }

void stp_destroy(stp_handle* h) {
  if (!h) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->dev);
  if (h->st) cudaStreamSynchronize(h->st);
  for (void* p : h->allocs) cudaFree(p);
  if (h->h_sc) cudaFreeHost(h->h_sc);
  if (h->h_flag) cudaFreeHost(h->h_flag);
  if (h->solve_exec) cudaGraphExecDestroy(h->solve_exec);
  if (h->solve_graph) cudaGraphDestroy(h->solve_graph);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->h_ctl) cudaFreeHost(h->h_ctl);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->own_stream && h->st) cudaStreamDestroy(h->st);
  cudaSetDevice(cur);
  delete h;
}

int stp_srj_schedule(const stp_config* cfg, int M, double* omega, int* M_out, double* mu_min, double* mu_max) {
  std::string why;
  if (int rc = validate(cfg, &why)) return fail(nullptr, rc, why);
  if (M != 0 && (!pow2(M) || M > 1024)) return fail(nullptr, STP_EINVAL, "M must be 0 or a power of two <= 1024");
  double mn, mx;
  solve_bounds(*cfg, &mn, &mx);
  if (M == 0) M = auto_cycle(mn, mx);
  const std::vector<double> om = chebyshev(mn, mx, M);
  if (omega) std::copy(om.begin(), om.end(), omega);
  if (M_out) *M_out = M;
  if (mu_min) *mu_min = mn;
  if (mu_max) *mu_max = mx;
  return STP_OK;
}

int stp_init(const stp_config* cfg, stp_handle** out) {
  if (!out) return fail(nullptr, STP_EINVAL, "out is NULL");
  *out = nullptr;
  std::string why;
  if (int rc = validate(cfg, &why)) return fail(nullptr, rc, why);
  stp_handle* h = new (std::nothrow) stp_handle();
  if (!h) return fail(nullptr, STP_ENOMEM, "host allocation failed");
  h->cfg = *cfg;
  h->cfg.srj_omega = nullptr;
  h->prec = cfg->precision;
  h->dev = cfg->device;
  h->nx = cfg->nx;
  h->ny = cfg->ny;
  h->nz = cfg->nz;
  h->nplane = (size_t)cfg->nx * cfg->ny;
  h->nc = h->nplane * cfg->nz;
  h->nw = h->nplane * (cfg->nz + 1);
  h->esz = h->prec == STP_FP64 ? sizeof(double) : sizeof(float);
  auto bail = [&](int rc) {
    g_init_error = h->err;
    stp_destroy(h);
    return rc;
  };
  cudaError_t e = cudaSetDevice(h->dev);
  if (e != cudaSuccess) return bail(fail(h, STP_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e)));
  if (cfg->stream) {
    h->st = (cudaStream_t)cfg->stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(fail(h, STP_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e)));
    h->own_stream = true;
  }
  if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(h, STP_ECUDA, "event or stream creation failed"));
  // schedule
  if (cfg->srj_omega) {
    h->omega.assign(cfg->srj_omega, cfg->srj_omega + cfg->srj_m);
  } else {
    double mn, mx;
    solve_bounds(*cfg, &mn, &mx);
    const int M = cfg->srj_m > 0 ? cfg->srj_m : auto_cycle(mn, mx);
    h->omega = chebyshev(mn, mx, M);
  }
  h->cfg.srj_m = (int)h->omega.size();
  const ZGrid z = make_z(*cfg);
  h->cn_sweeps = cfg->cn_sweeps > 0 ? cfg->cn_sweeps : auto_cn_sweeps(*cfg, z);
  {
    const char* env = std::getenv("STP_HOST_SOLVE");
    h->host_solve = env && env[0] == '1';
  }
  // device memory
  const size_t es = h->esz, nc = h->nc, nw = h->nw;
  int rc = STP_OK;
  auto A = [&](void** p, size_t bytes) {
    if (rc == STP_OK) rc = dalloc(h, p, bytes);
  };
  const int L = h->nz + 1;
  A((void**)&h->m64, sizeof(double) * kMetricArrays * L);
  A((void**)&h->m32, sizeof(float) * (kMetricArrays + 4) * L);
  A(&h->u, es * nc);
  A(&h->v, es * nc);
  A(&h->w, es * nw);
  A(&h->ru, es * nc);
  A(&h->rv, es * nc);
  A(&h->rw, es * nw);
  A(&h->tu, es * nc);
  A(&h->tv, es * nc);
  A(&h->tw, es * nw);
  for (int l = 0; l < 3; l++) {
    A(&h->Nu[l], es * nc);
    A(&h->Nv[l], es * nc);
    A(&h->Nw[l], es * nw);
  }
  if (cfg->les) A(&h->nu, es * nc);
  A((void**)&h->b, sizeof(double) * nc);
  A((void**)&h->p, sizeof(double) * nc);
  A((void**)&h->p2, sizeof(double) * nc);
  if (h->prec == STP_FP32_REFINE) {
    A((void**)&h->d1, sizeof(float) * nc);
    A((void**)&h->d2, sizeof(float) * nc);
    A((void**)&h->r32, sizeof(float) * nc);
  }
  A((void**)&h->stage, sizeof(double) * nw);
  A(&h->bu, es * nc);
  A(&h->bv, es * nc);
  A(&h->bw, es * nw);
  A((void**)&h->bp, sizeof(double) * nc);
  if (cfg->cn_zline) A(&h->cn_scr, 2 * es * 3 * nw);
  const Launch big = {dim3((h->nx + 31) / 32, (h->ny + 7) / 8, h->nz + 1), dim3(32, 8, 1), 0};
  const size_t maxblocks = (size_t)big.grid.x * big.grid.y * big.grid.z + 152 * 32;
  A((void**)&h->red.partial, sizeof(double) * 2 * maxblocks);
  A((void**)&h->red.counter, sizeof(unsigned) * 4);
  A((void**)&h->red.gcount, sizeof(unsigned) * (maxblocks / 64 + 2));
  A((void**)&h->red.sc, sizeof(double) * SC_COUNT);
  A((void**)&h->red.flag, sizeof(int) * FL_COUNT);
  A((void**)&h->ctl, sizeof(SolveCtl));
  A((void**)&h->d_step, sizeof(int) * 4);
  A((void**)&h->d_omega32, sizeof(float) * h->omega.size());
  A((void**)&h->bar.count, sizeof(unsigned) * 4);
  if (rc) return bail(rc);
  h->bar.gen = h->bar.count + 1;
  h->bar.err = (int*)(h->bar.count + 2);
  {
    // persistent FP32 cycles (STP_PERSISTENT=1) need rows of whole float4
    // units; off by default: on GB300 a grid barrier between sweeps costs
    // more than a graph-launched kernel boundary
    const char* env = std::getenv("STP_PERSISTENT");
    const bool allow = env && env[0] == '1';
    if (allow && h->prec == STP_FP32_REFINE && h->nx % 4 == 0 && !cfg->zline)
      h->cycle_blocks = cycle_grid_f32(h->dev);
  }
  if (h->prec == STP_FP32_REFINE && cfg->zline && line_chunk_ok(h->nx, h->nz)) {
    // FP32 z-line sweeps solve their columns in registers where the grid
    // allows it; STP_LINE_VARIANT=0 keeps the shared-memory lock-step kernel
    const char* env = std::getenv("STP_LINE_VARIANT");
    h->line_variant = (env && env[0] == '0') ? 0 : 1;
  }
  {
    // persistent z-line cycles (STP_LINE_PERSISTENT=1): one cooperative
    // launch per SRJ cycle, tiles synchronised with their neighbours
    const char* env = std::getenv("STP_LINE_PERSISTENT");
    if (env && env[0] == '1' && h->prec == STP_FP32_REFINE && cfg->zline) {
      Geom<float> gtmp{};
      gtmp.nx = h->nx;
      gtmp.ny = h->ny;
      gtmp.nz = h->nz;
      const int rb = line_cycle_rows(gtmp, h->dev);
      if (rb > 0 && dalloc(h, (void**)&h->line_flags, sizeof(int) * line_cycle_tiles(gtmp, rb)) == STP_OK)
        h->line_rb = rb;
    }
  }
  if (cudaMallocHost((void**)&h->h_sc, sizeof(double) * SC_COUNT) != cudaSuccess ||
      cudaMallocHost((void**)&h->h_flag, sizeof(int) * FL_COUNT) != cudaSuccess ||
      cudaMallocHost((void**)&h->h_ctl, sizeof(SolveCtl)) != cudaSuccess)
    return bail(fail(h, STP_ENOMEM, "cudaMallocHost failed"));
  // metrics
  const std::vector<double> m = metric_pack(*cfg);
  std::vector<float> mf(m.begin(), m.end());
  {
    // {cup, cdn, tli, tlf} per level, after the arrays (see geom_from)
    const int L = h->nz + 1;
    mf.resize((size_t)(kMetricArrays + 4) * L, 0.f);
    float* pk = mf.data() + (size_t)kMetricArrays * L;
    for (int k = 0; k < h->nz; k++) {
      pk[4 * k + 0] = mf[5 * L + k];
      pk[4 * k + 1] = mf[6 * L + k];
      pk[4 * k + 2] = mf[13 * L + k];
      pk[4 * k + 3] = mf[14 * L + k];
    }
  }
  h->g64 = geom_from<double>(h, h->m64);
  h->g32 = geom_from<float>(h, h->m32);
  e = cudaMemcpyAsync(h->m64, m.data(), sizeof(double) * m.size(), cudaMemcpyHostToDevice, h->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->m32, mf.data(), sizeof(float) * mf.size(), cudaMemcpyHostToDevice, h->st);
  // every field starts at zero
  if (e == cudaSuccess) e = cudaMemsetAsync(h->u, 0, es * nc, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->v, 0, es * nc, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->w, 0, es * nw, h->st);
  for (int l = 0; l < 3 && e == cudaSuccess; l++) {
    e = cudaMemsetAsync(h->Nu[l], 0, es * nc, h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->Nv[l], 0, es * nc, h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->Nw[l], 0, es * nw, h->st);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->p, 0, sizeof(double) * nc, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->p2, 0, sizeof(double) * nc, h->st);
  if (e == cudaSuccess && h->nu) e = cudaMemsetAsync(h->nu, 0, es * nc, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->red.counter, 0, sizeof(unsigned) * 4, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->red.gcount, 0, sizeof(unsigned) * (maxblocks / 64 + 2), h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->red.sc, 0, sizeof(double) * SC_COUNT, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->red.flag, 0, sizeof(int) * FL_COUNT, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->ctl, 0, sizeof(SolveCtl), h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->bar.count, 0, sizeof(unsigned) * 4, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_step, 0, sizeof(int) * 4, h->st);
  if (e == cudaSuccess) {
    std::vector<float> om32(h->omega.begin(), h->omega.end());
    e = cudaMemcpyAsync(h->d_omega32, om32.data(), sizeof(float) * om32.size(), cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return bail(fail(h, STP_ECUDA, std::string("init copies: ") + cudaGetErrorString(e)));
  *out = h;
  return STP_OK;
}

int stp_set_fields(stp_handle* h, const double* u, const double* v, const double* w, const double* p, int where) {
  if (!h) return STP_EINVAL;
  if (int rc = check_where(h, where)) return rc;
  if (!u || !v || !w) return fail(h, STP_EINVAL, "u, v and w are required");
  CUDA_TRY(h, cudaSetDevice(h->dev));
  // the wall planes of w must be zero
  std::vector<double> walls(2 * h->nplane);
  const cudaMemcpyKind k = where == STP_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost;
  CUDA_TRY(h, cudaMemcpyAsync(walls.data(), w, sizeof(double) * h->nplane, k, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(walls.data() + h->nplane, w + h->nplane * h->nz, sizeof(double) * h->nplane, k, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  for (double x : walls)
    if (x != 0.0) return fail(h, STP_EINVAL, "w must be zero on the wall planes k = 0 and k = nz");
  int rc;
  if ((rc = put_any(h, h->u, u, h->nc, where))) return rc;
  if ((rc = put_any(h, h->v, v, h->nc, where))) return rc;
  if ((rc = put_any(h, h->w, w, h->nw, where))) return rc;
  if (p) {
    CUDA_TRY(h, cudaMemcpyAsync(h->p, p, sizeof(double) * h->nc,
                                where == STP_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->st));
  } else {
    CUDA_TRY(h, cudaMemsetAsync(h->p, 0, sizeof(double) * h->nc, h->st));
  }
  CUDA_TRY(h, cudaMemsetAsync(h->d_step, 0, sizeof(int), h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  h->nhist = 0;
  h->step = 0;
  h->last_dpdx = 0.0;
  return STP_OK;
}

int stp_get_fields(stp_handle* h, double* u, double* v, double* w, double* p, double* nu_t, int where) {
  if (!h) return STP_EINVAL;
  if (int rc = check_where(h, where)) return rc;
  CUDA_TRY(h, cudaSetDevice(h->dev));
  int rc;
  if (u && (rc = get_any(h, u, h->u, h->nc, where))) return rc;
  if (v && (rc = get_any(h, v, h->v, h->nc, where))) return rc;
  if (w && (rc = get_any(h, w, h->w, h->nw, where))) return rc;
  if (p)
    CUDA_TRY(h, cudaMemcpyAsync(p, h->p, sizeof(double) * h->nc,
                                where == STP_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->st));
  if (nu_t) {
    if (h->cfg.les) {
      if ((rc = get_any(h, nu_t, h->nu, h->nc, where))) return rc;
    } else {
      CUDA_TRY(h, cudaStreamSynchronize(h->st));
      if ((rc = fill_const(h, nu_t, h->cfg.nu, h->nc, where))) return rc;
    }
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return STP_OK;
}

int stp_step(stp_handle* h, int nsteps, stp_step_stats* stats) {
  if (!h) return STP_EINVAL;
  if (nsteps < 0) return fail(h, STP_EINVAL, "nsteps < 0");
  CUDA_TRY(h, cudaSetDevice(h->dev));
  h->launches = 0;
  h->solve_sweeps = 0;
  h->solve_ms = 0.0;
  int rc = arm_solves(h, h->cfg.ptol, h->cfg.pmaxit);
  if (rc) return rc;
  SolveOut so;
  for (int n = 0; n < nsteps; n++) {
    // keep the fields of the last good step: a step that diverges or times
    // out is undone (its Adams-Bashforth slot held N^{n-3}, no longer used)
    const long long step0 = h->step;
    const int nhist0 = h->nhist;
    CUDA_TRY(h, cudaMemcpyAsync(h->bu, h->u, h->esz * h->nc, cudaMemcpyDeviceToDevice, h->st));
    CUDA_TRY(h, cudaMemcpyAsync(h->bv, h->v, h->esz * h->nc, cudaMemcpyDeviceToDevice, h->st));
    CUDA_TRY(h, cudaMemcpyAsync(h->bw, h->w, h->esz * h->nw, cudaMemcpyDeviceToDevice, h->st));
    CUDA_TRY(h, cudaMemcpyAsync(h->bp, h->p, sizeof(double) * h->nc, cudaMemcpyDeviceToDevice, h->st));
    rc = h->prec == STP_FP64 ? step_impl<double>(h, h->g64) : step_impl<float>(h, h->g32);
    if (rc) return rc;
    if ((rc = sync_scalars(h))) return rc;
    if ((rc = finish_solve(h, &so))) return rc;
    if (so.bad || h->h_flag[FL_BAD]) {
      CUDA_TRY(h, cudaMemcpyAsync(h->u, h->bu, h->esz * h->nc, cudaMemcpyDeviceToDevice, h->st));
      CUDA_TRY(h, cudaMemcpyAsync(h->v, h->bv, h->esz * h->nc, cudaMemcpyDeviceToDevice, h->st));
      CUDA_TRY(h, cudaMemcpyAsync(h->w, h->bw, h->esz * h->nw, cudaMemcpyDeviceToDevice, h->st));
      CUDA_TRY(h, cudaMemcpyAsync(h->p, h->bp, sizeof(double) * h->nc, cudaMemcpyDeviceToDevice, h->st));
      const int ds = (int)step0;
      CUDA_TRY(h, cudaMemcpyAsync(h->d_step, &ds, sizeof(int), cudaMemcpyHostToDevice, h->st));
      CUDA_TRY(h, cudaMemsetAsync(h->red.flag + FL_BAD, 0, sizeof(int), h->st));
      CUDA_TRY(h, cudaStreamSynchronize(h->st));
      h->step = step0;
      h->nhist = nhist0;
      if (so.bad == 2) return fail(h, STP_ETIMEOUT, "a grid barrier of the persistent SRJ cycle timed out");
      if (so.bad) return fail(h, STP_EDIVERGED, "NaN or Inf in the pressure residual");
      return fail(h, STP_EDIVERGED, "NaN or Inf in the velocity");
    }
  }
  if (h->cfg.forcing == 1 && nsteps > 0) h->last_dpdx = h->h_sc[SC_SHIFT] / h->cfg.dt;
  if (stats) {
    stats->poisson_sweeps = so.sweeps;
    stats->refine_passes = so.passes;
    stats->converged = nsteps > 0 ? so.nonconv == 0 : 1;
    stats->rel_residual = so.rel;
    stats->ubulk = h->h_sc[SC_BULK] + (h->cfg.forcing == 1 ? h->h_sc[SC_SHIFT] : 0.0);
    stats->umax = h->h_sc[SC_UMAX];
    stats->dpdx = h->last_dpdx;
    stats->step = h->step;
    stats->launches = h->launches + so.kernels;
    stats->solve_sweeps = so.tot_sweeps;
    stats->solve_ms = h->solve_ms;
  }
  if (nsteps > 0 && so.nonconv) return fail(h, STP_ENOTCONVERGED, "a pressure solve hit pmaxit");
  if (h->cfg.cfl_check && h->h_sc[SC_UMAX] * h->cfg.dt > 0.1 * h->cfg.Lx / h->nx)
    return fail(h, STP_ECFL, "U_max dt > 0.1 dx");
  return STP_OK;
}

int stp_poisson_solve(stp_handle* h, const double* rhs, double* p_inout, double tol, int maxit, int where,
                      stp_solve_stats* stats) {
  if (!h) return STP_EINVAL;
  if (int rc = check_where(h, where)) return rc;
  if (!rhs || !p_inout) return fail(h, STP_EINVAL, "rhs and p_inout are required");
  if (!(tol >= 0)) return fail(h, STP_EINVAL, "tol must be >= 0");
  CUDA_TRY(h, cudaSetDevice(h->dev));
  const cudaMemcpyKind kin = where == STP_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CUDA_TRY(h, cudaMemcpyAsync(h->b, rhs, sizeof(double) * h->nc, kin, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(h->p, p_inout, sizeof(double) * h->nc, kin, h->st));
  // L is singular (Neumann walls, periodic x and y): L p = rhs has a
  // solution only when the volume integral of rhs vanishes
  CUDA_TRY(h, launch_vsum(h->g64, h->b, h->red, h->st));
  int rc = sync_scalars(h);
  if (rc) return rc;
  if (std::fabs(h->h_sc[SC_VSUM]) > kMeanTol * h->h_sc[SC_VABS])
    return fail(h, STP_EINVAL, "rhs has a non-zero volume-weighted mean (" + std::to_string(h->h_sc[SC_VSUM]) +
                                   " against a volume sum of |rhs| of " + std::to_string(h->h_sc[SC_VABS]) +
                                   "): L p = rhs has no solution");
  CUDA_TRY(h, launch_norm(h->b, h->nc, SC_BNORM, h->red, h->st));
  CUDA_TRY(h, cudaMemsetAsync(h->red.sc + SC_BMEAN, 0, sizeof(double), h->st));
  rc = arm_solves(h, tol, maxit > 0 ? maxit : h->cfg.pmaxit);
  if (rc) return rc;
  h->solve_ms = 0.0;
  h->solve_sweeps = 0;
  if ((rc = harvest_before(h))) return rc;
  if ((rc = launch_solve(h))) return rc;
  if ((rc = harvest_after(h))) return rc;
  // gauge: the solution's volume-weighted mean is set to zero
  CUDA_TRY(h, launch_vsum(h->g64, h->p, h->red, h->st));
  CUDA_TRY(h, launch_sub_vmean(h->g64, h->p, h->cfg.Lz, h->red, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(p_inout, h->p, sizeof(double) * h->nc,
                              where == STP_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->st));
  if ((rc = sync_scalars(h))) return rc;
  SolveOut so;
  if ((rc = finish_solve(h, &so))) return rc;
  if (so.bad == 2) return fail(h, STP_ETIMEOUT, "a grid barrier of the persistent SRJ cycle timed out");
  if (so.bad) return fail(h, STP_EDIVERGED, "NaN or Inf in the pressure residual");
  if (stats) {
    stats->sweeps = so.sweeps;
    stats->refine_passes = so.passes;
    stats->converged = so.converged;
    stats->rel_residual = so.rel;
    stats->solve_ms = h->solve_ms;
  }
  return so.converged ? STP_OK : fail(h, STP_ENOTCONVERGED, "pressure solve hit maxit");
}

// state layout: header [4] (magic, nhist, step, nc) | u | v | w | p | Nu,Nv,Nw of levels n, n-1 (history)
long long stp_state_size(const stp_handle* h) {
  if (!h) return 0;
  const long long nc = h->nc, nw = h->nw;
  return 4 + 3 * state_words(h, nc) + state_words(h, nw) + nc + 2 * (2 * state_words(h, nc) + state_words(h, nw));
}

int stp_get_state(stp_handle* h, double* buf) {
  if (!h || !buf) return STP_EINVAL;
  CUDA_TRY(h, cudaSetDevice(h->dev));
  buf[0] = h->prec == STP_FP64 ? kStateTag64 : kStateTag32;
  buf[1] = h->nhist;
  buf[2] = (double)h->step;
  buf[3] = (double)h->nc;
  double* q = buf + 4;
  int rc;
  const long long nc = h->nc, nw = h->nw;
  // the latest history level is in slot (step - 1) % 3, the one before in (step - 2) % 3
  const int sl[2] = {(int)((h->step + 2) % 3), (int)((h->step + 1) % 3)};
  if ((rc = state_get(h, q, h->u, nc))) return rc;
  q += state_words(h, nc);
  if ((rc = state_get(h, q, h->v, nc))) return rc;
  q += state_words(h, nc);
  if ((rc = state_get(h, q, h->w, nw))) return rc;
  q += state_words(h, nw);
  CUDA_TRY(h, cudaMemcpyAsync(q, h->p, sizeof(double) * nc, cudaMemcpyDeviceToHost, h->st));
  q += nc;
  for (int i = 0; i < 2; i++) {
    const int l = sl[i];
    if ((rc = state_get(h, q, h->Nu[l], nc))) return rc;
    q += state_words(h, nc);
    if ((rc = state_get(h, q, h->Nv[l], nc))) return rc;
    q += state_words(h, nc);
    if ((rc = state_get(h, q, h->Nw[l], nw))) return rc;
    q += state_words(h, nw);
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return STP_OK;
}

int stp_set_state(stp_handle* h, const double* buf) {
  if (!h || !buf) return STP_EINVAL;
  if (buf[0] != (h->prec == STP_FP64 ? kStateTag64 : kStateTag32) || buf[3] != (double)h->nc)
    return fail(h, STP_EINVAL, "state buffer does not match (grid or precision)");
  CUDA_TRY(h, cudaSetDevice(h->dev));
  const double* q = buf + 4;
  int rc;
  const long long nc = h->nc, nw = h->nw;
  const long long step = (long long)buf[2];
  const int sl[2] = {(int)((step + 2) % 3), (int)((step + 1) % 3)};
  if ((rc = state_put(h, h->u, q, nc))) return rc;
  q += state_words(h, nc);
  if ((rc = state_put(h, h->v, q, nc))) return rc;
  q += state_words(h, nc);
  if ((rc = state_put(h, h->w, q, nw))) return rc;
  q += state_words(h, nw);
  CUDA_TRY(h, cudaMemcpyAsync(h->p, q, sizeof(double) * nc, cudaMemcpyHostToDevice, h->st));
  q += nc;
  for (int i = 0; i < 2; i++) {
    const int l = sl[i];
    if ((rc = state_put(h, h->Nu[l], q, nc))) return rc;
    q += state_words(h, nc);
    if ((rc = state_put(h, h->Nv[l], q, nc))) return rc;
    q += state_words(h, nc);
    if ((rc = state_put(h, h->Nw[l], q, nw))) return rc;
    q += state_words(h, nw);
  }
  const int dstep = (int)step;
  CUDA_TRY(h, cudaMemcpyAsync(h->d_step, &dstep, sizeof(int), cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  h->nhist = (int)buf[1];
  h->step = step;
  return STP_OK;
}

int stp_set_learned_guess(stp_handle* h, stp_unet* net) {
  if (!h) return STP_EINVAL;
  if (net && !unet_matches(net, h->nz, h->ny, h->nx))
    return fail(h, STP_EINVAL, "the network's grid does not match the channel");
  CUDA_TRY(h, cudaSetDevice(h->dev));
  if (net && (!h->r32 || !h->d1)) {
    int rc = STP_OK;
    if (!h->r32) rc = dalloc(h, (void**)&h->r32, sizeof(float) * h->nc);
    if (rc == STP_OK && !h->d1) rc = dalloc(h, (void**)&h->d1, sizeof(float) * h->nc);
    if (rc) return rc;
  }
  // the solve graph is rebuilt with (or without) the guess nodes
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  if (h->solve_exec) cudaGraphExecDestroy(h->solve_exec);
  if (h->solve_graph) cudaGraphDestroy(h->solve_graph);
  h->solve_exec = nullptr;
  h->solve_graph = nullptr;
  h->net = net;
  return STP_OK;
}

int stp_set_learned_mode(stp_handle* h, int mode) {
  if (!h) return STP_EINVAL;
  if (mode != 0 && mode != 1) return fail(h, STP_EINVAL, "learned mode must be 0 or 1");
  CUDA_TRY(h, cudaSetDevice(h->dev));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  if (h->solve_exec) cudaGraphExecDestroy(h->solve_exec);
  if (h->solve_graph) cudaGraphDestroy(h->solve_graph);
  h->solve_exec = nullptr;
  h->solve_graph = nullptr;
  h->learned_mode = mode;
  return STP_OK;
}

int stp_set_harvest(stp_handle* h, float* r_out, float* dp_out) {
  if (!h) return STP_EINVAL;
  if ((r_out == nullptr) != (dp_out == nullptr)) return fail(h, STP_EINVAL, "give both r_out and dp_out, or neither");
  CUDA_TRY(h, cudaSetDevice(h->dev));
  if (r_out && !h->p_prev) {
    int rc = dalloc(h, (void**)&h->p_prev, sizeof(double) * h->nc);
    if (rc) return rc;
  }
  h->hr = r_out;
  h->hdp = dp_out;
  return STP_OK;
}

int stp_eval(stp_handle* h, int term, double* a, double* b, double* c, int where) {
  if (!h) return STP_EINVAL;
  if (int rc = check_where(h, where)) return rc;
  if (!a) return fail(h, STP_EINVAL, "output a is required");
  CUDA_TRY(h, cudaSetDevice(h->dev));
  const stp_config& cf = h->cfg;
  int rc = STP_OK;
  auto visc = [&]() -> int {
    if (!cf.les) return STP_OK;
    if (h->prec == STP_FP64)
      CUDA_TRY(h, launch_viscosity<double>(h->g64, (double*)h->u, (double*)h->v, (double*)h->w, cf.nu,
                                           (double*)h->nu, h->st));
    else
      CUDA_TRY(h, launch_viscosity<float>(h->g32, (float*)h->u, (float*)h->v, (float*)h->w, (float)cf.nu,
                                          (float*)h->nu, h->st));
    return STP_OK;
  };
  switch (term) {
    case STP_TERM_VISCOSITY:
      if ((rc = visc())) return rc;
      return stp_get_fields(h, nullptr, nullptr, nullptr, nullptr, a, where);
    case STP_TERM_EXPLICIT:
    case STP_TERM_DIFFUSION: {
      if (!b || !c) return fail(h, STP_EINVAL, "velocity terms need a, b and c");
      if ((rc = visc())) return rc;
      const double fx = cf.forcing == 0 ? cf.fx : 0.0;
      if (h->prec == STP_FP64) {
        if (term == STP_TERM_EXPLICIT)
          CUDA_TRY(h, launch_explicit_only<double>(h->g64, cf.les != 0, (double*)h->u, (double*)h->v, (double*)h->w,
                                                   (double*)h->nu, cf.nu, fx, (double*)h->tu, (double*)h->tv,
                                                   (double*)h->tw, h->st));
        else
          CUDA_TRY(h, launch_diffusion_only<double>(h->g64, cf.les != 0, (double*)h->u, (double*)h->v, (double*)h->w,
                                                    (double*)h->nu, cf.nu, (double*)h->tu, (double*)h->tv,
                                                    (double*)h->tw, h->st));
      } else {
        if (term == STP_TERM_EXPLICIT)
          CUDA_TRY(h, launch_explicit_only<float>(h->g32, cf.les != 0, (float*)h->u, (float*)h->v, (float*)h->w,
                                                  (float*)h->nu, (float)cf.nu, (float)fx, (float*)h->tu,
                                                  (float*)h->tv, (float*)h->tw, h->st));
        else
          CUDA_TRY(h, launch_diffusion_only<float>(h->g32, cf.les != 0, (float*)h->u, (float*)h->v, (float*)h->w,
                                                   (float*)h->nu, (float)cf.nu, (float*)h->tu, (float*)h->tv,
                                                   (float*)h->tw, h->st));
      }
      if ((rc = get_any(h, a, h->tu, h->nc, where))) return rc;
      if ((rc = get_any(h, b, h->tv, h->nc, where))) return rc;
      if ((rc = get_any(h, c, h->tw, h->nw, where))) return rc;
      break;
    }
    case STP_TERM_DIVERGENCE:
      if (h->prec == STP_FP64)
        CUDA_TRY(h, launch_divergence_rhs<double>(h->g64, (double*)h->u, (double*)h->v, (double*)h->w, 1.0, h->stage,
                                                  h->red, cf.Lz, h->st));
      else
        CUDA_TRY(h, launch_divergence_rhs<float>(h->g32, (float*)h->u, (float*)h->v, (float*)h->w, 1.0, h->stage,
                                                 h->red, cf.Lz, h->st));
      CUDA_TRY(h, cudaMemcpyAsync(a, h->stage, sizeof(double) * h->nc,
                                  where == STP_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->st));
      break;
    case STP_TERM_LAPLACIAN:
      CUDA_TRY(h, launch_laplacian(h->g64, h->p, h->stage, h->st));
      CUDA_TRY(h, cudaMemcpyAsync(a, h->stage, sizeof(double) * h->nc,
                                  where == STP_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->st));
      break;
    default:
      return fail(h, STP_EINVAL, "unknown term");
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return STP_OK;
}

// ---------------------------------------------------------------------------
// batched channels
// ---------------------------------------------------------------------------
}  // extern "C"

// channels of a batch solved in lock step (same SRJ cycle length, FP32)
struct BatchGroup {
  std::vector<stp_handle*> hs;
  std::vector<int> idx;  // positions in the batch
  Group G{};
  void* mem = nullptr;   // device: GState | GChan[n] | soff | voff | pass_on | inner_on
  float sweep_us = 0.f;  // measured time of one grouped sweep over all channels
};

struct stp_batch {
  std::vector<stp_handle*> hs;
  int dev = 0;
  cudaStream_t st = nullptr, cap = nullptr;
  bool own = false;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t x = nullptr;
  int* d_ctr = nullptr;
  int* h_ctr = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  std::vector<BatchGroup> groups;
  std::vector<int> in_group;   // per channel: its group, or -1 (own solve)
  long long step_kernels = 0;  // kernels per step outside the pressure solves
  std::string err;
};

namespace {

int bfail(stp_batch* b, int code, const std::string& m) {
  b->err = m;
  return code;
}

#define BTRY(b, call)                                                                                  \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess) return bfail(b, STP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Channels eligible for a lock-step group: FP32 with refinement, rows of
// float4, no learned guess, no persistent-cycle kernel.  Groups are formed
// per SRJ cycle length when at least two channels share it;
// STP_BATCH_GROUPS=0 keeps every channel on its own solve.
void plan_groups(stp_batch* b) {
  b->in_group.assign(b->hs.size(), -1);
  const char* env = std::getenv("STP_BATCH_GROUPS");
  if (env && std::atoi(env) == 0) return;
  // Size class: only channels of at most 2^17 cells are grouped (their own
  // sweeps are launch-bound; larger channels sweep near the copy rate on
  // their own and would only wait for their group's slowest member);
  // STP_BATCH_GROUP_MAX_CHANNEL=<n> sets the limit (-1: no limit).
  long long max_ch = 1 << 17;
  if (const char* e = std::getenv("STP_BATCH_GROUP_MAX_CHANNEL")) max_ch = std::atoll(e);
  std::map<int, std::vector<int>> byM;
  for (size_t i = 0; i < b->hs.size(); i++) {
    stp_handle* h = b->hs[i];
    if (h->prec != STP_FP32_REFINE || h->nx % 4 || h->net || h->cycle_blocks > 0 || h->cfg.zline) continue;
    if (max_ch >= 0 && (long long)h->nc > max_ch) continue;
    byM[(int)h->omega.size()].push_back((int)i);
  }
  // A group's inner solve touches d, d' and r of all its channels every
  // sweep (12 bytes a cell).  Groups are split into parts whose inner
  // working set fills at most half the L2, so that consecutive sweeps of a
  // part hit in L2 (STP_BATCH_GROUP_CELLS=<n> sets the cap in cells, 0: no
  // split); largest channels first, each into the part with the fewest
  // cells that still has room.
  int l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, b->dev);
  long long cap = l2 > 0 ? (long long)l2 / 2 / 12 : 0;
  if (const char* e = std::getenv("STP_BATCH_GROUP_CELLS")) cap = std::atoll(e);
  for (auto& kv : byM) {
    if (kv.second.size() < 2) continue;
    std::vector<int> order = kv.second;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->hs[a]->nc > b->hs[c]->nc; });
    std::vector<std::vector<int>> parts;
    std::vector<long long> cells;
    for (int i : order) {
      const long long nc = (long long)b->hs[i]->nc;
      int best = -1;
      for (size_t q = 0; q < parts.size(); q++)
        if ((cap <= 0 || cells[q] + nc <= cap) && (best < 0 || cells[q] < cells[best])) best = (int)q;
      if (best < 0) {
        parts.emplace_back();
        cells.push_back(0);
        best = (int)parts.size() - 1;
      }
      parts[best].push_back(i);
      cells[best] += nc;
    }
    for (auto& part : parts) {
      if (part.size() < 2) continue;
      std::sort(part.begin(), part.end());
      BatchGroup grp;
      grp.idx = part;
      for (int i : part) {
        grp.hs.push_back(b->hs[i]);
        b->in_group[i] = (int)b->groups.size();
      }
      grp.G.M = kv.first;
      b->groups.push_back(grp);
    }
  }
}

// voff and the tile total of sweep variant v for the group's channels
bool group_voff(const BatchGroup& grp, int v, std::vector<int>& voff) {
  voff.assign(grp.hs.size() + 1, 0);
  for (size_t c = 0; c < grp.hs.size(); c++) {
    const stp_handle* h = grp.hs[c];
    const int t = group_sweep_tiles(v, h->nx, h->ny, h->nz);
    if (t < 0) return false;
    voff[c + 1] = voff[c] + t;
  }
  return true;
}

// Device tables of a group, and its sweep tile variant: every variant valid
// for all its channels is timed on the whole group (3 warm-up and 20 timed
// grouped sweeps, every channel active, CUDA events) and the fastest kept.
// STP_SWEEP_VARIANT=<v> forces a variant.  All variants compute the same values.
int setup_group(stp_batch* b, BatchGroup& grp) {
  const int n = (int)grp.hs.size();
  const size_t o_ch = align256(sizeof(GState));
  const size_t o_soff = o_ch + align256(sizeof(GChan) * n);
  const size_t o_voff = o_soff + align256(sizeof(int) * (n + 1));
  const size_t o_pass = o_voff + align256(sizeof(int) * (n + 1));
  const size_t o_inner = o_pass + align256(sizeof(int) * n);
  const size_t total = o_inner + align256(sizeof(int) * n);
  BTRY(b, cudaMalloc(&grp.mem, total));
  char* base = (char*)grp.mem;
  Group& G = grp.G;
  G.gs = (GState*)base;
  G.ch = (const GChan*)(base + o_ch);
  G.soff = (const int*)(base + o_soff);
  G.voff = (const int*)(base + o_voff);
  G.pass_on = (int*)(base + o_pass);
  G.inner_on = (int*)(base + o_inner);
  G.n = n;
  std::vector<GChan> ch(n);
  std::vector<int> soff(n + 1, 0);
  for (int c = 0; c < n; c++) {
    stp_handle* h = grp.hs[c];
    GChan& x = ch[c];
    x.g32 = h->g32;
    x.g64 = h->g64;
    x.p = h->p;
    x.b = h->b;
    x.d1 = h->d1;
    x.d2 = h->d2;
    x.r32 = h->r32;
    x.omega = h->d_omega32;
    x.ctl = h->ctl;
    x.red = h->red;
    soff[c + 1] = soff[c] + group_scalar_tiles(h->nx, h->ny, h->nz);
  }
  G.stiles = soff[n];
  BTRY(b, cudaMemcpy(base + o_ch, ch.data(), sizeof(GChan) * n, cudaMemcpyHostToDevice));
  BTRY(b, cudaMemcpy(base + o_soff, soff.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice));
  BTRY(b, cudaMemset(base, 0, o_ch));
  BTRY(b, cudaMemset(base + o_pass, 0, total - o_pass));
  std::vector<int> voff;
  int forced = -1;
  if (const char* env = std::getenv("STP_SWEEP_VARIANT")) forced = std::atoi(env);
  std::vector<int> cand;
  for (int v = 0; v < sweep_variant_count(); v++)
    if (group_voff(grp, v, voff) && (forced < 0 || v == forced)) cand.push_back(v);
  if (cand.empty()) cand.push_back(0);  // every member has nx % 4 == 0: variant 0 always fits
  int best_v = cand[0];
  if (cand.size() > 1) {
    // scratch contents for timing: d = 0, r = 0, every channel active
    for (stp_handle* h : grp.hs) {
      BTRY(b, cudaMemsetAsync(h->d1, 0, sizeof(float) * h->nc, b->st));
      BTRY(b, cudaMemsetAsync(h->r32, 0, sizeof(float) * h->nc, b->st));
    }
    BTRY(b, cudaMemsetAsync(G.inner_on, 1, sizeof(int) * n, b->st));
    std::vector<std::pair<int, float>> timed;
    for (int v : cand) {
      group_voff(grp, v, voff);
      BTRY(b, cudaMemcpyAsync(base + o_voff, voff.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, b->st));
      BTRY(b, cudaStreamSynchronize(b->st));
      G.variant = v;
      G.vtiles = voff[n];
      // 20 grouped sweeps captured into a graph, best of three launches after a warm-up
      cudaGraph_t gr = nullptr;
      cudaGraphExec_t gx = nullptr;
      BTRY(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
      cudaError_t e = cudaSuccess;
      for (int w = 0; w < 20 && e == cudaSuccess; w++) e = launch_group_sweep(G, w % G.M, b->cap);
      const cudaError_t e2 = cudaStreamEndCapture(b->cap, &gr);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&gx, gr, 0);
      float vbest = 1e30f;
      for (int r = 0; r < 4 && e == cudaSuccess; r++) {
        float ms = 0.f;
        e = cudaEventRecord(b->e0, b->st);
        if (e == cudaSuccess) e = cudaGraphLaunch(gx, b->st);
        if (e == cudaSuccess) e = cudaEventRecord(b->e1, b->st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b->e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, b->e0, b->e1);
        if (e == cudaSuccess && r > 0) vbest = std::min(vbest, ms);
      }
      if (gx) cudaGraphExecDestroy(gx);
      if (gr) cudaGraphDestroy(gr);
      if (e != cudaSuccess) return bfail(b, STP_ECUDA, std::string("group sweep autotuner: ") + cudaGetErrorString(e));
      timed.emplace_back(v, vbest * 1e3f / 20.f);
    }
    BTRY(b, cudaMemsetAsync(G.inner_on, 0, sizeof(int) * n, b->st));
    best_v = pick_variant(timed, &grp.sweep_us);
    if (const char* lg = std::getenv("STP_TUNE_LOG")) {
      if (std::atoi(lg)) {
        long long cells = 0;
        for (const stp_handle* h : grp.hs) cells += (long long)h->nc;
        std::fprintf(stderr, "stp: grouped sweep tiles, %d channels, %lld cells (us per sweep):", n, cells);
        for (const auto& t : timed) std::fprintf(stderr, " %d=%.3f", t.first, t.second);
        std::fprintf(stderr, " -> %d\n", best_v);
      }
    }
  }
  group_voff(grp, best_v, voff);
  BTRY(b, cudaMemcpyAsync(base + o_voff, voff.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, b->st));
  BTRY(b, cudaStreamSynchronize(b->st));
  G.variant = best_v;
  G.vtiles = voff[n];
  return STP_OK;
}

// graph pieces of the batch, captured on b->cap
int bcap_begin(stp_batch* b, cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd) {
  BTRY(b, cudaStreamBeginCaptureToGraph(b->cap, g, nd ? deps : nullptr, nullptr, nd, cudaStreamCaptureModeRelaxed));
  return STP_OK;
}
int bcap_end(stp_batch* b, cudaGraph_t g, cudaGraphNode_t* tail) {
  cudaStreamCaptureStatus st;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  if (tail) {
    BTRY(b, cudaStreamGetCaptureInfo(b->cap, &st, nullptr, nullptr, &deps, nullptr, &nd));
    *tail = nd ? deps[nd - 1] : nullptr;
  }
  cudaGraph_t out = g;
  BTRY(b, cudaStreamEndCapture(b->cap, &out));
  return STP_OK;
}
int badd_cond(stp_batch* b, cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle hc,
              cudaGraphConditionalNodeType type, cudaGraph_t* body, cudaGraphNode_t* node) {
  cudaGraphNodeParams prm = {};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = hc;
  prm.conditional.type = type;
  prm.conditional.size = 1;
  BTRY(b, cudaGraphAddNode(node, g, dep ? &dep : nullptr, nullptr, dep ? 1 : 0, &prm));
  *body = prm.conditional.phGraph_out[0];
  return STP_OK;
}

// The lock-step solve of a group after the nodes deps (the end of every
// member's velocity part); *last receives its final node.  Same loop
// structure as one channel's FP32 solve, with grouped kernels.
int append_group_solve(stp_batch* b, BatchGroup& grp, cudaGraph_t G, const std::vector<cudaGraphNode_t>& deps,
                       cudaGraphNode_t* last) {
  int rc;
  cudaGraphConditionalHandle h_pass, h_loop, h_body;
  cudaGraph_t pb, wb, ib;
  cudaGraphNode_t tail, pn, wn, ifn;
  BTRY(b, cudaGraphConditionalHandleCreate(&h_pass, G, 0, cudaGraphCondAssignDefault));
  if ((rc = bcap_begin(b, G, deps.data(), deps.size()))) return rc;
  BTRY(b, launch_group_begin(grp.G, b->cap));
  BTRY(b, launch_group_outer(grp.G, 0, h_pass, b->cap));
  if ((rc = bcap_end(b, G, &tail))) return rc;
  if ((rc = badd_cond(b, G, tail, h_pass, cudaGraphCondTypeWhile, &pb, &pn))) return rc;
  BTRY(b, cudaGraphConditionalHandleCreate(&h_loop, pb, 1, 0));
  if ((rc = bcap_begin(b, pb, nullptr, 0))) return rc;
  BTRY(b, launch_group_pass_begin(grp.G, h_loop, b->cap));
  if ((rc = bcap_end(b, pb, nullptr))) return rc;
  if ((rc = badd_cond(b, pb, leaf_node(pb), h_loop, cudaGraphCondTypeWhile, &wb, &wn))) return rc;
  BTRY(b, cudaGraphConditionalHandleCreate(&h_body, wb, 0, cudaGraphCondAssignDefault));
  if ((rc = bcap_begin(b, wb, nullptr, 0))) return rc;
  BTRY(b, launch_group_check(grp.G, h_loop, h_body, b->cap));
  if ((rc = bcap_end(b, wb, nullptr))) return rc;
  if ((rc = badd_cond(b, wb, leaf_node(wb), h_body, cudaGraphCondTypeIf, &ib, &ifn))) return rc;
  if ((rc = bcap_begin(b, ib, nullptr, 0))) return rc;
  for (int m = 0; m < grp.G.M; m++) BTRY(b, launch_group_sweep(grp.G, m, b->cap));
  if ((rc = bcap_end(b, ib, nullptr))) return rc;
  if ((rc = bcap_begin(b, pb, &wn, 1))) return rc;
  BTRY(b, launch_group_addcorr(grp.G, b->cap));
  BTRY(b, launch_group_outer(grp.G, 1, h_pass, b->cap));
  if ((rc = bcap_end(b, pb, nullptr))) return rc;
  *last = pn;
  return STP_OK;
}

int build_batch_graph(stp_batch* b) {
  plan_groups(b);
  for (BatchGroup& grp : b->groups)
    if (int rc = setup_group(b, grp)) return rc;
  cudaGraph_t G;
  BTRY(b, cudaGraphCreate(&G, 0));
  b->g = G;
  cudaGraphConditionalHandle h_steps;
  BTRY(b, cudaGraphConditionalHandleCreate(&h_steps, G, 0, cudaGraphCondAssignDefault));
  BTRY(b, cudaStreamBeginCaptureToGraph(b->cap, G, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  BTRY(b, launch_batch_begin(b->d_ctr, h_steps, b->cap));
  cudaGraph_t out = G;
  BTRY(b, cudaStreamEndCapture(b->cap, &out));
  cudaGraphNodeParams prm = {};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = h_steps;
  prm.conditional.type = cudaGraphCondTypeWhile;
  prm.conditional.size = 1;
  cudaGraphNode_t root = leaf_node(G), wn;
  BTRY(b, cudaGraphAddNode(&wn, G, &root, nullptr, 1, &prm));
  cudaGraph_t body = prm.conditional.phGraph_out[0];
  // per channel: velocity part -> its own solve, or its group's -> projection
  const size_t n = b->hs.size();
  std::vector<cudaGraphNode_t> pre(n), solved(n), tails;
  b->step_kernels = 0;
  for (size_t i = 0; i < n; i++) {
    stp_handle* h = b->hs[i];
    int rc;
    const long long l0 = h->launches;
    if ((rc = begin_capture(h, body, nullptr))) return bfail(b, rc, h->err);
    rc = h->prec == STP_FP64 ? step_pre<double>(h, h->g64, h->cap) : step_pre<float>(h, h->g32, h->cap);
    if (rc) return bfail(b, rc, h->err);
    if ((rc = end_capture_tail(h, body, &pre[i]))) return bfail(b, rc, h->err);
    b->step_kernels += h->launches - l0;
    if (b->in_group[i] < 0 && (rc = append_solve(h, body, pre[i], &solved[i]))) return bfail(b, rc, h->err);
  }
  // STP_BATCH_GROUP_CHAIN=1: one group's solve after another (each has the
  // L2 to itself); otherwise the groups' solves are independent branches
  const char* chain_env = std::getenv("STP_BATCH_GROUP_CHAIN");
  const bool chain = chain_env && std::atoi(chain_env) != 0;
  cudaGraphNode_t prev_group = nullptr;
  for (BatchGroup& grp : b->groups) {
    std::vector<cudaGraphNode_t> deps;
    for (int i : grp.idx) deps.push_back(pre[i]);
    if (chain && prev_group) deps.push_back(prev_group);
    cudaGraphNode_t last;
    if (int rc = append_group_solve(b, grp, body, deps, &last)) return rc;
    for (int i : grp.idx) solved[i] = last;
    prev_group = last;
  }
  for (size_t i = 0; i < n; i++) {
    stp_handle* h = b->hs[i];
    int rc;
    cudaGraphNode_t post;
    const long long l0 = h->launches;
    if ((rc = begin_capture(h, body, solved[i]))) return bfail(b, rc, h->err);
    rc = h->prec == STP_FP64 ? step_post<double>(h, h->g64, h->cap) : step_post<float>(h, h->g32, h->cap);
    if (rc) return bfail(b, rc, h->err);
    if ((rc = end_capture_tail(h, body, &post))) return bfail(b, rc, h->err);
    b->step_kernels += h->launches - l0;
    tails.push_back(post);
  }
  BTRY(b, cudaStreamBeginCaptureToGraph(b->cap, body, tails.data(), nullptr, tails.size(),
                                        cudaStreamCaptureModeRelaxed));
  BTRY(b, launch_batch_end(b->d_ctr, h_steps, b->cap));
  out = body;
  BTRY(b, cudaStreamEndCapture(b->cap, &out));
  BTRY(b, cudaGraphInstantiate(&b->x, G, 0));
  return STP_OK;
}

}  // namespace

extern "C" {

int stp_batch_create(stp_handle* const* hs, int n, void* stream, stp_batch** out) {
  if (!out || !hs || n < 1) return fail(nullptr, STP_EINVAL, "need at least one handle");
  *out = nullptr;
  for (int i = 0; i < n; i++) {
    if (!hs[i]) return fail(nullptr, STP_EINVAL, "NULL handle");
    if (hs[i]->dev != hs[0]->dev) return fail(nullptr, STP_EINVAL, "all channels must be on one device");
    if (hs[i]->host_solve) return fail(nullptr, STP_EINVAL, "host-driven solves cannot be batched");
    for (int j = 0; j < i; j++)
      if (hs[j] == hs[i]) return fail(nullptr, STP_EINVAL, "a handle appears twice");
  }
  stp_batch* b = new stp_batch();
  b->hs.assign(hs, hs + n);
  b->dev = hs[0]->dev;
  cudaSetDevice(b->dev);
  cudaError_t e = cudaSuccess;
  if (stream) {
    b->st = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
    b->own = true;
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_ctr, sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_ctr, sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaEventCreate(&b->e0);
  if (e == cudaSuccess) e = cudaEventCreate(&b->e1);
  if (e != cudaSuccess) {
    g_init_error = std::string("batch set-up: ") + cudaGetErrorString(e);
    stp_batch_destroy(b);
    return STP_ECUDA;
  }
  *out = b;
  return STP_OK;
}

void stp_batch_destroy(stp_batch* b) {
  if (!b) return;
  cudaSetDevice(b->dev);
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->x) cudaGraphExecDestroy(b->x);
  if (b->g) cudaGraphDestroy(b->g);
  if (b->d_ctr) cudaFree(b->d_ctr);
  if (b->h_ctr) cudaFreeHost(b->h_ctr);
  if (b->e0) cudaEventDestroy(b->e0);
  if (b->e1) cudaEventDestroy(b->e1);
  for (BatchGroup& grp : b->groups)
    if (grp.mem) cudaFree(grp.mem);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->own && b->st) cudaStreamDestroy(b->st);
  delete b;
}

const char* stp_batch_last_error(const stp_batch* b) { return b ? b->err.c_str() : ""; }

int stp_stats_reset(stp_handle* h, int kc) {
  if (!h) return STP_EINVAL;
  if (kc < -1 || kc >= h->nz) return fail(h, STP_EINVAL, "correlation level out of range");
  CUDA_TRY(h, cudaSetDevice(h->dev));
  if (!h->st_mom) {
    cudaError_t e = cudaMalloc((void**)&h->st_mom, sizeof(double) * kStatMoments * h->nz);
    if (e == cudaSuccess) {
      h->allocs.push_back(h->st_mom);
      e = cudaMalloc((void**)&h->st_corr, sizeof(double) * 3 * h->nx);
    }
    if (e != cudaSuccess) {
      h->st_mom = h->st_corr = nullptr;
      return fail(h, STP_ENOMEM, "statistics buffers");
    }
    h->allocs.push_back(h->st_corr);
  }
  h->st_kc = kc < 0 ? h->nz / 2 : kc;
  h->st_n = 0;
  CUDA_TRY(h, cudaMemsetAsync(h->st_mom, 0, sizeof(double) * kStatMoments * h->nz, h->st));
  CUDA_TRY(h, cudaMemsetAsync(h->st_corr, 0, sizeof(double) * 3 * h->nx, h->st));
  return STP_OK;
}

int stp_stats_accumulate(stp_handle* h) {
  if (!h) return STP_EINVAL;
  if (!h->st_mom) return fail(h, STP_EINVAL, "call stp_stats_reset first");
  CUDA_TRY(h, cudaSetDevice(h->dev));
  if (h->prec == STP_FP64)
    CUDA_TRY(h, launch_les_stats<double>(h->nx, h->ny, h->nz, h->st_kc, (const double*)h->u, (const double*)h->v,
                                         (const double*)h->w, h->st_mom, h->st_corr, h->st));
  else
    CUDA_TRY(h, launch_les_stats<float>(h->nx, h->ny, h->nz, h->st_kc, (const float*)h->u, (const float*)h->v,
                                        (const float*)h->w, h->st_mom, h->st_corr, h->st));
  h->st_n++;
  return STP_OK;
}

int stp_stats_read(stp_handle* h, double* moments, double* corr, long long* nsamples, int* kc) {
  if (!h) return STP_EINVAL;
  if (!h->st_mom) return fail(h, STP_EINVAL, "call stp_stats_reset first");
  if (nsamples) *nsamples = h->st_n;
  if (kc) *kc = h->st_kc;
  if (h->st_n == 0) return STP_OK;
  CUDA_TRY(h, cudaSetDevice(h->dev));
  std::vector<double> m((size_t)kStatMoments * h->nz), c((size_t)3 * h->nx);
  CUDA_TRY(h, cudaMemcpyAsync(m.data(), h->st_mom, sizeof(double) * m.size(), cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(c.data(), h->st_corr, sizeof(double) * c.size(), cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  const double inv = 1.0 / ((double)h->st_n * h->nx * h->ny);
  for (double& x : m) x *= inv;
  if (moments) std::copy(m.begin(), m.end(), moments);
  if (corr) {
    // R_cc(d) = <q_c(x + d) q_c(x)> - <q_c>^2 at the correlation level
    for (int comp = 0; comp < 3; comp++) {
      const double mean = m[(size_t)comp * h->nz + h->st_kc];
      for (int d = 0; d < h->nx; d++) corr[comp * h->nx + d] = c[(size_t)comp * h->nx + d] * inv - mean * mean;
    }
  }
  return STP_OK;
}

int stp_sweep_tile(const stp_handle* h, float* us) {
  if (!h) return STP_EINVAL;
  if (us) *us = h->sweep_us;
  return h->sweep_variant;
}

int stp_line_kernel(const stp_handle* h) {
  if (!h || !h->cfg.zline) return -1;
  return h->line_variant;
}

int stp_batch_groups(const stp_batch* b, int max_groups, stp_batch_group* out) {
  if (!b) return STP_EINVAL;
  const int n = (int)b->groups.size();
  for (int i = 0; i < n && i < max_groups && out; i++) {
    const BatchGroup& grp = b->groups[i];
    stp_batch_group& o = out[i];
    o.channels = grp.G.n;
    o.M = grp.G.M;
    o.variant = grp.G.variant;
    o.cells = 0;
    for (const stp_handle* h : grp.hs) o.cells += (long long)h->nc;
    o.sweep_us = grp.sweep_us;
  }
  return n;
}

int stp_batch_step(stp_batch* b, int nsteps, stp_batch_stats* stats, stp_step_stats* per_channel) {
  if (!b || nsteps < 0) return STP_EINVAL;
  BTRY(b, cudaSetDevice(b->dev));
  if (!b->x) {
    if (int rc = build_batch_graph(b)) return rc;
  }
  for (stp_handle* h : b->hs) {
    h->launches = 0;
    if (int rc = arm_solves(h, h->cfg.ptol, h->cfg.pmaxit)) return bfail(b, rc, h->err);
    BTRY(b, cudaStreamSynchronize(h->st));
  }
  for (BatchGroup& grp : b->groups) BTRY(b, cudaMemsetAsync(grp.G.gs, 0, sizeof(GState), b->st));
  b->h_ctr[0] = 0;
  b->h_ctr[1] = nsteps;
  BTRY(b, cudaMemcpyAsync(b->d_ctr, b->h_ctr, sizeof(int) * 2, cudaMemcpyHostToDevice, b->st));
  BTRY(b, cudaEventRecord(b->e0, b->st));
  BTRY(b, cudaGraphLaunch(b->x, b->st));
  BTRY(b, cudaEventRecord(b->e1, b->st));
  BTRY(b, cudaStreamSynchronize(b->st));
  float ms = 0.f;
  BTRY(b, cudaEventElapsedTime(&ms, b->e0, b->e1));
  stp_batch_stats out{};
  out.steps = nsteps;
  out.converged = 1;
  out.gpu_ms = ms;
  // kernels run: the velocity parts and projections, the step counter's
  // begin and per-step end, the channels' own solves and the grouped solves
  out.kernels = 1 + nsteps * (b->step_kernels + 1);
  for (BatchGroup& grp : b->groups) {
    GState gs;
    BTRY(b, cudaMemcpy(&gs, grp.G.gs, sizeof(GState), cudaMemcpyDeviceToHost));
    out.kernels += gs.kernels;
  }
  int status = STP_OK;
  for (size_t i = 0; i < b->hs.size(); i++) {
    stp_handle* h = b->hs[i];
    int rc = sync_scalars(h);
    if (rc) return bfail(b, rc, h->err);
    BTRY(b, cudaMemcpy(h->h_ctl, h->ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost));
    const SolveCtl& c = *h->h_ctl;
    h->step += nsteps;
    h->nhist = (int)std::min<long long>(3, h->nhist + nsteps);
    const int nonconv = nsteps > 0 ? c.nonconv + (c.converged ? 0 : 1) : 0;
    if (nonconv) {
      out.converged = 0;
      status = STP_ENOTCONVERGED;
    }
    if (c.bad || h->h_flag[FL_BAD]) status = STP_EDIVERGED;
    out.cells += (long long)h->nc;
    out.sweeps += nsteps > 0 ? c.tot_sweeps + c.sweeps : 0;
    if (b->in_group[i] < 0 && nsteps > 0) out.kernels += c.tot_kernels + c.kernels;
    if (per_channel) {
      stp_step_stats& st = per_channel[i];
      st.poisson_sweeps = c.sweeps;
      st.refine_passes = c.passes;
      st.converged = nonconv == 0;
      const double nb = h->h_sc[SC_BNORM];
      st.rel_residual = nb > 0 ? c.res / nb : c.res;
      st.ubulk = h->h_sc[SC_BULK] + (h->cfg.forcing == 1 ? h->h_sc[SC_SHIFT] : 0.0);
      st.umax = h->h_sc[SC_UMAX];
      st.dpdx = h->cfg.forcing == 1 ? h->h_sc[SC_SHIFT] / h->cfg.dt : 0.0;
      st.step = h->step;
      st.launches = 0;
      st.solve_sweeps = nsteps > 0 ? c.tot_sweeps + c.sweeps : 0;
      st.solve_ms = 0.0;
    }
  }
  if (stats) *stats = out;
  if (status == STP_EDIVERGED) return bfail(b, status, "NaN or Inf in a channel");
  if (status == STP_ENOTCONVERGED) return bfail(b, status, "a pressure solve hit pmaxit");
  return STP_OK;
}

}  // extern "C"

namespace stp {
// z couplings of the Poisson operator for a channel configuration (used by
// the allocation-free residual entry point)
void poisson_couplings(const stp_config& c, std::vector<double>& cup, std::vector<double>& cdn) {
  const ZGrid z = make_z(c);
  poisson_z(c, z, cup, cdn);
}
void set_thread_error(const std::string& msg) { g_init_error = msg; }
}  // namespace stp
