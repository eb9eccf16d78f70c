// Velocity-side kernels of the projection step (arXiv 1511.07800, Sec. 2.2
// and 3.1): eddy viscosity, explicit terms with the Adams-Bashforth
// combination and the Crank-Nicolson right-hand side, Crank-Nicolson Jacobi
// sweeps, divergence / Poisson right-hand side, velocity correction.
//
// Every kernel handles one output point per thread over an x-y tile of
// 32 x 8 threads and one z level per block row of the grid, reading its
// neighbours through the read-only cache.  x and y wrap periodically; at the
// walls u and v take the mirror ghost (minus the first interior value) and
// the wall planes of w are zero.
#include "device_util.cuh"
#include "stp_internal.cuh"

namespace stp {

namespace {

template <typename T>
struct Pt {
  const Geom<T>& g;
  int i, j, k, im, ip, jm, jp;
  __device__ Pt(const Geom<T>& g_, int i_, int j_, int k_) : g(g_), i(i_), j(j_), k(k_) {
    im = i == 0 ? g.nx - 1 : i - 1;
    ip = i == g.nx - 1 ? 0 : i + 1;
    jm = j == 0 ? g.ny - 1 : j - 1;
    jp = j == g.ny - 1 ? 0 : j + 1;
  }
  __device__ int wx(int a) const { return a < 0 ? a + g.nx : (a >= g.nx ? a - g.nx : a); }
  __device__ int wy(int b) const { return b < 0 ? b + g.ny : (b >= g.ny ? b - g.ny : b); }
  // u or v with the no-slip ghost; a, b already wrapped; c in [-1, nz]
  __device__ T vel(const T* f, int a, int b, int c) const {
    if (c < 0) return -__ldg(f + at(g.nx, g.ny, a, b, 0));
    if (c >= g.nz) return -__ldg(f + at(g.nx, g.ny, a, b, g.nz - 1));
    return __ldg(f + at(g.nx, g.ny, a, b, c));
  }
  // w, c in [0, nz]
  __device__ T wv(const T* f, int a, int b, int c) const { return __ldg(f + at(g.nx, g.ny, a, b, c)); }
};

// Viscosity lookups: constant nu0 without LES; with LES the cell-centred
// field with even reflection at the walls, averaged to edges.
template <typename T, bool LES>
struct Visc {
  const T* nu;
  T nu0;
  int nx, ny, nz;
  __device__ T c(int a, int b, int k) const {
    if (!LES) return nu0;
    k = k < 0 ? 0 : (k >= nz ? nz - 1 : k);
    return __ldg(nu + at(nx, ny, a, b, k));
  }
  // edge quantities; callers pass the two wrapped cell indices on each side
  __device__ T e4(int a0, int a1, int b0, int b1, int k) const {  // xy-edge: cells a0,a1 x b0,b1 at level k
    if (!LES) return nu0;
    return T(0.25) * (c(a0, b0, k) + c(a1, b0, k) + c(a0, b1, k) + c(a1, b1, k));
  }
  __device__ T ez_x(int a0, int a1, int b, int cz) const {  // xz-edge at face cz: cells a0,a1 x cz-1,cz
    if (!LES) return nu0;
    return T(0.25) * (c(a0, b, cz - 1) + c(a1, b, cz - 1) + c(a0, b, cz) + c(a1, b, cz));
  }
  __device__ T ez_y(int a, int b0, int b1, int cz) const {  // yz-edge at face cz: cells b0,b1 x cz-1,cz
    if (!LES) return nu0;
    return T(0.25) * (c(a, b0, cz - 1) + c(a, b1, cz - 1) + c(a, b0, cz) + c(a, b1, cz));
  }
};

// ---------------------------------------------------------------------------
// Sec. 2.2: nu_T = nu + (Cs Delta phi_w)^2 |S|, |S| = sqrt(2 S_ij S_ij);
// off-diagonal strain on its edges, averaged from the four edges around the
// centre.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBX* kBY) k_viscosity(Geom<T> g, const T* __restrict__ u,
                                                         const T* __restrict__ v, const T* __restrict__ w,
                                                         T nu0, T* __restrict__ nu) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  Pt<T> P(g, i, j, k);
  const int im = P.im, ip = P.ip, jm = P.jm, jp = P.jp;
  const T s11 = (P.vel(u, ip, j, k) - P.vel(u, i, j, k)) * g.idx;
  const T s22 = (P.vel(v, i, jp, k) - P.vel(v, i, j, k)) * g.idy;
  const T s33 = (P.wv(w, i, j, k + 1) - P.wv(w, i, j, k)) * __ldg(g.idz + k);
  auto e12 = [&](int a, int am, int b, int bm) {
    return T(0.5) * ((P.vel(u, a, b, k) - P.vel(u, a, bm, k)) * g.idy + (P.vel(v, a, b, k) - P.vel(v, am, b, k)) * g.idx);
  };
  auto e13 = [&](int a, int am, int c) {
    return T(0.5) * ((P.vel(u, a, j, c) - P.vel(u, a, j, c - 1)) * __ldg(g.idzf + c) +
                     (P.wv(w, a, j, c) - P.wv(w, am, j, c)) * g.idx);
  };
  auto e23 = [&](int b, int bm, int c) {
    return T(0.5) * ((P.vel(v, i, b, c) - P.vel(v, i, b, c - 1)) * __ldg(g.idzf + c) +
                     (P.wv(w, i, b, c) - P.wv(w, i, bm, c)) * g.idy);
  };
  const T s12 = T(0.25) * (e12(i, im, j, jm) + e12(ip, i, j, jm) + e12(i, im, jp, j) + e12(ip, i, jp, j));
  const T s13 = T(0.25) * (e13(i, im, k) + e13(ip, i, k) + e13(i, im, k + 1) + e13(ip, i, k + 1));
  const T s23 = T(0.25) * (e23(j, jm, k) + e23(jp, j, k) + e23(j, jm, k + 1) + e23(jp, j, k + 1));
  const T smag = sqrt(T(2) * (s11 * s11 + s22 * s22 + s33 * s33) + T(4) * (s12 * s12 + s13 * s13 + s23 * s23));
  nu[at(g.nx, g.ny, i, j, k)] = nu0 + __ldg(g.lm2 + k) * smag;
}

// ---------------------------------------------------------------------------
// Sec. 3.1 terms at one point.
// ---------------------------------------------------------------------------

// advective form u_j d_j u_i
template <typename T>
__device__ __forceinline__ T adv_u(const Pt<T>& P, const T* u, const T* v, const T* w) {
  const Geom<T>& g = P.g;
  const int i = P.i, j = P.j, k = P.k;
  const T vb = T(0.25) * (P.vel(v, P.im, j, k) + P.vel(v, i, j, k) + P.vel(v, P.im, P.jp, k) + P.vel(v, i, P.jp, k));
  const T wb = T(0.25) * (P.wv(w, P.im, j, k) + P.wv(w, i, j, k) + P.wv(w, P.im, j, k + 1) + P.wv(w, i, j, k + 1));
  const T dudx = (P.vel(u, P.ip, j, k) - P.vel(u, P.im, j, k)) * g.hidx;
  const T dudy = (P.vel(u, i, P.jp, k) - P.vel(u, i, P.jm, k)) * g.hidy;
  const T dudz = (P.vel(u, i, j, k + 1) - P.vel(u, i, j, k - 1)) * __ldg(g.i2dzc + k);
  return P.vel(u, i, j, k) * dudx + vb * dudy + wb * dudz;
}
template <typename T>
__device__ __forceinline__ T adv_v(const Pt<T>& P, const T* u, const T* v, const T* w) {
  const Geom<T>& g = P.g;
  const int i = P.i, j = P.j, k = P.k;
  const T ub = T(0.25) * (P.vel(u, i, P.jm, k) + P.vel(u, P.ip, P.jm, k) + P.vel(u, i, j, k) + P.vel(u, P.ip, j, k));
  const T wb = T(0.25) * (P.wv(w, i, P.jm, k) + P.wv(w, i, j, k) + P.wv(w, i, P.jm, k + 1) + P.wv(w, i, j, k + 1));
  const T dvdx = (P.vel(v, P.ip, j, k) - P.vel(v, P.im, j, k)) * g.hidx;
  const T dvdy = (P.vel(v, i, P.jp, k) - P.vel(v, i, P.jm, k)) * g.hidy;
  const T dvdz = (P.vel(v, i, j, k + 1) - P.vel(v, i, j, k - 1)) * __ldg(g.i2dzc + k);
  return ub * dvdx + P.vel(v, i, j, k) * dvdy + wb * dvdz;
}
// w at an interior face c = P.k
template <typename T>
__device__ __forceinline__ T adv_w(const Pt<T>& P, const T* u, const T* v, const T* w) {
  const Geom<T>& g = P.g;
  const int i = P.i, j = P.j, c = P.k;
  const T ub = T(0.25) * (P.vel(u, i, j, c - 1) + P.vel(u, P.ip, j, c - 1) + P.vel(u, i, j, c) + P.vel(u, P.ip, j, c));
  const T vb = T(0.25) * (P.vel(v, i, j, c - 1) + P.vel(v, i, P.jp, c - 1) + P.vel(v, i, j, c) + P.vel(v, i, P.jp, c));
  const T dwdx = (P.wv(w, P.ip, j, c) - P.wv(w, P.im, j, c)) * g.hidx;
  const T dwdy = (P.wv(w, i, P.jp, c) - P.wv(w, i, P.jm, c)) * g.hidy;
  const T dwdz = (P.wv(w, i, j, c + 1) - P.wv(w, i, j, c - 1)) * __ldg(g.idzw + c);
  return ub * dwdx + vb * dwdy + P.wv(w, i, j, c) * dwdz;
}

// Viscous fluxes.  For each component the "diffusive-like" part
// d_j(nu d_j u_i) (Crank-Nicolson) and the "convective-like" part
// d_j(nu d_i u_j) (Adams-Bashforth) share the edge viscosities.
template <typename T, bool LES>
struct ViscU {
  T diff, cross, diag;  // D u, C u, diagonal weight of D
};

template <typename T, bool LES>
__device__ __forceinline__ ViscU<T, LES> visc_u(const Pt<T>& P, const Visc<T, LES>& N, const T* u, const T* v,
                                                const T* w, bool need_cross) {
  const Geom<T>& g = P.g;
  const int i = P.i, j = P.j, k = P.k, im = P.im, ip = P.ip, jm = P.jm, jp = P.jp;
  const T c = P.vel(u, i, j, k);
  const T nxp = N.c(i, j, k), nxm = N.c(im, j, k);
  const T nyp = N.e4(im, i, j, jp, k), nym = N.e4(im, i, jm, j, k);
  const T nzp = N.ez_x(im, i, j, k + 1), nzm = N.ez_x(im, i, j, k);
  const T idz = __ldg(g.idz + k), izp = __ldg(g.idzf + k + 1), izm = __ldg(g.idzf + k);
  const T fx = (nxp * (P.vel(u, ip, j, k) - c) - nxm * (c - P.vel(u, im, j, k))) * g.idx2;
  const T fy = (nyp * (P.vel(u, i, jp, k) - c) - nym * (c - P.vel(u, i, jm, k))) * g.idy2;
  const T fz = (nzp * (P.vel(u, i, j, k + 1) - c) * izp - nzm * (c - P.vel(u, i, j, k - 1)) * izm) * idz;
  ViscU<T, LES> r;
  r.diff = fx + fy + fz;
  const T gu = (k == g.nz - 1) ? T(2) : T(1), gd = (k == 0) ? T(2) : T(1);
  r.diag = (nxp + nxm) * g.idx2 + (nyp + nym) * g.idy2 + (gu * nzp * izp + gd * nzm * izm) * idz;
  r.cross = T(0);
  if (need_cross) {
    const T cy = (nyp * (P.vel(v, i, jp, k) - P.vel(v, im, jp, k)) - nym * (P.vel(v, i, j, k) - P.vel(v, im, j, k))) * g.idxdy;
    const T cz = (nzp * (P.wv(w, i, j, k + 1) - P.wv(w, im, j, k + 1)) - nzm * (P.wv(w, i, j, k) - P.wv(w, im, j, k))) *
                 g.idx * idz;
    r.cross = fx + cy + cz;
  }
  return r;
}

template <typename T, bool LES>
__device__ __forceinline__ ViscU<T, LES> visc_v(const Pt<T>& P, const Visc<T, LES>& N, const T* u, const T* v,
                                                const T* w, bool need_cross) {
  const Geom<T>& g = P.g;
  const int i = P.i, j = P.j, k = P.k, im = P.im, ip = P.ip, jm = P.jm, jp = P.jp;
  const T c = P.vel(v, i, j, k);
  const T nxp = N.e4(i, ip, jm, j, k), nxm = N.e4(im, i, jm, j, k);
  const T nyp = N.c(i, j, k), nym = N.c(i, jm, k);
  const T nzp = N.ez_y(i, jm, j, k + 1), nzm = N.ez_y(i, jm, j, k);
  const T idz = __ldg(g.idz + k), izp = __ldg(g.idzf + k + 1), izm = __ldg(g.idzf + k);
  const T fx = (nxp * (P.vel(v, ip, j, k) - c) - nxm * (c - P.vel(v, im, j, k))) * g.idx2;
  const T fy = (nyp * (P.vel(v, i, jp, k) - c) - nym * (c - P.vel(v, i, jm, k))) * g.idy2;
  const T fz = (nzp * (P.vel(v, i, j, k + 1) - c) * izp - nzm * (c - P.vel(v, i, j, k - 1)) * izm) * idz;
  ViscU<T, LES> r;
  r.diff = fx + fy + fz;
  const T gu = (k == g.nz - 1) ? T(2) : T(1), gd = (k == 0) ? T(2) : T(1);
  r.diag = (nxp + nxm) * g.idx2 + (nyp + nym) * g.idy2 + (gu * nzp * izp + gd * nzm * izm) * idz;
  r.cross = T(0);
  if (need_cross) {
    const T cx = (nxp * (P.vel(u, ip, j, k) - P.vel(u, ip, jm, k)) - nxm * (P.vel(u, i, j, k) - P.vel(u, i, jm, k))) * g.idxdy;
    const T cz = (nzp * (P.wv(w, i, j, k + 1) - P.wv(w, i, jm, k + 1)) - nzm * (P.wv(w, i, j, k) - P.wv(w, i, jm, k))) *
                 g.idy * idz;
    r.cross = cx + fy + cz;
  }
  return r;
}

// w at interior face c
template <typename T, bool LES>
__device__ __forceinline__ ViscU<T, LES> visc_w(const Pt<T>& P, const Visc<T, LES>& N, const T* u, const T* v,
                                                const T* w, bool need_cross) {
  const Geom<T>& g = P.g;
  const int i = P.i, j = P.j, c = P.k, im = P.im, ip = P.ip, jm = P.jm, jp = P.jp;
  const T ctr = P.wv(w, i, j, c);
  const T nxp = N.ez_x(i, ip, j, c), nxm = N.ez_x(im, i, j, c);
  const T nyp = N.ez_y(i, j, jp, c), nym = N.ez_y(i, jm, j, c);
  const T nzp = N.c(i, j, c), nzm = N.c(i, j, c - 1);
  const T ih = __ldg(g.ihz + c), izp = __ldg(g.idz + c), izm = __ldg(g.idz + c - 1);
  const T fx = (nxp * (P.wv(w, ip, j, c) - ctr) - nxm * (ctr - P.wv(w, im, j, c))) * g.idx2;
  const T fy = (nyp * (P.wv(w, i, jp, c) - ctr) - nym * (ctr - P.wv(w, i, jm, c))) * g.idy2;
  const T fz = (nzp * (P.wv(w, i, j, c + 1) - ctr) * izp - nzm * (ctr - P.wv(w, i, j, c - 1)) * izm) * ih;
  ViscU<T, LES> r;
  r.diff = fx + fy + fz;
  r.diag = (nxp + nxm) * g.idx2 + (nyp + nym) * g.idy2 + (nzp * izp + nzm * izm) * ih;
  r.cross = T(0);
  if (need_cross) {
    const T cx = (nxp * (P.vel(u, ip, j, c) - P.vel(u, ip, j, c - 1)) - nxm * (P.vel(u, i, j, c) - P.vel(u, i, j, c - 1))) *
                 g.idx * ih;
    const T cy = (nyp * (P.vel(v, i, jp, c) - P.vel(v, i, jp, c - 1)) - nym * (P.vel(v, i, j, c) - P.vel(v, i, j, c - 1))) *
                 g.idy * ih;
    r.cross = cx + cy + fz;
  }
  return r;
}

// ---------------------------------------------------------------------------
// Explicit terms at time n, AB combination, CN right-hand side:
//   N^n = -u.grad u + C(u) + f e_x
//   rhs = u^n + dt (b0 N^n + b1 N^{n-1} + b2 N^{n-2}) + dt/2 D(u^n)
// grid z covers levels 0..nz (the last level only carries w).
// ---------------------------------------------------------------------------
template <typename T, bool LES>
__global__ void __launch_bounds__(kBX* kBY) k_momentum(Geom<T> g, const T* __restrict__ u, const T* __restrict__ v,
                                                        const T* __restrict__ w, Visc<T, LES> N, T fx, Hist<T> H,
                                                        T dt, T* __restrict__ ru, T* __restrict__ rv,
                                                        T* __restrict__ rw) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  // history slots and Adams-Bashforth coefficients of step n
  const int n = __ldg(H.step);
  const int s0 = n % 3, s1 = (n + 2) % 3, s2 = (n + 1) % 3;
  T b0 = T(1), b1 = T(0), b2 = T(0);
  if (n == 1) {
    b0 = T(1.5);
    b1 = T(-0.5);
  } else if (n >= 2) {
    b0 = T(23.0 / 12.0);
    b1 = T(-16.0 / 12.0);
    b2 = T(5.0 / 12.0);
  }
  // slot pointers by selection (a runtime index into the parameter arrays
  // would copy them to local memory)
  auto slot = [](T* const* a, int sl) { return sl == 0 ? a[0] : sl == 1 ? a[1] : a[2]; };
  T* __restrict__ Nu0 = slot(H.u, s0);
  T* __restrict__ Nv0 = slot(H.v, s0);
  T* __restrict__ Nw0 = slot(H.w, s0);
  const T* __restrict__ Nu1 = slot(H.u, s1);
  const T* __restrict__ Nv1 = slot(H.v, s1);
  const T* __restrict__ Nw1 = slot(H.w, s1);
  const T* __restrict__ Nu2 = slot(H.u, s2);
  const T* __restrict__ Nv2 = slot(H.v, s2);
  const T* __restrict__ Nw2 = slot(H.w, s2);
  Pt<T> P(g, i, j, k);
  const int q = at(g.nx, g.ny, i, j, k);
  const T hdt = T(0.5) * dt;
  // a history level whose coefficient is zero is not read: after the fields
  // are set its slot may hold anything, even the Inf of a run that diverged
  auto hist = [&](const T* __restrict__ f, int level) { return n >= level ? __ldg(f + q) : T(0); };
  if (k < g.nz) {
    const ViscU<T, LES> a = visc_u<T, LES>(P, N, u, v, w, true);
    const T n0 = -adv_u(P, u, v, w) + a.cross + fx;
    Nu0[q] = n0;
    ru[q] = __ldg(u + q) + dt * (b0 * n0 + b1 * hist(Nu1, 1) + b2 * hist(Nu2, 2)) + hdt * a.diff;
    const ViscU<T, LES> bb = visc_v<T, LES>(P, N, u, v, w, true);
    const T m0 = -adv_v(P, u, v, w) + bb.cross;
    Nv0[q] = m0;
    rv[q] = __ldg(v + q) + dt * (b0 * m0 + b1 * hist(Nv1, 1) + b2 * hist(Nv2, 2)) + hdt * bb.diff;
  }
  if (k == 0 || k == g.nz) {
    Nw0[q] = T(0);
    rw[q] = T(0);
  } else {
    const ViscU<T, LES> c = visc_w<T, LES>(P, N, u, v, w, true);
    const T l0 = -adv_w(P, u, v, w) + c.cross;
    Nw0[q] = l0;
    rw[q] = __ldg(w + q) + dt * (b0 * l0 + b1 * hist(Nw1, 1) + b2 * hist(Nw2, 2)) + hdt * c.diff;
  }
}

// Explicit terms only (checks).
template <typename T, bool LES>
__global__ void k_explicit(Geom<T> g, const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ w,
                           Visc<T, LES> N, T fx, T* Nu, T* Nv, T* Nw) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  Pt<T> P(g, i, j, k);
  const int q = at(g.nx, g.ny, i, j, k);
  if (k < g.nz) {
    Nu[q] = -adv_u(P, u, v, w) + visc_u<T, LES>(P, N, u, v, w, true).cross + fx;
    Nv[q] = -adv_v(P, u, v, w) + visc_v<T, LES>(P, N, u, v, w, true).cross;
  }
  Nw[q] = (k == 0 || k == g.nz) ? T(0) : -adv_w(P, u, v, w) + visc_w<T, LES>(P, N, u, v, w, true).cross;
}

template <typename T, bool LES>
__global__ void k_diffusion(Geom<T> g, const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ w,
                            Visc<T, LES> N, T* Du, T* Dv, T* Dw) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  Pt<T> P(g, i, j, k);
  const int q = at(g.nx, g.ny, i, j, k);
  if (k < g.nz) {
    Du[q] = visc_u<T, LES>(P, N, u, v, w, false).diff;
    Dv[q] = visc_v<T, LES>(P, N, u, v, w, false).diff;
  }
  Dw[q] = (k == 0 || k == g.nz) ? T(0) : visc_w<T, LES>(P, N, u, v, w, false).diff;
}

// ---------------------------------------------------------------------------
// One Jacobi sweep of (I - dt/2 D) a = rhs for the three components:
//   a_new = (rhs + dt/2 (D a + S_D a)) / (1 + dt/2 S_D)
// ---------------------------------------------------------------------------
template <typename T, bool LES>
__global__ void __launch_bounds__(kBX* kBY) k_cn_sweep(Geom<T> g, Visc<T, LES> N, T hdt, const T* __restrict__ ru,
                                                        const T* __restrict__ rv, const T* __restrict__ rw,
                                                        const T* __restrict__ au, const T* __restrict__ av,
                                                        const T* __restrict__ aw, T* __restrict__ ou,
                                                        T* __restrict__ ov, T* __restrict__ ow) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  Pt<T> P(g, i, j, k);
  const int q = at(g.nx, g.ny, i, j, k);
  if (k < g.nz) {
    const ViscU<T, LES> a = visc_u<T, LES>(P, N, au, av, aw, false);
    ou[q] = (__ldg(ru + q) + hdt * (a.diff + a.diag * __ldg(au + q))) / (T(1) + hdt * a.diag);
    const ViscU<T, LES> b = visc_v<T, LES>(P, N, au, av, aw, false);
    ov[q] = (__ldg(rv + q) + hdt * (b.diff + b.diag * __ldg(av + q))) / (T(1) + hdt * b.diag);
  }
  if (k == 0 || k == g.nz) {
    ow[q] = T(0);
  } else {
    const ViscU<T, LES> c = visc_w<T, LES>(P, N, au, av, aw, false);
    ow[q] = (__ldg(rw + q) + hdt * (c.diff + c.diag * __ldg(aw + q))) / (T(1) + hdt * c.diag);
  }
}

// ---------------------------------------------------------------------------
// One z-line Jacobi sweep of (I - dt/2 D) a = rhs for the three components:
// per column the z couplings of D stay implicit and the x-y neighbours come
// from the previous iterate a,
//   (1 + h S_D) x_k - h cz+_k x_{k+1} - h cz-_k x_{k-1}
//       = rhs_k + h sum_{x-y nb} c_nb a_nb,
// solved by the Thomas algorithm.  One thread per column and component
// (blockIdx.z: u, v, w), consecutive threads along x; the forward
// elimination keeps (c'_k, d'_k) in the scratch array, the back
// substitution reads them.  S_D, the couplings and the wall ghosts are those
// of the point sweep (visc_u / visc_v / visc_w).
// ---------------------------------------------------------------------------
template <typename T>
struct Pair;
template <>
struct Pair<float> {
  using V = float2;
};
template <>
struct Pair<double> {
  using V = double2;
};

template <typename T, bool LES>
__global__ void __launch_bounds__(128) k_cn_line(Geom<T> g, Visc<T, LES> N, T h, const T* __restrict__ ru,
                                                  const T* __restrict__ rv, const T* __restrict__ rw,
                                                  const T* __restrict__ au, const T* __restrict__ av,
                                                  const T* __restrict__ aw, T* __restrict__ ou, T* __restrict__ ov,
                                                  T* __restrict__ ow, typename Pair<T>::V* __restrict__ scr) {
  using V2 = typename Pair<T>::V;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, comp = blockIdx.z;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  if (i >= nx) return;
  const int im = i == 0 ? nx - 1 : i - 1, ip = i == nx - 1 ? 0 : i + 1;
  const int jm = j == 0 ? ny - 1 : j - 1, jp = j == ny - 1 ? 0 : j + 1;
  const int plane = nx * ny, c0 = j * nx + i;
  V2* __restrict__ S = scr + (size_t)comp * (nz + 1) * plane;
  const T idx2 = g.idx2, idy2 = g.idy2;
  // cell viscosity at (a, b) of level k, even reflection at the walls
  auto nuc = [&](int a, int b, int k) -> T {
    if (!LES) return N.nu0;
    k = k < 0 ? 0 : (k >= nz ? nz - 1 : k);
    return __ldg(N.nu + k * plane + b * nx + a);
  };
  T cprev = T(0), dprev = T(0);
  if (comp < 2) {
    // u: cells (im, i) of rows j (levels k-1, k, k+1), jp and jm (level k);
    // v: cells (i) of rows j, jm (levels k-1, k, k+1), ip and im of rows jm, j (level k).
    // The two cells carried along z are A (im, j | i, jm) and B (i, j).
    const int aA = comp == 0 ? im : i, bA = comp == 0 ? j : jm;
    const T* __restrict__ a = comp == 0 ? au : av;
    const T* __restrict__ r = comp == 0 ? ru : rv;
    T* __restrict__ o = comp == 0 ? ou : ov;
    T Am = nuc(aA, bA, -1), Bm = nuc(i, j, -1), A0 = nuc(aA, bA, 0), B0 = nuc(i, j, 0);
#pragma unroll 4
    for (int k = 0; k < nz; k++) {
      const int lev = k * plane;
      const T Ap = nuc(aA, bA, k + 1), Bp = nuc(i, j, k + 1);
      T nxp, nxm, nyp, nym;
      if (comp == 0) {
        const T c1 = nuc(im, jp, k), c2 = nuc(i, jp, k), c3 = nuc(im, jm, k), c4 = nuc(i, jm, k);
        nxp = B0;
        nxm = A0;
        nyp = T(0.25) * (A0 + B0 + c1 + c2);
        nym = T(0.25) * (c3 + c4 + A0 + B0);
      } else {
        const T c1 = nuc(ip, jm, k), c2 = nuc(ip, j, k), c3 = nuc(im, jm, k), c4 = nuc(im, j, k);
        nxp = T(0.25) * (A0 + c1 + B0 + c2);
        nxm = T(0.25) * (c3 + A0 + c4 + B0);
        nyp = B0;
        nym = A0;
      }
      const T nzp = T(0.25) * (A0 + B0 + Ap + Bp), nzm = T(0.25) * (Am + Bm + A0 + B0);
      const T idz = __ldg(g.idz + k), izp = __ldg(g.idzf + k + 1), izm = __ldg(g.idzf + k);
      const T gu = (k == nz - 1) ? T(2) : T(1), gd = (k == 0) ? T(2) : T(1);
      const T sd = (nxp + nxm) * idx2 + (nyp + nym) * idy2 + (gu * nzp * izp + gd * nzm * izm) * idz;
      const T xy = (nxp * __ldg(a + lev + j * nx + ip) + nxm * __ldg(a + lev + j * nx + im)) * idx2 +
                   (nyp * __ldg(a + lev + jp * nx + i) + nym * __ldg(a + lev + jm * nx + i)) * idy2;
      const T lo = k > 0 ? -h * nzm * izm * idz : T(0);
      const T up = k < nz - 1 ? -h * nzp * izp * idz : T(0);
      const T inv = T(1) / ((T(1) + h * sd) - lo * cprev);
      cprev = up * inv;
      dprev = (__ldg(r + lev + c0) + h * xy - lo * dprev) * inv;
      S[lev + c0] = V2{cprev, dprev};
      Am = A0;
      Bm = B0;
      A0 = Ap;
      B0 = Bp;
    }
    T x = T(0);
#pragma unroll 4
    for (int k = nz - 1; k >= 0; k--) {
      const V2 cd = S[k * plane + c0];
      x = cd.y - cd.x * x;
      o[k * plane + c0] = x;
    }
  } else {
    // w on the interior faces 1..nz-1 (the wall faces are zero): cells
    // (i, j), (ip, j), (im, j), (i, jp), (i, jm) of levels c-1 and c
    ow[c0] = T(0);
    ow[nz * plane + c0] = T(0);
    T q0 = nuc(i, j, 0), q1 = nuc(ip, j, 0), q2 = nuc(im, j, 0), q3 = nuc(i, jp, 0), q4 = nuc(i, jm, 0);
#pragma unroll 4
    for (int c = 1; c < nz; c++) {
      const int lev = c * plane;
      const T p0 = nuc(i, j, c), p1 = nuc(ip, j, c), p2 = nuc(im, j, c), p3 = nuc(i, jp, c), p4 = nuc(i, jm, c);
      const T nxp = T(0.25) * (q0 + q1 + p0 + p1), nxm = T(0.25) * (q2 + q0 + p2 + p0);
      const T nyp = T(0.25) * (q0 + q3 + p0 + p3), nym = T(0.25) * (q4 + q0 + p4 + p0);
      const T nzp = p0, nzm = q0;
      const T ih = __ldg(g.ihz + c), izp = __ldg(g.idz + c), izm = __ldg(g.idz + c - 1);
      const T sd = (nxp + nxm) * idx2 + (nyp + nym) * idy2 + (nzp * izp + nzm * izm) * ih;
      const T xy = (nxp * __ldg(aw + lev + j * nx + ip) + nxm * __ldg(aw + lev + j * nx + im)) * idx2 +
                   (nyp * __ldg(aw + lev + jp * nx + i) + nym * __ldg(aw + lev + jm * nx + i)) * idy2;
      const T lo = c > 1 ? -h * nzm * izm * ih : T(0);
      const T up = c < nz - 1 ? -h * nzp * izp * ih : T(0);
      const T inv = T(1) / ((T(1) + h * sd) - lo * cprev);
      cprev = up * inv;
      dprev = (__ldg(rw + lev + c0) + h * xy - lo * dprev) * inv;
      S[lev + c0] = V2{cprev, dprev};
      q0 = p0;
      q1 = p1;
      q2 = p2;
      q3 = p3;
      q4 = p4;
    }
    T x = T(0);
#pragma unroll 4
    for (int c = nz - 1; c >= 1; c--) {
      const V2 cd = S[c * plane + c0];
      x = cd.y - cd.x * x;
      ow[c * plane + c0] = x;
    }
  }
}

// The z-line Crank-Nicolson sweep in level chunks.  Within a step nu_T is
// fixed, so the column matrices of every sweep are the same: the forward
// pivots m_k of each column (one-sided Thomas from the bottom wall,
// m_0 = di_0, m_k = di_k - lo_k up_{k-1} / m_{k-1}) are formed once per
// step (k_cn_pivots, 1/m_k stored), and each sweep then runs two linear
// recurrences per column,
//   y_k = rhs'_k / m_k + f_k y_{k-1},   f_k = -lo_k / m_k,
//   x_k = y_k + e_k x_{k+1},            e_k = -up_k / m_k,
// with rhs'_k = rhs_k + h (x-y neighbour terms of the previous iterate).
// The rows of a column are cut into NCH chunks; each thread holds one
// column's rows of one chunk in registers, runs each recurrence inside the
// chunk from zero and adds the carry entering the chunk times the running
// product of its coefficients (the carries come from the chunk boundary
// values in shared memory).  In exact arithmetic this is the Thomas solve
// of k_cn_line; the rounding differs by a few units in the last place.
//
// Row m of component comp (u, v: level m; w: interior face m + 1) of column
// (i, j): lo x_{m-1} + di x_m + up x_{m+1} = rhs_m + h xy, the coefficients
// and wall ghosts of the point sweep (visc_u / visc_v / visc_w); xy only
// when a is given.
template <typename T>
struct CnRow {
  T lo, di, up, xy;
};

template <typename T, bool LES>
__device__ __forceinline__ CnRow<T> cn_row(const Geom<T>& g, const Visc<T, LES>& N, T h, int comp, int i, int j,
                                           int m, const T* __restrict__ a) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int im = i == 0 ? nx - 1 : i - 1, ip = i == nx - 1 ? 0 : i + 1;
  const int jm = j == 0 ? ny - 1 : j - 1, jp = j == ny - 1 ? 0 : j + 1;
  const int plane = nx * ny;
  const T idx2 = g.idx2, idy2 = g.idy2;
  CnRow<T> r;
  T nxp, nxm, nyp, nym, sd;
  int lev;
  if (comp < 2) {
    const int k = m;
    lev = k * plane;
    const int aA = comp == 0 ? im : i, bA = comp == 0 ? j : jm;
    const T A0 = N.c(aA, bA, k), B0 = N.c(i, j, k);
    const T Am = N.c(aA, bA, k - 1), Bm = N.c(i, j, k - 1), Ap = N.c(aA, bA, k + 1), Bp = N.c(i, j, k + 1);
    if (comp == 0) {
      nxp = B0;
      nxm = A0;
      nyp = T(0.25) * (A0 + B0 + N.c(im, jp, k) + N.c(i, jp, k));
      nym = T(0.25) * (N.c(im, jm, k) + N.c(i, jm, k) + A0 + B0);
    } else {
      nxp = T(0.25) * (A0 + N.c(ip, jm, k) + B0 + N.c(ip, j, k));
      nxm = T(0.25) * (N.c(im, jm, k) + A0 + N.c(im, j, k) + B0);
      nyp = B0;
      nym = A0;
    }
    const T nzp = T(0.25) * (A0 + B0 + Ap + Bp), nzm = T(0.25) * (Am + Bm + A0 + B0);
    const T idz = __ldg(g.idz + k), izp = __ldg(g.idzf + k + 1), izm = __ldg(g.idzf + k);
    const T gu = (k == nz - 1) ? T(2) : T(1), gd = (k == 0) ? T(2) : T(1);
    sd = (nxp + nxm) * idx2 + (nyp + nym) * idy2 + (gu * nzp * izp + gd * nzm * izm) * idz;
    r.lo = k > 0 ? -h * nzm * izm * idz : T(0);
    r.up = k < nz - 1 ? -h * nzp * izp * idz : T(0);
  } else {
    const int c = m + 1;
    lev = c * plane;
    const T p0 = N.c(i, j, c), p1 = N.c(ip, j, c), p2 = N.c(im, j, c), p3 = N.c(i, jp, c), p4 = N.c(i, jm, c);
    const T q0 = N.c(i, j, c - 1), q1 = N.c(ip, j, c - 1), q2 = N.c(im, j, c - 1), q3 = N.c(i, jp, c - 1),
            q4 = N.c(i, jm, c - 1);
    nxp = T(0.25) * (q0 + q1 + p0 + p1);
    nxm = T(0.25) * (q2 + q0 + p2 + p0);
    nyp = T(0.25) * (q0 + q3 + p0 + p3);
    nym = T(0.25) * (q4 + q0 + p4 + p0);
    const T nzp = p0, nzm = q0;
    const T ih = __ldg(g.ihz + c), izp = __ldg(g.idz + c), izm = __ldg(g.idz + c - 1);
    sd = (nxp + nxm) * idx2 + (nyp + nym) * idy2 + (nzp * izp + nzm * izm) * ih;
    r.lo = c > 1 ? -h * nzm * izm * ih : T(0);
    r.up = c < nz - 1 ? -h * nzp * izp * ih : T(0);
  }
  r.di = T(1) + h * sd;
  r.xy = a ? (nxp * __ldg(a + lev + j * nx + ip) + nxm * __ldg(a + lev + j * nx + im)) * idx2 +
                 (nyp * __ldg(a + lev + jp * nx + i) + nym * __ldg(a + lev + jm * nx + i)) * idy2
           : T(0);
  return r;
}

// 1/m_k of every column and component (piv: three arrays of (nz + 1)
// levels x ny x nx, row m at level m for u and v, at face m + 1 for w);
// one thread a column and component.
template <typename T, bool LES>
__global__ void __launch_bounds__(128) k_cn_pivots(Geom<T> g, Visc<T, LES> N, T h, T* __restrict__ piv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, comp = blockIdx.z;
  if (i >= g.nx) return;
  const int plane = g.nx * g.ny, n = comp < 2 ? g.nz : g.nz - 1, off = comp < 2 ? 0 : 1;
  T* __restrict__ P = piv + (size_t)comp * (g.nz + 1) * plane + j * g.nx + i;
  T cp = T(0);
  for (int m = 0; m < n; m++) {
    const CnRow<T> r = cn_row<T, LES>(g, N, h, comp, i, j, m, nullptr);
    const T inv = T(1) / (r.di - r.lo * cp);
    cp = r.up * inv;
    P[(m + off) * plane] = inv;
  }
}

// The sweep: a block is 32 consecutive x columns of one row and one
// component x NCH chunks (a warp is one chunk, so row loads are coalesced).
template <typename T, bool LES, int NCH, int LMAX>
__global__ void __launch_bounds__(32 * NCH, sizeof(T) == 4 ? 2 : 1) k_cn_line_chunk(Geom<T> g, Visc<T, LES> N, T h,
                                                                const T* __restrict__ ru, const T* __restrict__ rv,
                                                                const T* __restrict__ rw, const T* __restrict__ au,
                                                                const T* __restrict__ av, const T* __restrict__ aw,
                                                                T* __restrict__ ou, T* __restrict__ ov,
                                                                T* __restrict__ ow, const T* __restrict__ piv) {
  __shared__ T ZB[NCH][32], FB[NCH][32];
  const int nx = g.nx, nz = g.nz, comp = blockIdx.z, j = blockIdx.y;
  const int col = threadIdx.x & 31, c = threadIdx.x >> 5;
  const int i0 = blockIdx.x * 32 + col;
  const bool act = i0 < nx;
  const int i = act ? i0 : nx - 1;  // in-bounds stand-in for columns past the row end
  const int plane = nx * g.ny, n = comp < 2 ? nz : nz - 1, off = comp < 2 ? 0 : 1;
  const int k0 = c * n / NCH, k1 = (c + 1) * n / NCH, L = k1 - k0;
  const T* __restrict__ a = comp == 0 ? au : comp == 1 ? av : aw;
  const T* __restrict__ rr = comp == 0 ? ru : comp == 1 ? rv : rw;
  T* __restrict__ o = comp == 0 ? ou : comp == 1 ? ov : ow;
  const T* __restrict__ P = piv + (size_t)comp * (nz + 1) * plane;
  const int c0 = j * nx + i;
  T G[LMAX], F[LMAX], E[LMAX];
#pragma unroll
  for (int q = 0; q < LMAX; q++)
    if (q < L) {
      const int m = k0 + q, lev = (m + off) * plane;
      const CnRow<T> r = cn_row<T, LES>(g, N, h, comp, i, j, m, a);
      const T inv = __ldg(P + lev + c0);
      G[q] = (__ldg(rr + lev + c0) + h * r.xy) * inv;
      F[q] = -r.lo * inv;
      E[q] = -r.up * inv;
    }
  // elimination inside the chunk from zero, then the carry from below
  T z = T(0), Fp = T(1);
#pragma unroll
  for (int q = 0; q < LMAX; q++)
    if (q < L) {
      z = G[q] + F[q] * z;
      Fp *= F[q];
      G[q] = z;
    }
  ZB[c][col] = z;
  FB[c][col] = Fp;
  __syncthreads();
  T carry = T(0);
  for (int cc = 0; cc < c; cc++) carry = ZB[cc][col] + FB[cc][col] * carry;
  Fp = T(1);
#pragma unroll
  for (int q = 0; q < LMAX; q++)
    if (q < L) {
      Fp *= F[q];
      G[q] += Fp * carry;
    }
  __syncthreads();  // every carry read before the buffers take the substitution's values
  // substitution inside the chunk from zero, then the carry from above
  T w = T(0), Ep = T(1);
#pragma unroll
  for (int q = LMAX - 1; q >= 0; q--)
    if (q < L) {
      w = G[q] + E[q] * w;
      Ep *= E[q];
      G[q] = w;
    }
  ZB[c][col] = w;
  FB[c][col] = Ep;
  __syncthreads();
  carry = T(0);
  for (int cc = NCH - 1; cc > c; cc--) carry = ZB[cc][col] + FB[cc][col] * carry;
  Ep = T(1);
#pragma unroll
  for (int q = LMAX - 1; q >= 0; q--)
    if (q < L) {
      Ep *= E[q];
      G[q] += Ep * carry;
    }
  if (act) {
#pragma unroll
    for (int q = 0; q < LMAX; q++)
      if (q < L) o[(k0 + q + off) * plane + c0] = G[q];
    if (comp == 2 && c == 0) {
      o[c0] = T(0);
      o[nz * plane + c0] = T(0);
    }
  }
}

// ---------------------------------------------------------------------------
// Eq. presdiv right-hand side b = D u* / dt, with ||b||_2 reduced in FP64.
// Also clears the convergence flags of the coming solve.  The three terms
// of b nearly cancel (u* is divergence-free up to O(dt)), so plain FP32
// arithmetic here would put rounding of the size of the terms into b; the
// differences and their products with the metric are kept to FP64 accuracy
// (FP64 fields: FP64 arithmetic; FP32 fields: exact two-float differences
// and products, see below), so the sum of b over the box telescopes to
// zero to FP64 rounding and b has no mean the Poisson iteration could not
// remove (sc[SC_BMEAN] = 0).  FP32 fields sum the squares in FP32 per warp
// and FP64 across warps.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBX* kBY) k_divergence(Geom<T> g, const T* __restrict__ u, const T* __restrict__ v,
                                                          const T* __restrict__ w, double idt, double* __restrict__ b,
                                                          Red red, unsigned nblocks) {
  __shared__ double sh[32];
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  double bt = 0.0;
  if (i < g.nx && j < g.ny) {
    const int ip = i == g.nx - 1 ? 0 : i + 1, jp = j == g.ny - 1 ? 0 : j + 1;
    const int q = at(g.nx, g.ny, i, j, k);
    double d;
    if constexpr (sizeof(T) == sizeof(float)) {
      // FP32 fields: each face difference and its product with the metric
      // carried exactly as an unevaluated sum of two floats (Knuth's
      // two-sum, the fma product error), the three terms added with their
      // errors; only the final value goes through the FP64 pipe (GB300 runs
      // FP64 at 1/64 of FP32).  Accurate to about 2^-46 of the terms, as the
      // FP64 arithmetic it replaces.
      auto term = [](float a, float bb, float c, float& lo) {
        const float s = __fsub_rn(a, bb);
        const float bp = __fsub_rn(s, a), ap = __fsub_rn(s, bp);
        const float e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(-bb, bp));  // a - bb = s + e exactly
        const float hi = __fmul_rn(s, c);
        lo = __fmaf_rn(e, c, __fmaf_rn(s, c, -hi));  // s c = hi + (fma error) exactly; plus e c
        return hi;
      };
      float l1, l2, l3;
      const float t1 = term(__ldg(u + at(g.nx, g.ny, ip, j, k)), __ldg(u + q), g.idx, l1);
      const float t2 = term(__ldg(v + at(g.nx, g.ny, i, jp, k)), __ldg(v + q), g.idy, l2);
      const float t3 = term(__ldg(w + q + g.nx * g.ny), __ldg(w + q), __ldg(g.idz + k), l3);
      auto two_sum = [](float a, float bb, float& err) {
        const float s = __fadd_rn(a, bb);
        const float bp = __fsub_rn(s, a), ap = __fsub_rn(s, bp);
        err = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(bb, bp));
        return s;
      };
      float e1, e2;
      const float h1 = two_sum(t1, t2, e1);
      const float h2 = two_sum(h1, t3, e2);
      const float lo = __fadd_rn(__fadd_rn(__fadd_rn(l1, l2), __fadd_rn(l3, e1)), e2);
      d = (double)h2 + (double)lo;
    } else {
      d = (__ldg(u + at(g.nx, g.ny, ip, j, k)) - __ldg(u + q)) * g.idx +
          (__ldg(v + at(g.nx, g.ny, i, jp, k)) - __ldg(v + q)) * g.idy +
          (__ldg(w + q + g.nx * g.ny) - __ldg(w + q)) * __ldg(g.idz + k);
    }
    bt = d * idt;
    b[q] = bt;
  }
  double s;
  if constexpr (sizeof(T) == sizeof(float)) {
    const float bf = (float)bt;
    s = block_sum_f32(bf * bf, sh);
  } else {
    s = block_sum(bt * bt, sh);
  }
  if (publish_partial_tree(red, nblocks, s, 0.0, false)) {
    const double tot = final_sum(red.partial, nblocks, sh);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if (tid == 0) {
      red.sc[SC_BNORM] = sqrt(tot);
      red.sc[SC_BMEAN] = 0.0;
      red.flag[FL_DONE] = 0;
      red.flag[FL_INNER_DONE] = 0;
      *red.counter = 0u;
    }
  }
}

// ---------------------------------------------------------------------------
// Eq. project u_p_1: u = u* - dt G p with w = 0 on the walls; reduces the
// volume-weighted mean of u and max |u| (FP64).  Grid z covers 0..nz.
//   FP64 fields: FP64 arithmetic.
//   FP32 fields: the pressure differences in FP64 (p is FP64 and may carry
//     a large constant), everything else in FP32; the sums in FP32 per warp,
//     FP64 across warps.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBX* kBY) k_correct(Geom<T> g, const double* __restrict__ p, double dt,
                                                       T* __restrict__ u, T* __restrict__ v, T* __restrict__ w,
                                                       const double* __restrict__ ihz64, const double* __restrict__ dz64,
                                                       double inv_vol, Red red, unsigned nblocks) {
  __shared__ double sh[32];
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  double bs, bm;
  if constexpr (sizeof(T) == sizeof(float)) {
    float s = 0.f, m = 0.f;
    if (i < g.nx && j < g.ny) {
      const int im = i == 0 ? g.nx - 1 : i - 1, jm = j == 0 ? g.ny - 1 : j - 1;
      const int q = at(g.nx, g.ny, i, j, k);
      const float cx = (float)dt * g.idx, cy = (float)dt * g.idy;
      if (k < g.nz) {
        const double pc = __ldg(p + q);
        const float dpx = (float)(pc - __ldg(p + at(g.nx, g.ny, im, j, k)));
        const float dpy = (float)(pc - __ldg(p + at(g.nx, g.ny, i, jm, k)));
        const float ut = u[q] - cx * dpx;
        u[q] = ut;
        v[q] = v[q] - cy * dpy;
        s = ut * __ldg(g.dzv + k);
        m = fabsf(ut);
      }
      if (k == 0 || k == g.nz) {
        w[q] = 0.f;
      } else {
        const float dpz = (float)(__ldg(p + q) - __ldg(p + q - g.nx * g.ny));
        w[q] = w[q] - (float)dt * __ldg(g.ihz + k) * dpz;
      }
    }
    bs = block_sum_f32(s, sh);
    bm = block_max_f32(m, sh);
  } else {
    double s = 0.0, m = 0.0;
    if (i < g.nx && j < g.ny) {
      const int im = i == 0 ? g.nx - 1 : i - 1, jm = j == 0 ? g.ny - 1 : j - 1;
      const int q = at(g.nx, g.ny, i, j, k);
      if (k < g.nz) {
        const double pc = __ldg(p + q);
        const double un = (double)u[q] - dt * (pc - __ldg(p + at(g.nx, g.ny, im, j, k))) * (double)g.idx;
        const double vn = (double)v[q] - dt * (pc - __ldg(p + at(g.nx, g.ny, i, jm, k))) * (double)g.idy;
        const T ut = (T)un;
        u[q] = ut;
        v[q] = (T)vn;
        s = (double)ut * __ldg(dz64 + k);
        m = fabs((double)ut);
      }
      if (k == 0 || k == g.nz) {
        w[q] = T(0);
      } else {
        const double wn = (double)w[q] - dt * (__ldg(p + q) - __ldg(p + q - g.nx * g.ny)) * __ldg(ihz64 + k);
        w[q] = (T)wn;
      }
    }
    bs = block_sum(s, sh);
    bm = block_max(m, sh);
  }
  if (publish_partial_tree(red, nblocks, bs, bm, true)) {
    const double tot = final_sum(red.partial, nblocks, sh);
    const double mx = final_max(red.partial + nblocks, nblocks, sh);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if (tid == 0) {
      red.sc[SC_BULK] = tot * inv_vol;
      red.sc[SC_UMAX] = mx;
      if (!(tot == tot) || !(mx == mx) || isinf(mx)) red.flag[FL_BAD] = 1;
      *red.counter = 0u;
    }
  }
}

template <typename T>
__global__ void k_flux_shift(int n, T* __restrict__ u, double target, Red red) {
  const double shift = target - __ldcg(red.sc + SC_BULK);
  if constexpr (sizeof(T) == sizeof(float)) {
    // FP32 fields: the shift rounded once, the additions in FP32
    const float sh = (float)shift;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) u[q] += sh;
  } else {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) u[q] += shift;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) red.sc[SC_SHIFT] = shift;
}

template <typename Td, typename Ts>
__global__ void k_convert(Td* __restrict__ d, const Ts* __restrict__ s, size_t n) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
    d[q] = (Td)s[q];
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

template <typename T>
cudaError_t launch_viscosity(const Geom<T>& g, const T* u, const T* v, const T* w, T nu0, T* nu, cudaStream_t s) {
  Launch l = plane_launch(g.nx, g.ny, g.nz);
  k_viscosity<T><<<l.grid, l.block, 0, s>>>(g, u, v, w, nu0, nu);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_momentum(const Geom<T>& g, bool les, const T* u, const T* v, const T* w, const T* nu, T nu0,
                            T fx, Hist<T> H, T dt, T* ru, T* rv, T* rw, cudaStream_t s) {
  Launch l = plane_launch(g.nx, g.ny, g.nz + 1);
  if (les) {
    Visc<T, true> N{nu, nu0, g.nx, g.ny, g.nz};
    k_momentum<T, true><<<l.grid, l.block, 0, s>>>(g, u, v, w, N, fx, H, dt, ru, rv, rw);
  } else {
    Visc<T, false> N{nu, nu0, g.nx, g.ny, g.nz};
    k_momentum<T, false><<<l.grid, l.block, 0, s>>>(g, u, v, w, N, fx, H, dt, ru, rv, rw);
  }
  return cudaGetLastError();
}

__global__ void k_step_end(int* step) { *step += 1; }

__global__ void k_batch_begin(int* c, cudaGraphConditionalHandle h) {
  c[0] = 0;
  cudaGraphSetConditional(h, c[1] > 0 ? 1u : 0u);
}
__global__ void k_batch_end(int* c, cudaGraphConditionalHandle h) {
  c[0] += 1;
  cudaGraphSetConditional(h, c[0] < c[1] ? 1u : 0u);
}

cudaError_t launch_batch_begin(int* counter, cudaGraphConditionalHandle h_steps, cudaStream_t s) {
  k_batch_begin<<<1, 1, 0, s>>>(counter, h_steps);
  return cudaGetLastError();
}
cudaError_t launch_batch_end(int* counter, cudaGraphConditionalHandle h_steps, cudaStream_t s) {
  k_batch_end<<<1, 1, 0, s>>>(counter, h_steps);
  return cudaGetLastError();
}

cudaError_t launch_step_end(int* step, cudaStream_t s) {
  k_step_end<<<1, 1, 0, s>>>(step);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cn_sweep(const Geom<T>& g, bool les, const T* nu, T nu0, T hdt, const T* ru, const T* rv,
                            const T* rw, const T* au, const T* av, const T* aw, T* ou, T* ov, T* ow,
                            cudaStream_t s) {
  Launch l = plane_launch(g.nx, g.ny, g.nz + 1);
  if (les) {
    Visc<T, true> N{nu, nu0, g.nx, g.ny, g.nz};
    k_cn_sweep<T, true><<<l.grid, l.block, 0, s>>>(g, N, hdt, ru, rv, rw, au, av, aw, ou, ov, ow);
  } else {
    Visc<T, false> N{nu, nu0, g.nx, g.ny, g.nz};
    k_cn_sweep<T, false><<<l.grid, l.block, 0, s>>>(g, N, hdt, ru, rv, rw, au, av, aw, ou, ov, ow);
  }
  return cudaGetLastError();
}

// chunks of the z-line Crank-Nicolson sweep and rows a chunk holds at most:
// columns of up to 16 x 12 = 192 rows
constexpr int kCnChunks = 16, kCnChunkRows = 12;

bool cn_chunk_ok(int nz) { return nz >= 2 && nz <= kCnChunks * kCnChunkRows; }

template <typename T>
cudaError_t launch_cn_pivots(const Geom<T>& g, bool les, const T* nu, T nu0, T hdt, T* piv, cudaStream_t s) {
  const dim3 block(128), grid((g.nx + 127) / 128, g.ny, 3);
  if (les) {
    Visc<T, true> N{nu, nu0, g.nx, g.ny, g.nz};
    k_cn_pivots<T, true><<<grid, block, 0, s>>>(g, N, hdt, piv);
  } else {
    Visc<T, false> N{nu, nu0, g.nx, g.ny, g.nz};
    k_cn_pivots<T, false><<<grid, block, 0, s>>>(g, N, hdt, piv);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cn_line(const Geom<T>& g, bool les, const T* nu, T nu0, T hdt, const T* ru, const T* rv,
                           const T* rw, const T* au, const T* av, const T* aw, T* ou, T* ov, T* ow, void* scratch,
                           const T* piv, cudaStream_t s) {
  if (piv && cn_chunk_ok(g.nz)) {
    const dim3 block(32 * kCnChunks), grid((g.nx + 31) / 32, g.ny, 3);
    if (les) {
      Visc<T, true> N{nu, nu0, g.nx, g.ny, g.nz};
      k_cn_line_chunk<T, true, kCnChunks, kCnChunkRows><<<grid, block, 0, s>>>(g, N, hdt, ru, rv, rw, au, av, aw,
                                                                                ou, ov, ow, piv);
    } else {
      Visc<T, false> N{nu, nu0, g.nx, g.ny, g.nz};
      k_cn_line_chunk<T, false, kCnChunks, kCnChunkRows><<<grid, block, 0, s>>>(g, N, hdt, ru, rv, rw, au, av, aw,
                                                                                 ou, ov, ow, piv);
    }
    return cudaGetLastError();
  }
  const dim3 block(128), grid((g.nx + 127) / 128, g.ny, 3);
  using V2 = typename Pair<T>::V;
  if (les) {
    Visc<T, true> N{nu, nu0, g.nx, g.ny, g.nz};
    k_cn_line<T, true><<<grid, block, 0, s>>>(g, N, hdt, ru, rv, rw, au, av, aw, ou, ov, ow, (V2*)scratch);
  } else {
    Visc<T, false> N{nu, nu0, g.nx, g.ny, g.nz};
    k_cn_line<T, false><<<grid, block, 0, s>>>(g, N, hdt, ru, rv, rw, au, av, aw, ou, ov, ow, (V2*)scratch);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_explicit_only(const Geom<T>& g, bool les, const T* u, const T* v, const T* w, const T* nu,
                                 T nu0, T fx, T* Nu, T* Nv, T* Nw, cudaStream_t s) {
  Launch l = plane_launch(g.nx, g.ny, g.nz + 1);
  if (les) {
    Visc<T, true> N{nu, nu0, g.nx, g.ny, g.nz};
    k_explicit<T, true><<<l.grid, l.block, 0, s>>>(g, u, v, w, N, fx, Nu, Nv, Nw);
  } else {
    Visc<T, false> N{nu, nu0, g.nx, g.ny, g.nz};
    k_explicit<T, false><<<l.grid, l.block, 0, s>>>(g, u, v, w, N, fx, Nu, Nv, Nw);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_diffusion_only(const Geom<T>& g, bool les, const T* u, const T* v, const T* w, const T* nu,
                                  T nu0, T* Du, T* Dv, T* Dw, cudaStream_t s) {
  Launch l = plane_launch(g.nx, g.ny, g.nz + 1);
  if (les) {
    Visc<T, true> N{nu, nu0, g.nx, g.ny, g.nz};
    k_diffusion<T, true><<<l.grid, l.block, 0, s>>>(g, u, v, w, N, Du, Dv, Dw);
  } else {
    Visc<T, false> N{nu, nu0, g.nx, g.ny, g.nz};
    k_diffusion<T, false><<<l.grid, l.block, 0, s>>>(g, u, v, w, N, Du, Dv, Dw);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_divergence_rhs(const Geom<T>& g, const T* u, const T* v, const T* w, double idt, double* b,
                                  Red red, double Lz, cudaStream_t s) {
  Launch l = plane_launch(g.nx, g.ny, g.nz);
  (void)Lz;
  k_divergence<T><<<l.grid, l.block, 0, s>>>(g, u, v, w, idt, b, red, l.nblocks);
  return cudaGetLastError();
}

// ihz64 / dz64 are FP64 copies of the metrics; they sit at fixed offsets of
// the FP64 metric pack, passed in by the caller through Geom<double> below.
template <typename T>
cudaError_t launch_correct_impl(const Geom<T>& g, const double* p, double dt, T* u, T* v, T* w,
                                const double* ihz64, const double* dz64, double inv_vol, Red red, cudaStream_t s) {
  Launch l = plane_launch(g.nx, g.ny, g.nz + 1);
  k_correct<T><<<l.grid, l.block, 0, s>>>(g, p, dt, u, v, w, ihz64, dz64, inv_vol, red, l.nblocks);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_flux_shift(const Geom<T>& g, T* u, double target, Red red, cudaStream_t s) {
  const int n = g.nx * g.ny * g.nz;
  int blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_flux_shift<T><<<blocks, 256, 0, s>>>(n, u, target, red);
  return cudaGetLastError();
}

template <typename Td, typename Ts>
cudaError_t launch_convert(Td* dst, const Ts* src, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_convert<Td, Ts><<<(unsigned)blocks, 256, 0, s>>>(dst, src, n);
  return cudaGetLastError();
}

#define STP_INST(T)                                                                                                 \
  template cudaError_t launch_viscosity<T>(const Geom<T>&, const T*, const T*, const T*, T, T*, cudaStream_t);      \
  template cudaError_t launch_momentum<T>(const Geom<T>&, bool, const T*, const T*, const T*, const T*, T, T,     \
                                          Hist<T>, T, T*, T*, T*, cudaStream_t);                                    \
  template cudaError_t launch_cn_sweep<T>(const Geom<T>&, bool, const T*, T, T, const T*, const T*, const T*,      \
                                          const T*, const T*, const T*, T*, T*, T*, cudaStream_t);                  \
  template cudaError_t launch_cn_line<T>(const Geom<T>&, bool, const T*, T, T, const T*, const T*, const T*,       \
                                         const T*, const T*, const T*, T*, T*, T*, void*, const T*, cudaStream_t);  \
  template cudaError_t launch_cn_pivots<T>(const Geom<T>&, bool, const T*, T, T, T*, cudaStream_t);               \
  template cudaError_t launch_explicit_only<T>(const Geom<T>&, bool, const T*, const T*, const T*, const T*, T, T, \
                                               T*, T*, T*, cudaStream_t);                                           \
  template cudaError_t launch_diffusion_only<T>(const Geom<T>&, bool, const T*, const T*, const T*, const T*, T,   \
                                                T*, T*, T*, cudaStream_t);                                          \
  template cudaError_t launch_divergence_rhs<T>(const Geom<T>&, const T*, const T*, const T*, double, double*, Red,\
                                                double, cudaStream_t);                                              \
  template cudaError_t launch_correct_impl<T>(const Geom<T>&, const double*, double, T*, T*, T*, const double*,    \
                                              const double*, double, Red, cudaStream_t);                            \
  template cudaError_t launch_flux_shift<T>(const Geom<T>&, T*, double, Red, cudaStream_t);

STP_INST(double)
STP_INST(float)

template cudaError_t launch_convert<double, float>(double*, const float*, size_t, cudaStream_t);
template cudaError_t launch_convert<float, double>(float*, const double*, size_t, cudaStream_t);
template cudaError_t launch_convert<double, double>(double*, const double*, size_t, cudaStream_t);

}  // namespace stp
