// Device side of the matrix-element library: HELAS-style external wavefunctions,
// FFV / VVV / VVVV vertex currents with propagators, root-vertex amplitudes, the
// colour-matrix quadratic form, the helicity sum and helicity / colour selection.
//
// One thread evaluates one event: it walks the process's op table (emitted by the
// process compiler) and computes every off-shell current once per helicity state
// of its own external legs ("variants"), keeping the variants in a per-event
// workspace laid out [offset][thread] so that a warp's accesses are coalesced.
// Every diagram term is closed at the root vertex through a root bilinear; terms with
// the same colour vector up to a phase form a group, terms of a group sharing a
// bilinear are summed first (a "sum current" over the same legs, once per helicity
// state of those legs) and closed with one product per good helicity, and each group
// amplitude is added to its colour flows (jamps).  The colour sum J^dagger C J, the
// helicity sum and the selections follow in the same thread.
// The arithmetic is templated on its real type R: double or float.
//
// Feynman rules (all momenta incoming at a vertex; metric +---; chiral gamma basis):
//   f f V : gamma^mu (cL P_L + cR P_R)      qqg: cL = cR = i g_s; photon -i e Q; Z -i gL, -i gR
//   g g g : g_s [g^mn (k1-k2)^r + g^nr (k2-k3)^m + g^rm (k3-k1)^n]  (colour f^abc)
//   gggg  : -i g_s^2 G_j, j = 0..2 one per colour structure
//   fermion propagator i (kslash + m)/(k^2 - m^2 + i m w); vector -i (g - k k/M^2)/(k^2 - M^2 + i M w)
#pragma once
#include <cstdint>

#include "real.cuh"

namespace mgx {

enum { OP_EXT = 1, OP_FFV_F = 2, OP_FFV_FB = 3, OP_FFV_V = 4, OP_VVV = 5, OP_VVVV = 6, OP_AMP = 7, OP_BIL = 8, OP_RBIL = 9,
       OP_SUM = 10 };
enum { EXT_U = 0, EXT_V = 1, EXT_UBAR = 2, EXT_VBAR = 3, EXT_EPS_IN = 4, EXT_EPS_OUT = 5 };
enum { CPL_GS = 1, CPL_CHIRAL = 2 };

constexpr int MAXCPL = 8;
constexpr int MAXMASS = 4;
constexpr int MAXHEL = 128;
constexpr int MAXNPAR = 8;

struct KParams {
  const int4* ops;       // 4 int4 (16 int32 fields) per op
  const int2* flows;     // (colour flow, phase code 0..3 for 1, i, -1, -i; | 4 on a flow's first update)
  const int4* terms;     // 2 int4 per diagram term: (bilinear base, mask, other base, mask), (phase, kind, -, -)
  const double* colsym;  // ncol*ncol: C_ii on the diagonal, 2 C_ij above it
  const float* colsym_f;
  int nops, ncol, npar, nin, ngood;
  int cur_doubles, jamp_off, mh_off, colw_off, ws_doubles;
  double avg;            // 1 / (4 Ncol_in S)
  int gs_power;          // |M|^2 carries (4 pi alpha_s)^gs_power; vertices use g_s = 1
  int jamp_zero;         // jamps need zeroing (a flow no group updates); else first updates write
  double cpl[MAXCPL][4]; // cL.re cL.im cR.re cR.im
  int cplflags[MAXCPL];
  double mass[MAXMASS], width[MAXMASS];
  int massive[MAXMASS];  // mass[i] > 0, tested without a float64 compare
  int good[MAXHEL];      // canonical indices of the good helicities
  signed char hidx[MAXHEL];  // rank of canonical helicity h among the good ones, -1 if not good
};

template <class R>
struct cxT {
  R r, i;
};
using cx = cxT<double>;

template <class R> __device__ __forceinline__ cxT<R> operator+(cxT<R> a, cxT<R> b) { return {a.r + b.r, a.i + b.i}; }
template <class R> __device__ __forceinline__ cxT<R> operator-(cxT<R> a, cxT<R> b) { return {a.r - b.r, a.i - b.i}; }
template <class R> __device__ __forceinline__ cxT<R> cneg(cxT<R> a) { return {-a.r, -a.i}; }
template <class R> __device__ __forceinline__ cxT<R> cmul(cxT<R> a, cxT<R> b) {
  return {fma(a.r, b.r, -(a.i * b.i)), fma(a.r, b.i, a.i * b.r)};
}
// acc + a*b
template <class R> __device__ __forceinline__ cxT<R> cfma(cxT<R> a, cxT<R> b, cxT<R> acc) {
  return {fma(a.r, b.r, fma(-a.i, b.i, acc.r)), fma(a.r, b.i, fma(a.i, b.r, acc.i))};
}
template <class R> __device__ __forceinline__ cxT<R> rmul(R s, cxT<R> a) { return {s * a.r, s * a.i}; }
template <class R> __device__ __forceinline__ cxT<R> rfma(R s, cxT<R> a, cxT<R> acc) {
  return {fma(s, a.r, acc.r), fma(s, a.i, acc.i)};
}
template <class R> __device__ __forceinline__ cxT<R> conjx(cxT<R> a) { return {a.r, -a.i}; }
// Minkowski dot of complex 4-vectors (upper components)
template <class R> __device__ __forceinline__ cxT<R> mdot(const cxT<R>* a, const cxT<R>* b) {
  cxT<R> s = cmul(a[0], b[0]);
  s = cfma(cneg(a[1]), b[1], s);
  s = cfma(cneg(a[2]), b[2], s);
  s = cfma(cneg(a[3]), b[3], s);
  return s;
}
// Minkowski dot of a real and a complex 4-vector
template <class R> __device__ __forceinline__ cxT<R> rdot(const R* k, const cxT<R>* a) {
  cxT<R> s = rmul(k[0], a[0]);
  s = rfma(-k[1], a[1], s);
  s = rfma(-k[2], a[2], s);
  s = rfma(-k[3], a[3], s);
  return s;
}

// ---- bit helpers: variants of a current are indexed by the helicity bits of its legs
__device__ __forceinline__ int pext(int x, int mask) {
  int r = 0, k = 0;
  while (mask) {
    const int low = mask & -mask;
    if (x & low) r |= 1 << k;
    ++k;
    mask ^= low;
  }
  return r;
}
__device__ __forceinline__ int pdep(int v, int mask) {
  int r = 0, k = 0;
  while (mask) {
    const int low = mask & -mask;
    if ((v >> k) & 1) r |= low;
    ++k;
    mask ^= low;
  }
  return r;
}

// Per-event workspace view: element `off` of this thread is base[off * stride], one R per
// element (8 bytes for double, 4 for float), so a warp's accesses coalesce.
template <class R>
struct WST {
  R* base;
  int64_t stride;
  __device__ __forceinline__ R& operator[](int off) const { return base[(int64_t)off * stride]; }
  __device__ __forceinline__ void load4(int off, cxT<R>* w) const {
#pragma unroll
    for (int j = 0; j < 4; ++j) w[j] = cxT<R>{(*this)[off + 2 * j], (*this)[off + 2 * j + 1]};
  }
  __device__ __forceinline__ void store4(int off, const cxT<R>* w) const {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      (*this)[off + 2 * j] = w[j].r;
      (*this)[off + 2 * j + 1] = w[j].i;
    }
  }
  __device__ __forceinline__ void loadk(int off, R* k) const {
#pragma unroll
    for (int j = 0; j < 4; ++j) k[j] = (*this)[off + j];
  }
  __device__ __forceinline__ void storek(int off, const R* k) const {
#pragma unroll
    for (int j = 0; j < 4; ++j) (*this)[off + j] = k[j];
  }
};
using WS = WST<double>;

// ---- external wavefunctions (HELAS conventions, helicity eigenstates in the given frame)
// two-component helicity spinors chi_lam(p)
template <class R>
__device__ inline void chi(const R* p, R pp, int lam, cxT<R>* c) {
  using T = Real<R>;
  const R zero = T::from(0.0), one = T::from(1.0);
  const R a = pp + p[3];
  if (T::positive(a)) {
    const R n = T::rcp(T::sqrt_(T::from(2.0) * pp * a));
    if (lam > 0) {
      c[0] = {a * n, zero};
      c[1] = {p[1] * n, p[2] * n};
    } else {
      c[0] = {-(p[1] * n), p[2] * n};
      c[1] = {a * n, zero};
    }
  } else if (T::positive(pp)) {  // along -z
    if (lam > 0) { c[0] = {zero, zero}; c[1] = {one, zero}; }
    else { c[0] = {-one, zero}; c[1] = {zero, zero}; }
  } else {                       // at rest: quantise along +z
    if (lam > 0) { c[0] = {one, zero}; c[1] = {zero, zero}; }
    else { c[0] = {zero, zero}; c[1] = {one, zero}; }
  }
}

template <class R>
__device__ __forceinline__ R norm3(const R* p) {
  return Real<R>::sqrt_(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
}

// u(p, lam): (sqrt(E - lam|p|) chi_lam, sqrt(E + lam|p|) chi_lam); massless: exact chirality
template <class R>
__device__ inline void ext_u(const R* p, double m, int lam, cxT<R>* w) {
  using T = Real<R>;
  const R pp = norm3(p);
  cxT<R> c[2];
  chi(p, pp, lam, c);
  R wu, wl;
  if (m == 0.0) {
    const R s = T::sqrt_(T::from(2.0) * p[0]);
    wu = lam < 0 ? s : T::from(0.0);
    wl = lam < 0 ? T::from(0.0) : s;
  } else {
    const R lp = lam > 0 ? pp : -pp;
    wu = T::sqrt_(T::max0(p[0] - lp));
    wl = T::sqrt_(T::max0(p[0] + lp));
  }
  w[0] = rmul(wu, c[0]); w[1] = rmul(wu, c[1]);
  w[2] = rmul(wl, c[0]); w[3] = rmul(wl, c[1]);
}

// v(p, lam): (sqrt(E + lam|p|) chi_-lam, -sqrt(E - lam|p|) chi_-lam)
template <class R>
__device__ inline void ext_v(const R* p, double m, int lam, cxT<R>* w) {
  using T = Real<R>;
  const R pp = norm3(p);
  cxT<R> c[2];
  chi(p, pp, -lam, c);
  R wu, wl;
  if (m == 0.0) {
    const R s = T::sqrt_(T::from(2.0) * p[0]);
    wu = lam > 0 ? s : T::from(0.0);
    wl = lam > 0 ? T::from(0.0) : -s;
  } else {
    const R lp = lam > 0 ? pp : -pp;
    wu = T::sqrt_(T::max0(p[0] + lp));
    wl = -T::sqrt_(T::max0(p[0] - lp));
  }
  w[0] = rmul(wu, c[0]); w[1] = rmul(wu, c[1]);
  w[2] = rmul(wl, c[0]); w[3] = rmul(wl, c[1]);
}

// psi-bar = psi^dagger gamma^0: swap halves and conjugate
template <class R>
__device__ __forceinline__ void to_bar(cxT<R>* w) {
  const cxT<R> a = w[0], b = w[1];
  w[0] = conjx(w[2]); w[1] = conjx(w[3]);
  w[2] = conjx(a); w[3] = conjx(b);
}

// eps^mu(k, lam) = (-lam e1 - i e2)/sqrt2 (upper index); outgoing: complex conjugate
template <class R>
__device__ inline void ext_eps(const R* k, int lam, bool outgoing, cxT<R>* w) {
  using T = Real<R>;
  const R zero = T::from(0.0);
  const R kk = norm3(k);
  const R pt = T::sqrt_(k[1] * k[1] + k[2] * k[2]);
  R cth = T::from(1.0), sth = zero, cph = T::from(1.0), sph = zero;
  if (T::positive(kk)) { const R ik = T::rcp(kk); cth = k[3] * ik; sth = pt * ik; }
  if (T::positive(pt)) { const R ip = T::rcp(pt); cph = k[1] * ip; sph = k[2] * ip; }
  const R r = T::from(0.70710678118654752440);
  const R l = T::from(lam > 0 ? 1.0 : -1.0);
  const R rs = outgoing ? -r : r;
  w[0] = {zero, zero};
  w[1] = {-(l * cth * cph * r), sph * rs};
  w[2] = {-(l * cth * sph * r), -(cph * rs)};
  w[3] = {l * sth * r, zero};
}

// ---- vertex building blocks
// A = V^0 - V.sigma, B = V^0 + V.sigma for a complex 4-vector V (upper components)
template <class R>
struct SlashT {
  cxT<R> a00, a01, a10, a11;  // A
  cxT<R> b00, b01, b10, b11;  // B
};
template <class R>
__device__ __forceinline__ SlashT<R> slash(const cxT<R>* V) {
  SlashT<R> s;
  s.a00 = V[0] - V[3];
  s.a11 = V[0] + V[3];
  s.b00 = s.a11;
  s.b11 = s.a00;
  const cxT<R> v12m = {V[1].r + V[2].i, V[1].i - V[2].r};  // V1 - i V2
  const cxT<R> v12p = {V[1].r - V[2].i, V[1].i + V[2].r};  // V1 + i V2
  s.a01 = cneg(v12m);
  s.a10 = cneg(v12p);
  s.b01 = v12m;
  s.b10 = v12p;
  return s;
}

// complex 1/(re + i im)
template <class R>
__device__ __forceinline__ cxT<R> cinv(R re, R im) {
  const R d = Real<R>::rcp(fma(re, re, im * im));
  return {re * d, -(im * d)};
}
template <class R>
__device__ __forceinline__ R msq(const R* k) {
  return fma(k[0], k[0], -fma(k[1], k[1], fma(k[2], k[2], k[3] * k[3])));
}

}  // namespace mgx
