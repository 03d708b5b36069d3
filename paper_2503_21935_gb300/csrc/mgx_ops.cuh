// Op executors of the amplitude program (conventions in mgx_kernel.cuh), templated on the
// real type R and on the storage view S (per-thread global workspace or shared memory).
//
// Every current op is split into a header, computed once per event (incoming
// momentum, propagator prefactor and derived momenta), and one variant per
// helicity state of its legs.  A current's storage block is
//   [header (H(kind) slots) | variant 0 (4 complex) | variant 1 | ...]
// The op table carries the child block offsets (momenta at +0) and the child
// variant bases (fields 13-15), so no op needs to know its children's kinds.
// Sum currents (OP_SUM) have no header; their summand list lives in the term table.
#pragma once
#include <type_traits>

#include "mgx_kernel.cuh"

namespace mgx {

struct Op {
  int code, dst, a, b, c, mdst, ma, mb, mc, cpl, mass, aux, aux2, va, vb, vc;
};

__device__ __forceinline__ Op load_op(const int4* ops, int i) {
  const int4 x = __ldg(ops + 4 * i), y = __ldg(ops + 4 * i + 1), z = __ldg(ops + 4 * i + 2),
             w = __ldg(ops + 4 * i + 3);
  return Op{x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w, z.x, z.y, z.z, z.w, w.x, w.y, w.z, w.w};
}

// Which helicity variants a thread computes.  AllHel: every variant of every current (one thread
// per event).  GroupHel: the helicity-parallel mapping, in which the 2^|fix| threads of one event
// each take the helicities whose bits on the fixed legs (mask fix, in the helicity-index bit
// positions) equal `bits`: a thread computes only the variants of each current that such a
// helicity uses, and only those helicities' amplitudes.  Variants keep their full-size slots.
struct AllHel {
  __device__ __forceinline__ int count(int m) const { return 1 << __popc(m); }   // variants of leg mask m
  __device__ __forceinline__ int var(int u, int) const { return u; }             // u-th of them
  __device__ __forceinline__ bool ok(int) const { return true; }                 // helicity h taken
};
struct GroupHel {
  int fix, bits;
  __device__ __forceinline__ int count(int m) const { return 1 << __popc(m & ~fix); }
  __device__ __forceinline__ int var(int u, int m) const;
  __device__ __forceinline__ bool ok(int h) const { return (h & fix) == bits; }
};

// Shared-memory storage view (contiguous 8-byte slots).
template <class R>
struct SST {
  R* base;
  __device__ __forceinline__ R& operator[](int off) const { return base[off]; }
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
using SS = SST<double>;

// coupling (cL, cR) of an op, g_s applied when flagged
template <class R>
__device__ __forceinline__ void coupling(const KParams& P, int ci, double gs, cxT<R>& cl, cxT<R>& cr,
                                         bool& chiral) {
  using T = Real<R>;
  const double s = (P.cplflags[ci] & CPL_GS) ? gs : 1.0;
  cl = {T::from(s * P.cpl[ci][0]), T::from(s * P.cpl[ci][1])};
  cr = {T::from(s * P.cpl[ci][2]), T::from(s * P.cpl[ci][3])};
  chiral = (P.cplflags[ci] & CPL_CHIRAL) != 0;
}

// out = pref * x for the prefactor of a root bilinear: exactly i (QCD vertex) and pure
// imaginary prefactors skip the complex multiply (an exact +0.0 real part is tested by bits)
template <class R>
__device__ __forceinline__ void apply_pref(cxT<R> pref, const cxT<R>* x, cxT<R>* out) {
  using T = Real<R>;
  if (T::is_zero(pref.r) && T::is_one(pref.i)) {
#pragma unroll
    for (int j = 0; j < 4; ++j) out[j] = {T::neg(x[j].i), x[j].r};
  } else if (T::is_zero(pref.r)) {
#pragma unroll
    for (int j = 0; j < 4; ++j) out[j] = {-(pref.i * x[j].i), pref.i * x[j].r};
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) out[j] = cmul(pref, x[j]);
  }
}

// phase(code) * a, code 0..3 for 1, i, -1, -i: a swap of the parts and sign flips done on the
// sign bits (integer operations, no floating-point arithmetic)
__device__ __forceinline__ double neg_if(double x, bool c) {
  return __longlong_as_double(__double_as_longlong(x) ^ ((long long)c << 63));
}
__device__ __forceinline__ float neg_if(float x, bool c) {
  return __int_as_float(__float_as_int(x) ^ ((int)c << 31));
}
template <class R>
__device__ __forceinline__ cxT<R> rot_phase(int code, cxT<R> a) {
  const bool swap = code & 1;
  const R r = swap ? a.i : a.r, i = swap ? a.r : a.i;
  return {neg_if(r, code == 1 || code == 2), neg_if(i, code >= 2)};
}

// The slash blocks of a vector current variant V (A = V^0 - V.sigma, B = V^0 + V.sigma) are four
// complex numbers: a00 = V0 - V3, a11 = V0 + V3, m = V1 - i V2, p = V1 + i V2 (A = [[a00, -m], [-p, a11]],
// B = [[a11, m], [p, a00]]).  Fermion-vector vertices keep them per V variant in their header; a
// fermion current stores them times its propagator prefactor (a scalar, so it commutes with every
// factor of the current), which is then paid once per vector variant instead of once per variant.
template <class R, class S>
__device__ __forceinline__ void store_slash(const S& W, int off, const cxT<R>* V) {
  const cxT<R> sl[4] = {V[0] - V[3], V[0] + V[3], cxT<R>{V[1].r + V[2].i, V[1].i - V[2].r},
                        cxT<R>{V[1].r - V[2].i, V[1].i + V[2].r}};
  W.store4(off, sl);
}
template <class R, class S>
__device__ __forceinline__ void store_slash(const S& W, int off, const cxT<R>* V, cxT<R> pref) {
  const cxT<R> sl[4] = {cmul(pref, V[0] - V[3]), cmul(pref, V[0] + V[3]),
                        cmul(pref, cxT<R>{V[1].r + V[2].i, V[1].i - V[2].r}),
                        cmul(pref, cxT<R>{V[1].r - V[2].i, V[1].i + V[2].r})};
  W.store4(off, sl);
}
template <class R, class S>
__device__ __forceinline__ SlashT<R> load_slash(const S& W, int off) {
  cxT<R> sl[4];
  W.load4(off, sl);
  SlashT<R> s;
  s.a00 = sl[0]; s.a11 = sl[1]; s.b00 = sl[1]; s.b11 = sl[0];
  s.a01 = cneg(sl[2]); s.a10 = cneg(sl[3]); s.b01 = sl[2]; s.b10 = sl[3];
  return s;
}
// slash blocks of every (taken) variant of child b (the vector) into the header from offset 6
template <class R, class S, class H>
__device__ __forceinline__ void header_slashes(const Op& o, const S& W, const H& hs) {
  const int nv = hs.count(o.mb);
  for (int u = 0; u < nv; ++u) {
    const int i = hs.var(u, o.mb);
    cxT<R> V[4];
    W.load4(o.vb + 8 * i, V);
    store_slash<R>(W, o.dst + 6 + 8 * i, V);
  }
}
template <class R, class S, class H>
__device__ __forceinline__ void header_slashes(const Op& o, const S& W, cxT<R> pref, const H& hs) {
  const int nv = hs.count(o.mb);
  for (int u = 0; u < nv; ++u) {
    const int i = hs.var(u, o.mb);
    cxT<R> V[4];
    W.load4(o.vb + 8 * i, V);
    store_slash<R>(W, o.dst + 6 + 8 * i, V, pref);
  }
}

__device__ __forceinline__ int GroupHel::var(int u, int m) const { return pext(pdep(u, m & ~fix) | (bits & m), m); }

// VVVV colour structure j needs the dot products of two child pairs (children 0, 1, 2 = e1, e2, e3):
// j = 0: (e1.e3, e2.e3), j = 1: (e1.e2, e2.e3), j = 2: (e1.e2, e1.e3)
__device__ __forceinline__ void vvvv_pairs(int j, int& x0, int& y0, int& x1, int& y1) {
  x0 = 0;
  y0 = j == 0 ? 2 : 1;
  x1 = j == 2 ? 0 : 1;
  y1 = 2;
}
// child k of an op: variant base and helicity mask
__device__ __forceinline__ int child_base(const Op& o, int k) { return k == 0 ? o.va : (k == 1 ? o.vb : o.vc); }
__device__ __forceinline__ int child_mask(const Op& o, int k) { return k == 0 ? o.ma : (k == 1 ? o.mb : o.mc); }
__device__ __forceinline__ int nvar_of(int mask) { return 1 << __popc(mask); }

// ================================================================ headers
template <class R, class S, class H = AllHel>
__device__ inline void op_header(const KParams& P, const Op& o, double gs, const double* pe, const S& W,
                                 const H& hs = H()) {
  using T = Real<R>;
  if (o.code == OP_SUM) return;   // no header
  if (o.code == OP_EXT) {
    const double* p = pe + 4 * o.aux;
    const double sgn = o.aux < P.nin ? 1.0 : -1.0;  // incoming momentum
    R k[4] = {T::from(sgn * p[0]), T::from(sgn * p[1]), T::from(sgn * p[2]), T::from(sgn * p[3])};
    W.storek(o.dst, k);
    return;
  }
  if (o.code == OP_BIL || o.code == OP_RBIL) {
    // root bilinears: no propagator; a non-chiral coupling is the prefactor
    cxT<R> cl, cr;
    bool chiral;
    coupling<R>(P, o.cpl, gs, cl, cr, chiral);
    W[o.dst + 4] = chiral ? T::from(1.0) : cl.r;
    W[o.dst + 5] = chiral ? T::from(0.0) : cl.i;
    if (o.code == OP_RBIL) header_slashes<R>(o, W, hs);
    return;
  }
  R ka[4], kb[4], k[4];
  W.loadk(o.a, ka);
  W.loadk(o.b, kb);
#pragma unroll
  for (int j = 0; j < 4; ++j) k[j] = ka[j] + kb[j];
  if (o.code == OP_VVVV) {
    R kc[4];
    W.loadk(o.c, kc);
#pragma unroll
    for (int j = 0; j < 4; ++j) k[j] = k[j] + kc[j];
    W.storek(o.dst, k);
    const R sv = -(T::from(gs * gs) * T::rcp(msq(k)));   // (-i)(-i g_s^2)/P^2
    W[o.dst + 4] = sv;
    // the structure's two pair tables: s (e_x0 . e_y0) and -s (e_x1 . e_y1) for every pair of variants
    int x0, y0, x1, y1;
    vvvv_pairs(o.aux, x0, y0, x1, y1);
    int base = o.dst + 6;
#pragma unroll 1
    for (int tab = 0; tab < 2; ++tab) {
      const int x = tab ? x1 : x0, y = tab ? y1 : y0;
      const int mx = child_mask(o, x), my = child_mask(o, y);
      const int nx = nvar_of(mx), ny = nvar_of(my);
      const R f = tab ? -sv : sv;
      for (int uy = 0; uy < hs.count(my); ++uy) {
        const int iy = hs.var(uy, my);
        cxT<R> ey[4];
        W.load4(child_base(o, y) + 8 * iy, ey);
        for (int ux = 0; ux < hs.count(mx); ++ux) {
          const int ix = hs.var(ux, mx);
          cxT<R> ex[4];
          W.load4(child_base(o, x) + 8 * ix, ex);
          const cxT<R> d = rmul(f, mdot(ex, ey));
          W[base + 2 * (ix + nx * iy)] = d.r;
          W[base + 2 * (ix + nx * iy) + 1] = d.i;
        }
      }
      base += 2 * nx * ny;
    }
    return;
  }
  W.storek(o.dst, k);
  if (o.code == OP_VVV) {
    // prefactor -i g_s/P^2 = i s, s folded into the momentum combinations of the vertex
    const R s = -(T::from(gs) * T::rcp(msq(k)));
    const R two = T::from(2.0);
    R q1[4], q2[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      W[o.dst + 6 + j] = s * (ka[j] - kb[j]);            // s (k1 - k2)
      q1[j] = s * fma(two, kb[j], ka[j]);                // s (k2 - k3) = s (k1 + 2 k2)
      q2[j] = -(s * fma(two, ka[j], kb[j]));             // s (k3 - k1) = -s (2 k1 + k2)
    }
    W.storek(o.dst + 10, q1);
    W.storek(o.dst + 14, q2);
    // per child variant: a1 = q1 . e1 and a2 = q2 . e2 (each depends on one child only)
    const int n1 = nvar_of(o.ma);
    for (int u1 = 0; u1 < hs.count(o.ma); ++u1) {
      const int v1 = hs.var(u1, o.ma);
      cxT<R> e[4];
      W.load4(o.va + 8 * v1, e);
      const cxT<R> a = rdot(q1, e);
      W[o.dst + 18 + 2 * v1] = a.r;
      W[o.dst + 18 + 2 * v1 + 1] = a.i;
    }
    for (int u2 = 0; u2 < hs.count(o.mb); ++u2) {
      const int v2 = hs.var(u2, o.mb);
      cxT<R> e[4];
      W.load4(o.vb + 8 * v2, e);
      const cxT<R> a = rdot(q2, e);
      W[o.dst + 18 + 2 * (n1 + v2)] = a.r;
      W[o.dst + 18 + 2 * (n1 + v2) + 1] = a.i;
    }
    return;
  }
  // f f V currents: fermion propagator i/(k^2 - m^2 + i m w) (row current uses -k, same k^2),
  // vector propagator -i/(k^2 - M^2 + i M w); non-chiral couplings folded in
  const double m = P.mass[o.mass], w = P.width[o.mass];
  const cxT<R> inv = cinv(msq(k) - T::from(m * m), T::from(m * w));
  cxT<R> pref = o.code == OP_FFV_V ? cxT<R>{inv.i, -inv.r} : cxT<R>{-inv.i, inv.r};
  cxT<R> cl, cr;
  bool chiral;
  coupling<R>(P, o.cpl, gs, cl, cr, chiral);
  if (!chiral) pref = cmul(pref, cl);
  if (o.code == OP_FFV_V) {
    W[o.dst + 4] = pref.r;
    W[o.dst + 5] = pref.i;
  } else {
    header_slashes<R>(o, W, pref, hs);
  }
}

// ================================================================ variants
template <class R, class S>
__device__ inline void var_ext(const KParams& P, const Op& o, int v, const double* pe, const S& W) {
  using T = Real<R>;
  const double* pd = pe + 4 * o.aux;
  const R p[4] = {T::from(pd[0]), T::from(pd[1]), T::from(pd[2]), T::from(pd[3])};
  const double m = P.mass[o.mass];
  const int lam = v ? 1 : -1;
  cxT<R> w[4];
  switch (o.aux2) {
    case EXT_U: ext_u(p, m, lam, w); break;
    case EXT_V: ext_v(p, m, lam, w); break;
    case EXT_UBAR: ext_u(p, m, lam, w); to_bar(w); break;
    case EXT_VBAR: ext_v(p, m, lam, w); to_bar(w); break;
    case EXT_EPS_IN: ext_eps(p, lam, false, w); break;
    default: ext_eps(p, lam, true, w); break;
  }
  W.store4(o.dst + 4 + 8 * v, w);
}

// Per-op values of the f f V fermion currents, loaded once for all variants of the op
template <class R>
struct FfvCtx {
  R k1, k2;       // the current's momentum as the propagator numerator sees it (-k for a row current)
  R a00, a11;     // k0 - k3, k0 + k3
  R m;
  bool massive, chiral;
  int out;        // workspace offset of variant 0
};
template <class R, class S>
__device__ __forceinline__ FfvCtx<R> ffv_ctx(const KParams& P, const Op& o, const S& W, bool row) {
  FfvCtx<R> c;
  R k[4];
  W.loadk(o.dst, k);
  if (row) {
#pragma unroll
    for (int j = 0; j < 4; ++j) k[j] = -k[j];
  }
  c.k1 = k[1];
  c.k2 = k[2];
  c.a00 = k[0] - k[3];
  c.a11 = k[0] + k[3];
  c.massive = P.massive[o.mass] != 0;
  c.m = Real<R>::from(P.mass[o.mass]);
  c.chiral = (P.cplflags[o.cpl] & CPL_CHIRAL) != 0;
  c.out = o.dst + 6 + 8 * nvar_of(o.mb);
  return c;
}

// psi' = (kslash + m) (pref Vslash) (cL PL + cR PR) psi, pref Vslash from the header
template <class R, class S>
__device__ inline void var_ffv_f(const KParams& P, const Op& o, int v, int ib, const cxT<R>* psi, double gs,
                                 const FfvCtx<R>& c, const S& W) {
  const SlashT<R> Sl = load_slash<R>(W, o.dst + 6 + 8 * ib);
  cxT<R> u0 = cfma(Sl.a01, psi[3], cmul(Sl.a00, psi[2]));
  cxT<R> u1 = cfma(Sl.a11, psi[3], cmul(Sl.a10, psi[2]));
  cxT<R> l0 = cfma(Sl.b01, psi[1], cmul(Sl.b00, psi[0]));
  cxT<R> l1 = cfma(Sl.b11, psi[1], cmul(Sl.b10, psi[0]));
  if (c.chiral) {
    cxT<R> cl, cr;
    bool ch;
    coupling<R>(P, o.cpl, gs, cl, cr, ch);
    u0 = cmul(cr, u0); u1 = cmul(cr, u1);
    l0 = cmul(cl, l0); l1 = cmul(cl, l1);
  }
  // upper = m phi_u + KA phi_l, lower = KB phi_u + m phi_l; KA = [[a00, -(k1-ik2)], [-(k1+ik2), a11]]
  const cxT<R> ka01 = {-c.k1, c.k2}, ka10 = {-c.k1, -c.k2};
  cxT<R> o0 = cfma(ka01, l1, rmul(c.a00, l0));
  cxT<R> o1 = cfma(ka10, l0, rmul(c.a11, l1));
  cxT<R> o2 = cfma(cxT<R>{c.k1, -c.k2}, u1, rmul(c.a11, u0));
  cxT<R> o3 = cfma(cxT<R>{c.k1, c.k2}, u0, rmul(c.a00, u1));
  if (c.massive) {
    o0 = rfma(c.m, u0, o0); o1 = rfma(c.m, u1, o1);
    o2 = rfma(c.m, l0, o2); o3 = rfma(c.m, l1, o3);
  }
  const cxT<R> out[4] = {o0, o1, o2, o3};
  W.store4(c.out + 8 * v, out);
}

// psibar' = psibar (pref Vslash) (cL PL + cR PR) (kslash' + m),  kslash' built from -k
template <class R, class S>
__device__ inline void var_ffv_fb(const KParams& P, const Op& o, int v, int ib, const cxT<R>* pb, double gs,
                                  const FfvCtx<R>& c, const S& W) {
  const SlashT<R> Sl = load_slash<R>(W, o.dst + 6 + 8 * ib);
  const cxT<R> ka01 = {-c.k1, c.k2}, ka10 = {-c.k1, -c.k2};
  cxT<R> xu0 = cfma(pb[3], Sl.b10, cmul(pb[2], Sl.b00));
  cxT<R> xu1 = cfma(pb[3], Sl.b11, cmul(pb[2], Sl.b01));
  cxT<R> xl0 = cfma(pb[1], Sl.a10, cmul(pb[0], Sl.a00));
  cxT<R> xl1 = cfma(pb[1], Sl.a11, cmul(pb[0], Sl.a01));
  if (c.chiral) {
    cxT<R> cl, cr;
    bool ch;
    coupling<R>(P, o.cpl, gs, cl, cr, ch);
    xu0 = cmul(cl, xu0); xu1 = cmul(cl, xu1);
    xl0 = cmul(cr, xl0); xl1 = cmul(cr, xl1);
  }
  // x (kslash + m) = (m x_u + x_l KB, x_u KA + m x_l)
  cxT<R> o0 = cfma(xl1, cneg(ka10), rmul(c.a11, xl0));
  cxT<R> o1 = cfma(xl0, cneg(ka01), rmul(c.a00, xl1));
  cxT<R> o2 = cfma(xu1, ka10, rmul(c.a00, xu0));
  cxT<R> o3 = cfma(xu0, ka01, rmul(c.a11, xu1));
  if (c.massive) {
    o0 = rfma(c.m, xu0, o0); o1 = rfma(c.m, xu1, o1);
    o2 = rfma(c.m, xl0, o2); o3 = rfma(c.m, xl1, o3);
  }
  const cxT<R> out[4] = {o0, o1, o2, o3};
  W.store4(c.out + 8 * v, out);
}

// J = pref (C - k (k.C)/M^2),  C^mu = cL rbar_l sigmabar^mu c_L + cR rbar_u sigma^mu c_R
// (also the column root bilinear, without propagator)
template <class R, class S>
__device__ inline void var_ffv_v(const KParams& P, const Op& o, int v, double gs, const S& W) {
  using T = Real<R>;
  const int hb = pdep(v, o.mdst);
  cxT<R> r[4], c[4];
  W.load4(o.va + 8 * pext(hb, o.ma), r);
  W.load4(o.vb + 8 * pext(hb, o.mb), c);
  const cxT<R> pref = {W[o.dst + 4], W[o.dst + 5]};
  const cxT<R> R00 = cmul(r[0], c[2]), R11 = cmul(r[1], c[3]), R01 = cmul(r[0], c[3]), R10 = cmul(r[1], c[2]);
  const cxT<R> L00 = cmul(r[2], c[0]), L11 = cmul(r[3], c[1]), L01 = cmul(r[2], c[1]), L10 = cmul(r[3], c[0]);
  const cxT<R> Rv[4] = {R00 + R11, R01 + R10, cxT<R>{-(R10.i - R01.i), R10.r - R01.r}, R00 - R11};
  const cxT<R> Lv[4] = {L00 + L11, cneg(L01 + L10), cxT<R>{L10.i - L01.i, -(L10.r - L01.r)}, cneg(L00 - L11)};
  cxT<R> C[4];
  if (P.cplflags[o.cpl] & CPL_CHIRAL) {
    cxT<R> cl, cr;
    bool ch;
    coupling<R>(P, o.cpl, gs, cl, cr, ch);
#pragma unroll
    for (int j = 0; j < 4; ++j) C[j] = cfma(cl, Lv[j], cmul(cr, Rv[j]));
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) C[j] = Lv[j] + Rv[j];
  }
  const double M = P.mass[o.mass];
  if (P.massive[o.mass]) {
    R k[4];
    W.loadk(o.dst, k);
    const cxT<R> f = rmul(T::from(1.0 / (M * M)), rdot(k, C));
#pragma unroll
    for (int j = 0; j < 4; ++j) C[j] = C[j] - rmul(k[j], f);
  }
  cxT<R> out[4];
  apply_pref(pref, C, out);
  W.store4(o.dst + 6 + 8 * v, out);
}

// row bilinear R = pref psibar_root Vslash (cL PL + cR PR): a row spinor, closed later by R . psi
template <class R, class S>
__device__ inline void var_rbil(const KParams& P, const Op& o, int v, double gs, const S& W) {
  const int hb = pdep(v, o.mdst);
  cxT<R> pb[4];
  W.load4(o.va + 8 * pext(hb, o.ma), pb);
  const SlashT<R> Sl = load_slash<R>(W, o.dst + 6 + 8 * pext(hb, o.mb));
  const cxT<R> pref = {W[o.dst + 4], W[o.dst + 5]};
  // psibar Vslash = (psibar_l B, psibar_u A)
  cxT<R> x[4] = {cfma(pb[3], Sl.b10, cmul(pb[2], Sl.b00)), cfma(pb[3], Sl.b11, cmul(pb[2], Sl.b01)),
                 cfma(pb[1], Sl.a10, cmul(pb[0], Sl.a00)), cfma(pb[1], Sl.a11, cmul(pb[0], Sl.a01))};
  if (P.cplflags[o.cpl] & CPL_CHIRAL) {
    cxT<R> cl, cr;
    bool ch;
    coupling<R>(P, o.cpl, gs, cl, cr, ch);
    x[0] = cmul(cl, x[0]); x[1] = cmul(cl, x[1]);
    x[2] = cmul(cr, x[2]); x[3] = cmul(cr, x[3]);
  }
  cxT<R> out[4];
  apply_pref(pref, x, out);
  W.store4(o.dst + 6 + 8 * (nvar_of(o.mb) + v), out);
}

// J^r = i [ (e1.e2) s(k1-k2)^r + e2^r (s(k2-k3).e1) + e1^r (s(k3-k1).e2) ],  s = -g_s/P^2;
// the two single-child dot products come from the header's per-variant tables
template <class R, class S>
__device__ inline void var_vvv(const KParams& P, const Op& o, int v, const S& W) {
  const int hb = pdep(v, o.mdst);
  const int i1 = pext(hb, o.ma), i2 = pext(hb, o.mb);
  const int n1 = nvar_of(o.ma), n2 = nvar_of(o.mb);
  cxT<R> e1[4], e2[4];
  W.load4(o.va + 8 * i1, e1);
  W.load4(o.vb + 8 * i2, e2);
  R d[4];
  W.loadk(o.dst + 6, d);
  const cxT<R> s12 = mdot(e1, e2);
  const cxT<R> a1 = {W[o.dst + 18 + 2 * i1], W[o.dst + 18 + 2 * i1 + 1]};
  const cxT<R> a2 = {W[o.dst + 18 + 2 * (n1 + i2)], W[o.dst + 18 + 2 * (n1 + i2) + 1]};
  cxT<R> out[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const cxT<R> t = cfma(e1[j], a2, cfma(e2[j], a1, rmul(d[j], s12)));
    out[j] = {Real<R>::neg(t.i), t.r};
  }
  W.store4(o.dst + 18 + 2 * (n1 + n2) + 8 * v, out);
}

// the same for a pair loop that holds the first child, its dot and s (k1 - k2) already
template <class R, class S>
__device__ inline void var_vvv_pair(const Op& o, int v, const cxT<R>* e1, cxT<R> a1, int i2, const R* d, int n1,
                               const S& W) {
  cxT<R> e2[4];
  W.load4(o.vb + 8 * i2, e2);
  const cxT<R> s12 = mdot(e1, e2);
  const cxT<R> a2 = {W[o.dst + 18 + 2 * (n1 + i2)], W[o.dst + 18 + 2 * (n1 + i2) + 1]};
  const int n2 = nvar_of(o.mb);
  cxT<R> out[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const cxT<R> t = cfma(e1[j], a2, cfma(e2[j], a1, rmul(d[j], s12)));
    out[j] = {Real<R>::neg(t.i), t.r};
  }
  W.store4(o.dst + 18 + 2 * (n1 + n2) + 8 * v, out);
}

// J = s { j=0: (e1.e3) e2 - (e2.e3) e1 ; j=1: (e1.e2) e3 - (e2.e3) e1 ; j=2: (e1.e2) e3 - (e1.e3) e2 },
// i.e. J = X e_m0 + Y e_m1 with X = s (pair 0 dot), Y = -s (pair 1 dot) from the header's pair
// tables and m0, m1 the children outside pair 0, pair 1
template <class R, class S>
__device__ inline void var_vvvv(const KParams& P, const Op& o, int v, const S& W) {
  const int hb = pdep(v, o.mdst);
  int x0, y0, x1, y1;
  vvvv_pairs(o.aux, x0, y0, x1, y1);
  const int ix0 = pext(hb, child_mask(o, x0)), iy0 = pext(hb, child_mask(o, y0));
  const int ix1 = pext(hb, child_mask(o, x1)), iy1 = pext(hb, child_mask(o, y1));
  const int nx0 = nvar_of(child_mask(o, x0)), ny0 = nvar_of(child_mask(o, y0));
  const int nx1 = nvar_of(child_mask(o, x1)), ny1 = nvar_of(child_mask(o, y1));
  const int t0 = o.dst + 6, t1 = t0 + 2 * nx0 * ny0;
  const cxT<R> X = {W[t0 + 2 * (ix0 + nx0 * iy0)], W[t0 + 2 * (ix0 + nx0 * iy0) + 1]};
  const cxT<R> Y = {W[t1 + 2 * (ix1 + nx1 * iy1)], W[t1 + 2 * (ix1 + nx1 * iy1) + 1]};
  const int m0 = 3 - x0 - y0, m1 = 3 - x1 - y1;
  cxT<R> a[4], b[4];
  W.load4(child_base(o, m0) + 8 * pext(hb, child_mask(o, m0)), a);
  W.load4(child_base(o, m1) + 8 * pext(hb, child_mask(o, m1)), b);
  cxT<R> out[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) out[j] = cfma(X, a[j], cmul(Y, b[j]));
  W.store4(t1 + 2 * nx1 * ny1 + 8 * v, out);
}

// sum current: variant v = sum_t phase_t Y_t[v] over currents Y_t on the same legs; list entries
// (Y variant base, -, -, -), (phase, -, -, -) in the term table from aux, aux2 of them
template <class R, class S>
__device__ inline void var_sum(const KParams& P, const Op& o, int v, const S& W) {
  cxT<R> s[4], y[4];
  for (int t = 0; t < o.aux2; ++t) {
    const int4 a = __ldg(P.terms + 2 * (o.aux + t));
    const int4 b = __ldg(P.terms + 2 * (o.aux + t) + 1);
    W.load4(a.x + 8 * v, y);
    if (t == 0) {
#pragma unroll
      for (int j = 0; j < 4; ++j) s[j] = rot_phase(b.x, y[j]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) s[j] = s[j] + rot_phase(b.x, y[j]);
    }
  }
  W.store4(o.dst + 8 * v, s);
}

template <class R, class S>
__device__ inline void op_variant(const KParams& P, const Op& o, int v, double gs, const double* pe, const S& W) {
  switch (o.code) {
    case OP_EXT: var_ext<R>(P, o, v, pe, W); break;
    case OP_FFV_F:
    case OP_FFV_FB: {
      // variant v = (spinor child variant ia, vector child variant ib)
      const int hb = pdep(v, o.mdst);
      cxT<R> psi[4];
      W.load4(o.va + 8 * pext(hb, o.ma), psi);
      if (o.code == OP_FFV_F)
        var_ffv_f<R>(P, o, v, pext(hb, o.mb), psi, gs, ffv_ctx<R>(P, o, W, false), W);
      else
        var_ffv_fb<R>(P, o, v, pext(hb, o.mb), psi, gs, ffv_ctx<R>(P, o, W, true), W);
      break;
    }
    case OP_FFV_V:
    case OP_BIL: var_ffv_v<R>(P, o, v, gs, W); break;   // the column bilinear is the vertex current without propagator
    case OP_RBIL: var_rbil<R>(P, o, v, gs, W); break;
    case OP_VVV: var_vvv<R>(P, o, v, W); break;
    case OP_SUM: var_sum<R>(P, o, v, W); break;
    default: var_vvvv<R>(P, o, v, W); break;
  }
}

// all nv variants of one op (the thread-per-event kernel): per-op values loaded once
template <class R, class S, class H = AllHel>
__device__ inline void op_variants(const KParams& P, const Op& o, double gs, const double* pe, const S& W,
                                   const H& hs = H()) {
  if (std::is_same<R, float>::value && o.code == OP_VVV) {
    // variants as (first child variant, second child variant) pairs, first child loaded once
    // (float path only: in the float64 kernel the values kept live across the pairs cost spills
    // that outweigh the saved loads)
    R d[4];
    W.loadk(o.dst + 6, d);
    const int n1 = nvar_of(o.ma);
    for (int u1 = 0; u1 < hs.count(o.ma); ++u1) {
      const int i1 = hs.var(u1, o.ma);
      cxT<R> e1[4];
      W.load4(o.va + 8 * i1, e1);
      const cxT<R> a1 = {W[o.dst + 18 + 2 * i1], W[o.dst + 18 + 2 * i1 + 1]};
      const int h1 = pdep(i1, o.ma);
      for (int u2 = 0; u2 < hs.count(o.mb); ++u2) {
        const int i2 = hs.var(u2, o.mb);
        var_vvv_pair<R>(o, pext(h1 | pdep(i2, o.mb), o.mdst), e1, a1, i2, d, n1, W);
      }
    }
    return;
  }
  if (o.code == OP_FFV_F || o.code == OP_FFV_FB) {
    // variants as (spinor child variant, vector child variant) pairs: each spinor variant is
    // loaded once (the op's legs are the disjoint union of its children's)
    const bool row = o.code == OP_FFV_FB;
    const FfvCtx<R> c = ffv_ctx<R>(P, o, W, row);
    for (int ua = 0; ua < hs.count(o.ma); ++ua) {
      const int ia = hs.var(ua, o.ma);
      cxT<R> psi[4];
      W.load4(o.va + 8 * ia, psi);
      const int ha = pdep(ia, o.ma);
      for (int ub = 0; ub < hs.count(o.mb); ++ub) {
        const int ib = hs.var(ub, o.mb);
        const int v = pext(ha | pdep(ib, o.mb), o.mdst);
        if (row)
          var_ffv_fb<R>(P, o, v, ib, psi, gs, c, W);
        else
          var_ffv_f<R>(P, o, v, ib, psi, gs, c, W);
      }
    }
    return;
  }
  for (int u = 0; u < hs.count(o.mdst); ++u) op_variant<R>(P, o, hs.var(u, o.mdst), gs, pe, W);
}

// ================================================================ diagram amplitudes
// A group of diagram terms sharing one colour vector (up to a phase): sum over the group of
// phase_t * amp_t(h), where amp_t = X_t . Y_t with X_t a root bilinear and Y_t the term's other
// current: kind 0, Q . V (column bilinear Q^mu = psibar gamma^mu (..) psi_C, Minkowski dot with
// the vector current) or kind 1, R . psi_C (row bilinear R = psibar Vslash (..), spinor dot with
// the column current); couplings are inside the bilinears.  Terms sharing a bilinear are adjacent
// (a run): the run's phased Y_t are summed first and closed with one product.
// AMP op fields: aux = first term, aux2 = terms, cpl = first flow, mass = flows.
// Term entry: (X base, X mask, Y base, Y mask), (phase, kind, run start, run end).
template <class R, class S>
__device__ __forceinline__ cxT<R> group_amp(const int4* terms, const Op& o, int h, const S& W) {
  const R zero = Real<R>::from(0.0);
  cxT<R> acc{zero, zero}, sum[4];
  bool first_run = true;
  for (int t = 0; t < o.aux2; ++t) {
    const int4 a = __ldg(terms + 2 * (o.aux + t));
    const int4 b = __ldg(terms + 2 * (o.aux + t) + 1);
    cxT<R> Y[4];
    W.load4(a.z + 8 * pext(h, a.w), Y);
    if (b.z) {
#pragma unroll
      for (int j = 0; j < 4; ++j) sum[j] = rot_phase(b.x, Y[j]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) sum[j] = sum[j] + rot_phase(b.x, Y[j]);
    }
    if (b.w) {
      cxT<R> X[4];
      W.load4(a.x + 8 * pext(h, a.y), X);
      cxT<R> amp;
      if (b.y == 0) {
        amp = mdot(X, sum);
      } else {
        amp = cmul(X[0], sum[0]);
        amp = cfma(X[1], sum[1], amp);
        amp = cfma(X[2], sum[2], amp);
        amp = cfma(X[3], sum[3], amp);
      }
      if (first_run) acc = amp;
      else acc = acc + amp;
      first_run = false;
    }
  }
  return acc;
}

}  // namespace mgx
