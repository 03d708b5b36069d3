// Op executors of the amplitude program (see mgx_kernel.cuh for conventions).
#pragma once
#include "mgx_kernel.cuh"

namespace mgx {

struct Op {
  int code, dst, a, b, c, mdst, ma, mb, mc, cpl, mass, aux, aux2, r0, r1, r2;
};

__device__ __forceinline__ Op load_op(const int4* ops, int i) {
  const int4 x = __ldg(ops + 4 * i), y = __ldg(ops + 4 * i + 1), z = __ldg(ops + 4 * i + 2),
             w = __ldg(ops + 4 * i + 3);
  return Op{x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w, z.x, z.y, z.z, z.w, w.x, w.y, w.z, w.w};
}

// coupling (cL, cR) of an op, g_s applied when flagged
__device__ __forceinline__ void coupling(const KParams& P, int ci, double gs, cx& cl, cx& cr, bool& chiral) {
  const double s = (P.cplflags[ci] & CPL_GS) ? gs : 1.0;
  cl = cx{s * P.cpl[ci][0], s * P.cpl[ci][1]};
  cr = cx{s * P.cpl[ci][2], s * P.cpl[ci][3]};
  chiral = (P.cplflags[ci] & CPL_CHIRAL) != 0;
}

// ---------------------------------------------------------------- externals
__device__ inline void op_ext(const KParams& P, const Op& o, const double* pe, const WS& W) {
  const int leg = o.aux, type = o.aux2;
  const double* p = pe + 4 * leg;
  const double m = P.mass[o.mass];
  double k[4];
  const double sgn = leg < P.nin ? 1.0 : -1.0;  // incoming momentum
#pragma unroll
  for (int j = 0; j < 4; ++j) k[j] = sgn * p[j];
  W.storek(o.dst, k);
  for (int v = 0; v < 2; ++v) {
    const int lam = v ? 1 : -1;
    cx w[4];
    switch (type) {
      case EXT_U: ext_u(p, m, lam, w); break;
      case EXT_V: ext_v(p, m, lam, w); break;
      case EXT_UBAR: ext_u(p, m, lam, w); to_bar(w); break;
      case EXT_VBAR: ext_v(p, m, lam, w); to_bar(w); break;
      case EXT_EPS_IN: ext_eps(p, lam, false, w); break;
      default: ext_eps(p, lam, true, w); break;
    }
    W.store4(var_off(o.dst, v), w);
  }
}

// ---------------------------------------------------------------- f f V -> column spinor
// psi' = i (kslash + m)/(k^2 - m^2 + i m w) * Vslash (cL PL + cR PR) psi,  k = incoming momentum
__device__ inline void op_ffv_f(const KParams& P, const Op& o, double gs, const WS& W) {
  double ka[4], kb[4], k[4];
  W.loadk(o.a, ka);
  W.loadk(o.b, kb);
#pragma unroll
  for (int j = 0; j < 4; ++j) k[j] = ka[j] + kb[j];
  W.storek(o.dst, k);
  const double m = P.mass[o.mass], w = P.width[o.mass];
  const cx inv = cinv(msq(k) - m * m, m * w);
  cx pref = cx{-inv.i, inv.r};  // i / den
  cx cl, cr;
  bool chiral;
  coupling(P, o.cpl, gs, cl, cr, chiral);
  if (!chiral) pref = cmul(pref, cl);
  const KSlash K = kslash(k);
  const int nv = 1 << __popc(o.mdst);
  for (int v = 0; v < nv; ++v) {
    const int hb = pdep(v, o.mdst);
    cx psi[4], V[4];
    W.load4(var_off(o.a, pext(hb, o.ma)), psi);
    W.load4(var_off(o.b, pext(hb, o.mb)), V);
    const Slash S = slash(V);
    // phi_u = A psi_R, phi_l = B psi_L
    cx u0 = cfma(S.a01, psi[3], cmul(S.a00, psi[2]));
    cx u1 = cfma(S.a11, psi[3], cmul(S.a10, psi[2]));
    cx l0 = cfma(S.b01, psi[1], cmul(S.b00, psi[0]));
    cx l1 = cfma(S.b11, psi[1], cmul(S.b10, psi[0]));
    if (chiral) {
      u0 = cmul(cr, u0); u1 = cmul(cr, u1);
      l0 = cmul(cl, l0); l1 = cmul(cl, l1);
    }
    // (kslash + m) phi: upper = m phi_u + KA phi_l, lower = KB phi_u + m phi_l
    cx o0 = cfma(K.a01, l1, rmul(K.a00, l0));
    cx o1 = cfma(K.a10, l0, rmul(K.a11, l1));
    cx o2 = cfma(cx{-K.a01.r, -K.a01.i}, u1, rmul(K.a11, u0));
    cx o3 = cfma(cx{-K.a10.r, -K.a10.i}, u0, rmul(K.a00, u1));
    if (m != 0.0) {
      o0 = rfma(m, u0, o0); o1 = rfma(m, u1, o1);
      o2 = rfma(m, l0, o2); o3 = rfma(m, l1, o3);
    }
    cx out[4] = {cmul(pref, o0), cmul(pref, o1), cmul(pref, o2), cmul(pref, o3)};
    W.store4(var_off(o.dst, v), out);
  }
}

// ---------------------------------------------------------------- f f V -> row spinor
// psibar' = psibar Vslash (cL PL + cR PR) i (kslash + m)/(k^2 - m^2 + i m w), k = -(incoming momentum)
__device__ inline void op_ffv_fb(const KParams& P, const Op& o, double gs, const WS& W) {
  double ka[4], kb[4], kin[4], k[4];
  W.loadk(o.a, ka);
  W.loadk(o.b, kb);
#pragma unroll
  for (int j = 0; j < 4; ++j) { kin[j] = ka[j] + kb[j]; k[j] = -kin[j]; }
  W.storek(o.dst, kin);
  const double m = P.mass[o.mass], w = P.width[o.mass];
  const cx inv = cinv(msq(k) - m * m, m * w);
  cx pref = cx{-inv.i, inv.r};
  cx cl, cr;
  bool chiral;
  coupling(P, o.cpl, gs, cl, cr, chiral);
  if (!chiral) pref = cmul(pref, cl);
  const KSlash K = kslash(k);
  const int nv = 1 << __popc(o.mdst);
  for (int v = 0; v < nv; ++v) {
    const int hb = pdep(v, o.mdst);
    cx pb[4], V[4];
    W.load4(var_off(o.a, pext(hb, o.ma)), pb);
    W.load4(var_off(o.b, pext(hb, o.mb)), V);
    const Slash S = slash(V);
    // x_u = psibar_l B, x_l = psibar_u A   (row vector times matrix)
    cx xu0 = cfma(pb[3], S.b10, cmul(pb[2], S.b00));
    cx xu1 = cfma(pb[3], S.b11, cmul(pb[2], S.b01));
    cx xl0 = cfma(pb[1], S.a10, cmul(pb[0], S.a00));
    cx xl1 = cfma(pb[1], S.a11, cmul(pb[0], S.a01));
    if (chiral) {
      xu0 = cmul(cl, xu0); xu1 = cmul(cl, xu1);
      xl0 = cmul(cr, xl0); xl1 = cmul(cr, xl1);
    }
    // x (kslash + m) = (m x_u + x_l KB, x_u KA + m x_l)
    cx o0 = cfma(xl1, cx{-K.a10.r, -K.a10.i}, rmul(K.a11, xl0));
    cx o1 = cfma(xl0, cx{-K.a01.r, -K.a01.i}, rmul(K.a00, xl1));
    cx o2 = cfma(xu1, K.a10, rmul(K.a00, xu0));
    cx o3 = cfma(xu0, K.a01, rmul(K.a11, xu1));
    if (m != 0.0) {
      o0 = rfma(m, xu0, o0); o1 = rfma(m, xu1, o1);
      o2 = rfma(m, xl0, o2); o3 = rfma(m, xl1, o3);
    }
    cx out[4] = {cmul(pref, o0), cmul(pref, o1), cmul(pref, o2), cmul(pref, o3)};
    W.store4(var_off(o.dst, v), out);
  }
}

// ---------------------------------------------------------------- f f -> V
// C^mu = cL psibar_l sigmabar^mu psi_L + cR psibar_u sigma^mu psi_R;  J = -i (C - k (k.C)/M^2)/den
__device__ inline void op_ffv_v(const KParams& P, const Op& o, double gs, const WS& W) {
  double ka[4], kb[4], k[4];
  W.loadk(o.a, ka);
  W.loadk(o.b, kb);
#pragma unroll
  for (int j = 0; j < 4; ++j) k[j] = ka[j] + kb[j];
  W.storek(o.dst, k);
  const double M = P.mass[o.mass], w = P.width[o.mass];
  const cx inv = cinv(msq(k) - M * M, M * w);
  cx pref = cx{inv.i, -inv.r};  // -i / den
  cx cl, cr;
  bool chiral;
  coupling(P, o.cpl, gs, cl, cr, chiral);
  if (!chiral) pref = cmul(pref, cl);
  const double invm2 = M > 0.0 ? 1.0 / (M * M) : 0.0;
  const int nv = 1 << __popc(o.mdst);
  for (int v = 0; v < nv; ++v) {
    const int hb = pdep(v, o.mdst);
    cx r[4], c[4];
    W.load4(var_off(o.a, pext(hb, o.ma)), r);
    W.load4(var_off(o.b, pext(hb, o.mb)), c);
    // right-handed: r_u sigma^mu c_R with r_u = (r0, r1), c_R = (c2, c3)
    const cx R00 = cmul(r[0], c[2]), R11 = cmul(r[1], c[3]), R01 = cmul(r[0], c[3]), R10 = cmul(r[1], c[2]);
    // left-handed: r_l sigmabar^mu c_L with r_l = (r2, r3), c_L = (c0, c1)
    const cx L00 = cmul(r[2], c[0]), L11 = cmul(r[3], c[1]), L01 = cmul(r[2], c[1]), L10 = cmul(r[3], c[0]);
    cx Rv[4] = {R00 + R11, R01 + R10, cx{-(R10.i - R01.i), R10.r - R01.r}, R00 - R11};
    cx Lv[4] = {L00 + L11, cx{-(L01.r + L10.r), -(L01.i + L10.i)}, cx{L10.i - L01.i, -(L10.r - L01.r)},
                cx{-(L00.r - L11.r), -(L00.i - L11.i)}};
    cx C[4];
    if (chiral) {
#pragma unroll
      for (int j = 0; j < 4; ++j) C[j] = cfma(cl, Lv[j], cmul(cr, Rv[j]));
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) C[j] = Lv[j] + Rv[j];
    }
    if (invm2 != 0.0) {
      const cx kc = rdot(k, C);
      const cx f = rmul(invm2, kc);
#pragma unroll
      for (int j = 0; j < 4; ++j) C[j] = C[j] - rmul(k[j], f);
    }
    cx out[4] = {cmul(pref, C[0]), cmul(pref, C[1]), cmul(pref, C[2]), cmul(pref, C[3])};
    W.store4(var_off(o.dst, v), out);
  }
}

// ---------------------------------------------------------------- g g -> g
// J^r = -i g_s/P^2 [ (e1.e2)(k1-k2)^r + e2^r ((k2-k3).e1) + e1^r ((k3-k1).e2) ],  k3 = -(k1+k2)
__device__ inline void op_vvv(const KParams& P, const Op& o, double gs, const WS& W) {
  double k1[4], k2[4], k[4], d[4], q1[4], q2[4];
  W.loadk(o.a, k1);
  W.loadk(o.b, k2);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    k[j] = k1[j] + k2[j];
    d[j] = k1[j] - k2[j];
    q1[j] = k1[j] + 2.0 * k2[j];   // k2 - k3
    q2[j] = -(2.0 * k1[j] + k2[j]); // k3 - k1
  }
  W.storek(o.dst, k);
  const double s = -gs / msq(k);   // pref = -i g_s / P^2 = i s
  const int nv = 1 << __popc(o.mdst);
  for (int v = 0; v < nv; ++v) {
    const int hb = pdep(v, o.mdst);
    cx e1[4], e2[4];
    W.load4(var_off(o.a, pext(hb, o.ma)), e1);
    W.load4(var_off(o.b, pext(hb, o.mb)), e2);
    const cx s12 = mdot(e1, e2);
    const cx a1 = rdot(q1, e1);
    const cx a2 = rdot(q2, e2);
    cx out[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const cx t = cfma(e1[j], a2, cfma(e2[j], a1, rmul(d[j], s12)));
      out[j] = cx{-s * t.i, s * t.r};  // i s t
    }
    W.store4(var_off(o.dst, v), out);
  }
}

// ---------------------------------------------------------------- g g g -> g (one colour structure)
// J = -g_s^2/P^2 * { j=0: (e1.e3) e2 - (e2.e3) e1 ; j=1: (e1.e2) e3 - (e2.e3) e1 ; j=2: (e1.e2) e3 - (e1.e3) e2 }
__device__ inline void op_vvvv(const KParams& P, const Op& o, double gs, const WS& W) {
  double k1[4], k2[4], k3[4], k[4];
  W.loadk(o.a, k1);
  W.loadk(o.b, k2);
  W.loadk(o.c, k3);
#pragma unroll
  for (int j = 0; j < 4; ++j) k[j] = k1[j] + k2[j] + k3[j];
  W.storek(o.dst, k);
  const double s = -gs * gs / msq(k);
  const int nv = 1 << __popc(o.mdst);
  const int st = o.aux;
  for (int v = 0; v < nv; ++v) {
    const int hb = pdep(v, o.mdst);
    cx e1[4], e2[4], e3[4];
    W.load4(var_off(o.a, pext(hb, o.ma)), e1);
    W.load4(var_off(o.b, pext(hb, o.mb)), e2);
    W.load4(var_off(o.c, pext(hb, o.mc)), e3);
    cx out[4];
    if (st == 0) {
      const cx x = rmul(s, mdot(e1, e3)), y = rmul(-s, mdot(e2, e3));
#pragma unroll
      for (int j = 0; j < 4; ++j) out[j] = cfma(x, e2[j], cmul(y, e1[j]));
    } else if (st == 1) {
      const cx x = rmul(s, mdot(e1, e2)), y = rmul(-s, mdot(e2, e3));
#pragma unroll
      for (int j = 0; j < 4; ++j) out[j] = cfma(x, e3[j], cmul(y, e1[j]));
    } else {
      const cx x = rmul(s, mdot(e1, e2)), y = rmul(-s, mdot(e1, e3));
#pragma unroll
      for (int j = 0; j < 4; ++j) out[j] = cfma(x, e3[j], cmul(y, e2[j]));
    }
    W.store4(var_off(o.dst, v), out);
  }
}

// ---------------------------------------------------------------- root-vertex amplitude
// amp(h) = psibar_root Vslash (cL PL + cR PR) psi, added with its colour phases to the jamps of h
__device__ inline void op_amp(const KParams& P, const Op& o, double gs, const WS& W) {
  cx cl, cr;
  bool chiral;
  coupling(P, o.cpl, gs, cl, cr, chiral);
  const int2* fl = P.flows + o.aux;
  const int nf = o.aux2;
  for (int ih = 0; ih < P.ngood; ++ih) {
    const int h = P.good[ih];
    cx pb[4], psi[4], V[4];
    W.load4(var_off(o.a, pext(h, o.ma)), pb);
    W.load4(var_off(o.b, pext(h, o.mb)), psi);
    W.load4(var_off(o.c, pext(h, o.mc)), V);
    const Slash S = slash(V);
    // right: psibar_u . (A psi_R), left: psibar_l . (B psi_L)
    const cx u0 = cfma(S.a01, psi[3], cmul(S.a00, psi[2]));
    const cx u1 = cfma(S.a11, psi[3], cmul(S.a10, psi[2]));
    const cx l0 = cfma(S.b01, psi[1], cmul(S.b00, psi[0]));
    const cx l1 = cfma(S.b11, psi[1], cmul(S.b10, psi[0]));
    const cx R = cfma(pb[1], u1, cmul(pb[0], u0));
    const cx L = cfma(pb[3], l1, cmul(pb[2], l0));
    cx amp = chiral ? cfma(cl, L, cmul(cr, R)) : cmul(cl, L + R);
    const int jb = P.jamp_off + 2 * P.ncol * ih;
    for (int f = 0; f < nf; ++f) {
      const int2 q = __ldg(fl + f);
      double& jr = W[jb + 2 * q.x];
      double& ji = W[jb + 2 * q.x + 1];
      switch (q.y) {
        case 0: jr += amp.r; ji += amp.i; break;   // +1
        case 1: jr -= amp.i; ji += amp.r; break;   // +i
        case 2: jr -= amp.r; ji -= amp.i; break;   // -1
        default: jr += amp.i; ji -= amp.r; break;  // -i
      }
    }
  }
}

}  // namespace mgx
