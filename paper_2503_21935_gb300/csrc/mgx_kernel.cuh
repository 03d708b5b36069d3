// Device side of the matrix-element library: HELAS-style external wavefunctions,
// FFV / VVV / VVVV vertex currents with propagators, root-vertex amplitudes, the
// colour-matrix quadratic form, the helicity sum and helicity / colour selection.
//
// One thread evaluates one event: it walks the process's op table (emitted by the
// process compiler) and computes every off-shell current once per helicity state
// of its own external legs ("variants"), keeping the variants in a per-event
// workspace laid out [offset][thread] so that a warp's accesses are coalesced.
// Diagram amplitudes (one per diagram term) are closed at the root vertex for every
// good helicity and added to the colour-flow amplitudes (jamps); the colour sum
// J^dagger C J, the helicity sum and the selections follow in the same thread.
//
// Feynman rules (all momenta incoming at a vertex; metric +---; chiral gamma basis):
//   f f V : gamma^mu (cL P_L + cR P_R)      qqg: cL = cR = i g_s; photon -i e Q; Z -i gL, -i gR
//   g g g : g_s [g^mn (k1-k2)^r + g^nr (k2-k3)^m + g^rm (k3-k1)^n]  (colour f^abc)
//   gggg  : -i g_s^2 G_j, j = 0..2 one per colour structure
//   fermion propagator i (kslash + m)/(k^2 - m^2 + i m w); vector -i (g - k k/M^2)/(k^2 - M^2 + i M w)
#pragma once
#include <cstdint>

namespace mgx {

enum { OP_EXT = 1, OP_FFV_F = 2, OP_FFV_FB = 3, OP_FFV_V = 4, OP_VVV = 5, OP_VVVV = 6, OP_AMP = 7, OP_BIL = 8, OP_RBIL = 9 };
enum { EXT_U = 0, EXT_V = 1, EXT_UBAR = 2, EXT_VBAR = 3, EXT_EPS_IN = 4, EXT_EPS_OUT = 5 };
enum { CPL_GS = 1, CPL_CHIRAL = 2 };

constexpr int MAXCPL = 8;
constexpr int MAXMASS = 4;
constexpr int MAXHEL = 128;
constexpr int MAXNPAR = 8;

struct KParams {
  const int4* ops;       // 4 int4 (16 int32 fields) per op
  const int2* flows;     // (colour flow, phase code 0..3 for 1, i, -1, -i)
  const int4* terms;     // 2 int4 per diagram term: (bilinear base, mask, other base, mask), (phase, kind, -, -)
  const double* colsym;  // ncol*ncol: C_ii on the diagonal, 2 C_ij above it
  const float* colsym_f;
  int nops, ncol, npar, nin, ngood;
  int cur_doubles, jamp_off, mh_off, colw_off, ws_doubles;
  double avg;            // 1 / (4 Ncol_in S)
  int gs_power;          // |M|^2 carries (4 pi alpha_s)^gs_power; vertices use g_s = 1
  double cpl[MAXCPL][4]; // cL.re cL.im cR.re cR.im
  int cplflags[MAXCPL];
  double mass[MAXMASS], width[MAXMASS];
  int good[MAXHEL];      // canonical indices of the good helicities
};

struct cx {
  double r, i;
};

__device__ __forceinline__ cx cmk(double r, double i) { return cx{r, i}; }
__device__ __forceinline__ cx operator+(cx a, cx b) { return cx{a.r + b.r, a.i + b.i}; }
__device__ __forceinline__ cx operator-(cx a, cx b) { return cx{a.r - b.r, a.i - b.i}; }
__device__ __forceinline__ cx cmul(cx a, cx b) {
  return cx{fma(a.r, b.r, -a.i * b.i), fma(a.r, b.i, a.i * b.r)};
}
// acc + a*b
__device__ __forceinline__ cx cfma(cx a, cx b, cx acc) {
  return cx{fma(a.r, b.r, fma(-a.i, b.i, acc.r)), fma(a.r, b.i, fma(a.i, b.r, acc.i))};
}
__device__ __forceinline__ cx rmul(double s, cx a) { return cx{s * a.r, s * a.i}; }
__device__ __forceinline__ cx rfma(double s, cx a, cx acc) { return cx{fma(s, a.r, acc.r), fma(s, a.i, acc.i)}; }
__device__ __forceinline__ cx conjx(cx a) { return cx{a.r, -a.i}; }
// Minkowski dot of complex 4-vectors (upper components)
__device__ __forceinline__ cx mdot(const cx* a, const cx* b) {
  cx s = cmul(a[0], b[0]);
  s = cfma(cmk(-a[1].r, -a[1].i), b[1], s);
  s = cfma(cmk(-a[2].r, -a[2].i), b[2], s);
  s = cfma(cmk(-a[3].r, -a[3].i), b[3], s);
  return s;
}
// Minkowski dot of a real and a complex 4-vector
__device__ __forceinline__ cx rdot(const double* k, const cx* a) {
  cx s = rmul(k[0], a[0]);
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

// Per-event workspace view: element `off` of this thread lives at base[off * stride].
struct WS {
  double* base;
  int64_t stride;
  __device__ __forceinline__ double& operator[](int off) const { return base[(int64_t)off * stride]; }
  __device__ __forceinline__ void load4(int off, cx* w) const {
#pragma unroll
    for (int j = 0; j < 4; ++j) w[j] = cx{base[(int64_t)(off + 2 * j) * stride], base[(int64_t)(off + 2 * j + 1) * stride]};
  }
  __device__ __forceinline__ void store4(int off, const cx* w) const {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      base[(int64_t)(off + 2 * j) * stride] = w[j].r;
      base[(int64_t)(off + 2 * j + 1) * stride] = w[j].i;
    }
  }
  __device__ __forceinline__ void loadk(int off, double* k) const {
#pragma unroll
    for (int j = 0; j < 4; ++j) k[j] = base[(int64_t)(off + j) * stride];
  }
  __device__ __forceinline__ void storek(int off, const double* k) const {
#pragma unroll
    for (int j = 0; j < 4; ++j) base[(int64_t)(off + j) * stride] = k[j];
  }
};

__device__ __forceinline__ int var_off(int block, int v) { return block + 4 + 8 * v; }

// ---- external wavefunctions (HELAS conventions, helicity eigenstates in the given frame)
// two-component helicity spinors chi_lam(p)
__device__ inline void chi(const double* p, double pp, int lam, cx* c) {
  const double a = pp + p[3];
  if (a > 0.0) {
    const double n = 1.0 / sqrt(2.0 * pp * a);
    if (lam > 0) {
      c[0] = cx{a * n, 0.0};
      c[1] = cx{p[1] * n, p[2] * n};
    } else {
      c[0] = cx{-p[1] * n, p[2] * n};
      c[1] = cx{a * n, 0.0};
    }
  } else if (pp > 0.0) {  // along -z
    if (lam > 0) { c[0] = cx{0.0, 0.0}; c[1] = cx{1.0, 0.0}; }
    else { c[0] = cx{-1.0, 0.0}; c[1] = cx{0.0, 0.0}; }
  } else {                // at rest: quantise along +z
    if (lam > 0) { c[0] = cx{1.0, 0.0}; c[1] = cx{0.0, 0.0}; }
    else { c[0] = cx{0.0, 0.0}; c[1] = cx{1.0, 0.0}; }
  }
}

// u(p, lam): (sqrt(E - lam|p|) chi_lam, sqrt(E + lam|p|) chi_lam); massless: exact chirality
__device__ inline void ext_u(const double* p, double m, int lam, cx* w) {
  const double pp = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
  cx c[2];
  chi(p, pp, lam, c);
  double wu, wl;
  if (m == 0.0) {
    const double s = sqrt(2.0 * p[0]);
    wu = lam < 0 ? s : 0.0;
    wl = lam < 0 ? 0.0 : s;
  } else {
    wu = sqrt(fmax(p[0] - lam * pp, 0.0));
    wl = sqrt(fmax(p[0] + lam * pp, 0.0));
  }
  w[0] = rmul(wu, c[0]); w[1] = rmul(wu, c[1]);
  w[2] = rmul(wl, c[0]); w[3] = rmul(wl, c[1]);
}

// v(p, lam): (sqrt(E + lam|p|) chi_-lam, -sqrt(E - lam|p|) chi_-lam)
__device__ inline void ext_v(const double* p, double m, int lam, cx* w) {
  const double pp = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
  cx c[2];
  chi(p, pp, -lam, c);
  double wu, wl;
  if (m == 0.0) {
    const double s = sqrt(2.0 * p[0]);
    wu = lam > 0 ? s : 0.0;
    wl = lam > 0 ? 0.0 : -s;
  } else {
    wu = sqrt(fmax(p[0] + lam * pp, 0.0));
    wl = -sqrt(fmax(p[0] - lam * pp, 0.0));
  }
  w[0] = rmul(wu, c[0]); w[1] = rmul(wu, c[1]);
  w[2] = rmul(wl, c[0]); w[3] = rmul(wl, c[1]);
}

// psi-bar = psi^dagger gamma^0: swap halves and conjugate
__device__ __forceinline__ void to_bar(cx* w) {
  const cx a = w[0], b = w[1];
  w[0] = conjx(w[2]); w[1] = conjx(w[3]);
  w[2] = conjx(a); w[3] = conjx(b);
}

// eps^mu(k, lam) = (-lam e1 - i e2)/sqrt2 (upper index); outgoing: complex conjugate
__device__ inline void ext_eps(const double* k, int lam, bool outgoing, cx* w) {
  const double kk = sqrt(k[1] * k[1] + k[2] * k[2] + k[3] * k[3]);
  const double pt = sqrt(k[1] * k[1] + k[2] * k[2]);
  double cth = 1.0, sth = 0.0, cph = 1.0, sph = 0.0;
  if (kk > 0.0) { cth = k[3] / kk; sth = pt / kk; }
  if (pt > 0.0) { cph = k[1] / pt; sph = k[2] / pt; }
  const double r = 0.70710678118654752440;
  const double l = (double)lam;
  const double sg = outgoing ? -1.0 : 1.0;
  w[0] = cx{0.0, 0.0};
  w[1] = cx{-l * cth * cph * r, sg * sph * r};
  w[2] = cx{-l * cth * sph * r, -sg * cph * r};
  w[3] = cx{l * sth * r, 0.0};
}

// ---- vertex building blocks
// A = V^0 - V.sigma, B = V^0 + V.sigma for a complex 4-vector V (upper components)
struct Slash {
  cx a00, a01, a10, a11;  // A
  cx b00, b01, b10, b11;  // B
};
__device__ __forceinline__ Slash slash(const cx* V) {
  Slash s;
  s.a00 = V[0] - V[3];
  s.a11 = V[0] + V[3];
  s.b00 = s.a11;
  s.b11 = s.a00;
  const cx v12m = cx{V[1].r + V[2].i, V[1].i - V[2].r};  // V1 - i V2
  const cx v12p = cx{V[1].r - V[2].i, V[1].i + V[2].r};  // V1 + i V2
  s.a01 = cx{-v12m.r, -v12m.i};
  s.a10 = cx{-v12p.r, -v12p.i};
  s.b01 = v12m;
  s.b10 = v12p;
  return s;
}
// real momentum: KA = k0 - k.sigma, KB = k0 + k.sigma (entries with real/imag parts from k)
struct KSlash {
  double a00, a11;  // k0 - k3, k0 + k3 (real)
  cx a01, a10;      // -(k1 - i k2), -(k1 + i k2)
};
__device__ __forceinline__ KSlash kslash(const double* k) {
  KSlash s;
  s.a00 = k[0] - k[3];
  s.a11 = k[0] + k[3];
  s.a01 = cx{-k[1], k[2]};
  s.a10 = cx{-k[1], -k[2]};
  return s;
}

// complex 1/(re + i im)
__device__ __forceinline__ cx cinv(double re, double im) {
  const double d = 1.0 / fma(re, re, im * im);
  return cx{re * d, -im * d};
}
__device__ __forceinline__ double msq(const double* k) {
  return fma(k[0], k[0], -fma(k[1], k[1], fma(k[2], k[2], k[3] * k[3])));
}

}  // namespace mgx
