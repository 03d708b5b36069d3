// Device-side event generation (the first two steps of the matrix-element generator chain of
// arXiv:2503.21935 Sec. 2, random numbers -> momenta, made data-parallel as in the paper's
// standalone application): Philox-4x32-10 counter-based random numbers (Salmon, Moraes, Dror,
// Shaw, SC'11) and flat phase space by RAMBO (Kleiss, Stirling, Ellis, CPC 40 (1986) 359), plus
// the generator-level cuts used for the surrogate workload.  One thread per event; every event's
// random numbers depend only on (seed, stream, event index).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mgx.h"
#include "philox.cuh"

namespace {

constexpr int kMaxFinal = 8;

__global__ void uniforms_kernel(int64_t n, int64_t first, uint64_t seed, uint32_t stream, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t w[4];
  philox_block(seed, stream, (uint64_t)(first + i), 0, w);
  // 53-bit uniform in [0, 1)
  out[i] = ((double)(w[0] >> 5) * 67108864.0 + (double)(w[1] >> 6)) * (1.0 / 9007199254740992.0);
}

// Real-type helpers of the phase-space kernels.  The float64 versions are the generator's reference
// arithmetic (bit-compatible with the host generator); the float32 versions make cheap proposals
// for the first stage of the unweighting (uniforms converted with rounding toward zero, so that
// r < 1 and -log(r) > 0 in single precision too).
template <class R> struct Ps;
template <> struct Ps<double> {
  static __device__ __forceinline__ double uniform(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }
  static __device__ __forceinline__ void cossin2pi(double r, double* c, double* s) {
    const double f = 2.0 * M_PI * r;
    *c = cos(f);
    *s = sin(f);
  }
  static __device__ __forceinline__ double log_(double x) { return log(x); }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double pow_(double x, double y) { return pow(x, y); }
  static constexpr double kNewtonTol = 1e-15;
};
template <> struct Ps<float> {
  static __device__ __forceinline__ float uniform(uint32_t w) {
    return __uint2float_rz(w) * (1.0f / 4294967296.0f) + (1.0f / 8589934592.0f);
  }
  static __device__ __forceinline__ void cossin2pi(float r, float* c, float* s) { sincospif(2.0f * r, s, c); }
  static __device__ __forceinline__ float log_(float x) { return logf(x); }
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float pow_(float x, float y) { return powf(x, y); }
  static constexpr float kNewtonTol = 1e-6f;
};

// Events first + (idx ? idx[i] : i), i < n, in real type R (momenta [n][nf + 2][4], weight [n]).  The
// final-state count is a template parameter (NF = nf), so the per-particle arrays stay in registers.
template <class R, int NF>
__global__ void rambo_kernel(int64_t n, int64_t first, const int32_t* __restrict__ idx, double sqrts_d,
                             const double* __restrict__ masses_d, uint64_t seed, uint32_t stream,
                             double massless_weight, R* __restrict__ mom, R* __restrict__ weight) {
  using M = Ps<R>;
  constexpr int nf = NF;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t e = (uint64_t)(first + (idx ? (int64_t)idx[i] : i));
  const R sqrts = (R)sqrts_d;
  R masses[NF];
  for (int j = 0; j < nf; ++j) masses[j] = (R)masses_d[j];
  R q[NF][4], p[NF][4];
  R Q[4] = {0, 0, 0, 0};
  for (int j = 0; j < nf; ++j) {
    uint32_t w[4];
    philox_block(seed, stream, e, (uint32_t)j, w);   // words 4j .. 4j+3 of the event
    const R r0 = M::uniform(w[0]), r1 = M::uniform(w[1]), r2 = M::uniform(w[2]), r3 = M::uniform(w[3]);
    const R c = (R)2 * r0 - (R)1, s = M::sqrt_(fmax((R)0, (R)1 - c * c));
    R cf, sf;
    M::cossin2pi(r1, &cf, &sf);
    const R q0 = -M::log_(r2 * r3);
    q[j][0] = q0; q[j][1] = q0 * s * cf; q[j][2] = q0 * s * sf; q[j][3] = q0 * c;
    for (int k = 0; k < 4; ++k) Q[k] += q[j][k];
  }
  const R Mq = M::sqrt_(Q[0] * Q[0] - Q[1] * Q[1] - Q[2] * Q[2] - Q[3] * Q[3]);
  const R b[3] = {-Q[1] / Mq, -Q[2] / Mq, -Q[3] / Mq};
  const R g = Q[0] / Mq, a = (R)1 / ((R)1 + g), x = sqrts / Mq;
  for (int j = 0; j < nf; ++j) {
    const R bq = b[0] * q[j][1] + b[1] * q[j][2] + b[2] * q[j][3];
    p[j][0] = x * (g * q[j][0] + bq);
    for (int k = 0; k < 3; ++k) p[j][1 + k] = x * (q[j][1 + k] + b[k] * q[j][0] + a * bq * b[k]);
  }
  R wt = (R)massless_weight;
  R msum = 0;
  bool massive = false;
  for (int j = 0; j < nf; ++j) { msum += masses[j]; massive |= masses[j] > (R)0; }
  if (massive) {
    // Newton iteration for the common rescaling xi of the three-momenta
    R xi = M::sqrt_((R)1 - (msum / sqrts) * (msum / sqrts));
    for (int it = 0; it < 60; ++it) {
      R fv = -sqrts, df = 0;
      for (int j = 0; j < nf; ++j) {
        const R en = M::sqrt_(masses[j] * masses[j] + xi * xi * p[j][0] * p[j][0]);
        fv += en;
        df += xi * p[j][0] * p[j][0] / en;
      }
      const R step = fv / df;
      xi -= step;
      if (fabs(step) <= M::kNewtonTol * xi) break;
    }
    for (int j = 0; j < nf; ++j) {
      const R e0 = p[j][0];
      p[j][0] = M::sqrt_(masses[j] * masses[j] + xi * xi * e0 * e0);
      for (int k = 1; k < 4; ++k) p[j][k] *= xi;
    }
  }
  // Repair: the boost loses digits when the generated momenta are nearly collinear, so remove
  // the residual three-momentum in proportion to the energies, rescale the three-momenta so the
  // energies (recomputed from them) add up to sqrt(s), and put every particle on its mass shell.
  {
    R r[3] = {0, 0, 0}, esum = 0;
    for (int j = 0; j < nf; ++j) {
      esum += p[j][0];
      for (int k = 0; k < 3; ++k) r[k] += p[j][1 + k];
    }
    R k2[NF];
    for (int j = 0; j < nf; ++j) {
      const R f = p[j][0] / esum;
      for (int k = 0; k < 3; ++k) p[j][1 + k] -= r[k] * f;
      k2[j] = p[j][1] * p[j][1] + p[j][2] * p[j][2] + p[j][3] * p[j][3];
    }
    R xi = 1;
    for (int it = 0; it < 8; ++it) {
      R fv = -sqrts, df = 0;
      for (int j = 0; j < nf; ++j) {
        const R en = M::sqrt_(masses[j] * masses[j] + xi * xi * k2[j]);
        fv += en;
        df += xi * k2[j] / en;
      }
      xi -= fv / df;
    }
    for (int j = 0; j < nf; ++j) {
      for (int k = 1; k < 4; ++k) p[j][k] *= xi;
      p[j][0] = M::sqrt_(masses[j] * masses[j] + p[j][1] * p[j][1] + p[j][2] * p[j][2] + p[j][3] * p[j][3]);
    }
  }
  if (massive) {
    R sk = 0, prod = 1, sk2e = 0;
    for (int j = 0; j < nf; ++j) {
      const R kabs = M::sqrt_(p[j][1] * p[j][1] + p[j][2] * p[j][2] + p[j][3] * p[j][3]);
      sk += kabs;
      prod *= kabs / p[j][0];
      sk2e += kabs * kabs / p[j][0];
    }
    wt *= M::pow_(sk / sqrts, (R)(2 * nf - 3)) * prod * sqrts / sk2e;
  }
  R* out = mom + i * (int64_t)(nf + 2) * 4;
  const R eb = (R)0.5 * sqrts;
  out[0] = eb; out[1] = 0; out[2] = 0; out[3] = eb;
  out[4] = eb; out[5] = 0; out[6] = 0; out[7] = -eb;
  for (int j = 0; j < nf; ++j)
    for (int k = 0; k < 4; ++k) out[8 + 4 * j + k] = p[j][k];
  if (weight) weight[i] = wt;
}

// 1 where every listed final-state particle has pT > ptmin and |eta| < etamax and every pair of
// them is separated by dR > drmin, else 0 (in real type R; the caller may widen the thresholds)
template <class R>
__global__ void cuts_kernel(int64_t n, int npar, const R* __restrict__ mom, int nlist, const int* __restrict__ list,
                            double ptmin_d, double etamax_d, double drmin_d, uint8_t* __restrict__ pass) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const R ptmin = (R)ptmin_d, etamax = (R)etamax_d, drmin = (R)drmin_d;
  const R* pe = mom + i * (int64_t)npar * 4;
  R eta[kMaxFinal], phi[kMaxFinal];
  bool ok = true;
  for (int a = 0; a < nlist; ++a) {
    const R* q = pe + 4 * list[a];
    const R pt = sqrt(q[1] * q[1] + q[2] * q[2]);
    const R pp = sqrt(pt * pt + q[3] * q[3]);
    eta[a] = (R)0.5 * log((pp + q[3]) / (pp - q[3]));
    phi[a] = atan2(q[2], q[1]);
    ok = ok && pt > ptmin && fabs(eta[a]) < etamax;
  }
  for (int a = 0; a < nlist && ok; ++a)
    for (int b2 = a + 1; b2 < nlist; ++b2) {
      R dphi = fabs(phi[a] - phi[b2]);
      if (dphi > (R)M_PI) dphi = (R)(2.0 * M_PI) - dphi;
      const R deta = eta[a] - eta[b2];
      ok = ok && (deta * deta + dphi * dphi > drmin * drmin);
    }
  pass[i] = ok ? 1 : 0;
}

template <class R>
void launch_rambo(int64_t n, int64_t first, const int32_t* idx, double sqrts, int nf, const double* masses,
                  uint64_t seed, double wmassless, R* mom, R* weight, cudaStream_t st) {
  const unsigned blocks = (unsigned)((n + 127) / 128);
  switch (nf) {
#define MGX_RAMBO_CASE(K)                                                                                       \
  case K:                                                                                                       \
    rambo_kernel<R, K><<<blocks, 128, 0, st>>>(n, first, idx, sqrts, masses, seed, 0u, wmassless, mom, weight); \
    break;
    MGX_RAMBO_CASE(2) MGX_RAMBO_CASE(3) MGX_RAMBO_CASE(4) MGX_RAMBO_CASE(5) MGX_RAMBO_CASE(6) MGX_RAMBO_CASE(7)
    MGX_RAMBO_CASE(8)
#undef MGX_RAMBO_CASE
    default: break;
  }
}

double rambo_massless_weight(int n, double sqrts) {
  const double po2 = 0.5 * M_PI;
  double w = std::pow(po2, n - 1) * std::pow(sqrts, 2 * n - 4) / (std::tgamma((double)n) * std::tgamma((double)n - 1));
  return w * std::pow(2.0 * M_PI, 4 - 3 * n);
}

}  // namespace

extern "C" int mgx_uniforms(int64_t n, int64_t first, uint64_t seed, uint32_t stream_id, double* out, void* stream) {
  if (n < 0 || first < 0 || (n > 0 && !out)) return MGX_ERR_INVALID_ARGUMENT;
  if (n == 0) return MGX_OK;
  uniforms_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, first, seed, stream_id, out);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

extern "C" int mgx_rambo(int64_t n, int64_t first, double sqrts, int nfinal, const double* masses_dev, uint64_t seed,
                         double* momenta, double* weight, void* stream) {
  if (n < 0 || first < 0 || nfinal < 2 || nfinal > kMaxFinal || !(sqrts > 0.0) || !masses_dev ||
      (n > 0 && !momenta))
    return MGX_ERR_INVALID_ARGUMENT;
  if (reinterpret_cast<uintptr_t>(momenta) % 16 != 0) return MGX_ERR_INVALID_ARGUMENT;
  if (n == 0) return MGX_OK;
  launch_rambo<double>(n, first, nullptr, sqrts, nfinal, masses_dev, seed, rambo_massless_weight(nfinal, sqrts), momenta,
                       weight, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

extern "C" int mgx_rambo_indexed(int64_t m, const int32_t* index, int64_t first, double sqrts, int nfinal,
                                 const double* masses_dev, uint64_t seed, double* momenta, double* weight,
                                 void* stream) {
  if (m < 0 || first < 0 || nfinal < 2 || nfinal > kMaxFinal || !(sqrts > 0.0) || !masses_dev ||
      (m > 0 && (!momenta || !index)))
    return MGX_ERR_INVALID_ARGUMENT;
  if (reinterpret_cast<uintptr_t>(momenta) % 16 != 0) return MGX_ERR_INVALID_ARGUMENT;
  if (m == 0) return MGX_OK;
  launch_rambo<double>(m, first, index, sqrts, nfinal, masses_dev, seed, rambo_massless_weight(nfinal, sqrts), momenta,
                       weight, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

extern "C" int mgx_rambo_f32(int64_t n, int64_t first, double sqrts, int nfinal, const double* masses_dev,
                             uint64_t seed, float* momenta, float* weight, void* stream) {
  if (n < 0 || first < 0 || nfinal < 2 || nfinal > kMaxFinal || !(sqrts > 0.0) || !masses_dev ||
      (n > 0 && !momenta))
    return MGX_ERR_INVALID_ARGUMENT;
  if (n == 0) return MGX_OK;
  launch_rambo<float>(n, first, nullptr, sqrts, nfinal, masses_dev, seed, rambo_massless_weight(nfinal, sqrts), momenta,
                      weight, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

extern "C" int mgx_cuts(int64_t n, int npar, const double* momenta, int nlist, const int* list_dev, double ptmin,
                        double etamax, double drmin, uint8_t* pass, void* stream) {
  if (n < 0 || npar < 3 || nlist < 0 || nlist > kMaxFinal || (n > 0 && (!momenta || !pass)) || (nlist > 0 && !list_dev))
    return MGX_ERR_INVALID_ARGUMENT;
  if (n == 0) return MGX_OK;
  cuts_kernel<double><<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, npar, momenta, nlist, list_dev,
                                                                                    ptmin, etamax, drmin, pass);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

extern "C" int mgx_cuts_f32(int64_t n, int npar, const float* momenta, int nlist, const int* list_dev, double ptmin,
                            double etamax, double drmin, double margin, uint8_t* pass, void* stream) {
  if (n < 0 || npar < 3 || nlist < 0 || nlist > kMaxFinal || (n > 0 && (!momenta || !pass)) ||
      (nlist > 0 && !list_dev) || !(margin >= 0.0 && margin < 0.5))
    return MGX_ERR_INVALID_ARGUMENT;
  if (n == 0) return MGX_OK;
  cuts_kernel<float><<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      n, npar, momenta, nlist, list_dev, ptmin * (1.0 - margin), etamax * (1.0 + margin), drmin * (1.0 - margin), pass);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}
