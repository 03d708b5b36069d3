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

namespace {

constexpr int kMaxFinal = 8;

__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t h0 = __umulhi(0xD2511F53u, c[0]), l0 = 0xD2511F53u * c[0];
    const uint32_t h1 = __umulhi(0xCD9E8D57u, c[2]), l1 = 0xCD9E8D57u * c[2];
    const uint32_t n0 = h1 ^ c[1] ^ k0, n2 = h0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = l1; c[2] = n2; c[3] = l0;
  }
}

// block `blk` of four words for event e: counter (e lo, blk, stream, e hi), key = seed
__device__ __forceinline__ void philox_block(uint64_t seed, uint32_t stream, uint64_t e, uint32_t blk, uint32_t w[4]) {
  w[0] = (uint32_t)e; w[1] = blk; w[2] = stream; w[3] = (uint32_t)(e >> 32);
  philox10(w, (uint32_t)seed, (uint32_t)(seed >> 32));
}

__global__ void uniforms_kernel(int64_t n, int64_t first, uint64_t seed, uint32_t stream, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t w[4];
  philox_block(seed, stream, (uint64_t)(first + i), 0, w);
  // 53-bit uniform in [0, 1)
  out[i] = ((double)(w[0] >> 5) * 67108864.0 + (double)(w[1] >> 6)) * (1.0 / 9007199254740992.0);
}

__global__ void rambo_kernel(int64_t n, int64_t first, double sqrts, int nf, const double* __restrict__ masses,
                             uint64_t seed, uint32_t stream, double massless_weight, double* __restrict__ mom,
                             double* __restrict__ weight) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t e = (uint64_t)(first + i);
  double q[kMaxFinal][4], p[kMaxFinal][4];
  double Q[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j = 0; j < nf; ++j) {
    uint32_t w[4];
    philox_block(seed, stream, e, (uint32_t)j, w);   // words 4j .. 4j+3 of the event
    const double r0 = ((double)w[0] + 0.5) * (1.0 / 4294967296.0), r1 = ((double)w[1] + 0.5) * (1.0 / 4294967296.0);
    const double r2 = ((double)w[2] + 0.5) * (1.0 / 4294967296.0), r3 = ((double)w[3] + 0.5) * (1.0 / 4294967296.0);
    const double c = 2.0 * r0 - 1.0, s = sqrt(fmax(0.0, 1.0 - c * c)), f = 2.0 * M_PI * r1;
    const double q0 = -log(r2 * r3);
    q[j][0] = q0; q[j][1] = q0 * s * cos(f); q[j][2] = q0 * s * sin(f); q[j][3] = q0 * c;
    for (int k = 0; k < 4; ++k) Q[k] += q[j][k];
  }
  const double M = sqrt(Q[0] * Q[0] - Q[1] * Q[1] - Q[2] * Q[2] - Q[3] * Q[3]);
  const double b[3] = {-Q[1] / M, -Q[2] / M, -Q[3] / M};
  const double g = Q[0] / M, a = 1.0 / (1.0 + g), x = sqrts / M;
  for (int j = 0; j < nf; ++j) {
    const double bq = b[0] * q[j][1] + b[1] * q[j][2] + b[2] * q[j][3];
    p[j][0] = x * (g * q[j][0] + bq);
    for (int k = 0; k < 3; ++k) p[j][1 + k] = x * (q[j][1 + k] + b[k] * q[j][0] + a * bq * b[k]);
  }
  double wt = massless_weight;
  double msum = 0.0;
  bool massive = false;
  for (int j = 0; j < nf; ++j) { msum += masses[j]; massive |= masses[j] > 0.0; }
  if (massive) {
    // Newton iteration for the common rescaling xi of the three-momenta
    double xi = sqrt(1.0 - (msum / sqrts) * (msum / sqrts));
    for (int it = 0; it < 60; ++it) {
      double fv = -sqrts, df = 0.0;
      for (int j = 0; j < nf; ++j) {
        const double en = sqrt(masses[j] * masses[j] + xi * xi * p[j][0] * p[j][0]);
        fv += en;
        df += xi * p[j][0] * p[j][0] / en;
      }
      const double step = fv / df;
      xi -= step;
      if (fabs(step) <= 1e-15 * xi) break;
    }
    for (int j = 0; j < nf; ++j) {
      const double e0 = p[j][0];
      p[j][0] = sqrt(masses[j] * masses[j] + xi * xi * e0 * e0);
      for (int k = 1; k < 4; ++k) p[j][k] *= xi;
    }
  }
  // Repair: the boost loses digits when the generated momenta are nearly collinear, so remove
  // the residual three-momentum in proportion to the energies, rescale the three-momenta so the
  // energies (recomputed from them) add up to sqrt(s), and put every particle on its mass shell.
  {
    double r[3] = {0.0, 0.0, 0.0}, esum = 0.0;
    for (int j = 0; j < nf; ++j) {
      esum += p[j][0];
      for (int k = 0; k < 3; ++k) r[k] += p[j][1 + k];
    }
    double k2[kMaxFinal];
    for (int j = 0; j < nf; ++j) {
      const double f = p[j][0] / esum;
      for (int k = 0; k < 3; ++k) p[j][1 + k] -= r[k] * f;
      k2[j] = p[j][1] * p[j][1] + p[j][2] * p[j][2] + p[j][3] * p[j][3];
    }
    double xi = 1.0;
    for (int it = 0; it < 8; ++it) {
      double fv = -sqrts, df = 0.0;
      for (int j = 0; j < nf; ++j) {
        const double en = sqrt(masses[j] * masses[j] + xi * xi * k2[j]);
        fv += en;
        df += xi * k2[j] / en;
      }
      xi -= fv / df;
    }
    for (int j = 0; j < nf; ++j) {
      for (int k = 1; k < 4; ++k) p[j][k] *= xi;
      p[j][0] = sqrt(masses[j] * masses[j] + p[j][1] * p[j][1] + p[j][2] * p[j][2] + p[j][3] * p[j][3]);
    }
  }
  if (massive) {
    double sk = 0.0, prod = 1.0, sk2e = 0.0;
    for (int j = 0; j < nf; ++j) {
      const double kabs = sqrt(p[j][1] * p[j][1] + p[j][2] * p[j][2] + p[j][3] * p[j][3]);
      sk += kabs;
      prod *= kabs / p[j][0];
      sk2e += kabs * kabs / p[j][0];
    }
    wt *= pow(sk / sqrts, 2 * nf - 3) * prod * sqrts / sk2e;
  }
  double* out = mom + i * (int64_t)(nf + 2) * 4;
  const double eb = 0.5 * sqrts;
  out[0] = eb; out[1] = 0.0; out[2] = 0.0; out[3] = eb;
  out[4] = eb; out[5] = 0.0; out[6] = 0.0; out[7] = -eb;
  for (int j = 0; j < nf; ++j)
    for (int k = 0; k < 4; ++k) out[8 + 4 * j + k] = p[j][k];
  if (weight) weight[i] = wt;
}

// 1 where every listed final-state particle has pT > ptmin and |eta| < etamax and every pair of
// them is separated by dR > drmin, else 0
__global__ void cuts_kernel(int64_t n, int npar, const double* __restrict__ mom, int nlist, const int* __restrict__ list,
                            double ptmin, double etamax, double drmin, uint8_t* __restrict__ pass) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* pe = mom + i * (int64_t)npar * 4;
  double eta[kMaxFinal], phi[kMaxFinal];
  bool ok = true;
  for (int a = 0; a < nlist; ++a) {
    const double* q = pe + 4 * list[a];
    const double pt = sqrt(q[1] * q[1] + q[2] * q[2]);
    const double pp = sqrt(pt * pt + q[3] * q[3]);
    eta[a] = 0.5 * log((pp + q[3]) / (pp - q[3]));
    phi[a] = atan2(q[2], q[1]);
    ok = ok && pt > ptmin && fabs(eta[a]) < etamax;
  }
  for (int a = 0; a < nlist && ok; ++a)
    for (int b2 = a + 1; b2 < nlist; ++b2) {
      double dphi = fabs(phi[a] - phi[b2]);
      if (dphi > M_PI) dphi = 2.0 * M_PI - dphi;
      const double deta = eta[a] - eta[b2];
      ok = ok && (deta * deta + dphi * dphi > drmin * drmin);
    }
  pass[i] = ok ? 1 : 0;
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
  rambo_kernel<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
      n, first, sqrts, nfinal, masses_dev, seed, 0u, rambo_massless_weight(nfinal, sqrts), momenta, weight);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

extern "C" int mgx_cuts(int64_t n, int npar, const double* momenta, int nlist, const int* list_dev, double ptmin,
                        double etamax, double drmin, uint8_t* pass, void* stream) {
  if (n < 0 || npar < 3 || nlist < 0 || nlist > kMaxFinal || (n > 0 && (!momenta || !pass)) || (nlist > 0 && !list_dev))
    return MGX_ERR_INVALID_ARGUMENT;
  if (n == 0) return MGX_OK;
  cuts_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, npar, momenta, nlist, list_dev, ptmin,
                                                                            etamax, drmin, pass);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}
