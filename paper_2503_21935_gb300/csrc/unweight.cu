// Kernels of the (two-stage) unweighting of weighted events.
//
// Plain hit-or-miss: keep an event with probability min(1, w/w_max) and give it the weight
// max(1, w/w_max).  Surrogate two-stage (Danziger, Janssen, Schumann, Siegert, arXiv:2109.11964):
// stage 1 keeps an event with probability min(1, s/s_max) from the cheap surrogate weight s;
// stage 2 evaluates the exact weight w of the survivors only and keeps them with probability
// min(1, (w/s)/r_max).  The kept event carries max(1, s/s_max) max(1, (w/s)/r_max), so the
// expected weight of every phase-space point is (s/s_max)(w/s)/r_max, proportional to w:
// the unweighted sample is unbiased whatever the surrogate's quality, which only sets the
// efficiency.  Survivors are compacted deterministically (scan, then scatter in event order).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "mgx.h"

namespace {

constexpr int kBlock = 256;

// x[i][j] = momenta[i][j] / scale (float32), j over the 4 npar components
__global__ void features_kernel(int64_t n, int ncomp, const double* __restrict__ mom, double inv_scale,
                                float* __restrict__ x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * ncomp) return;
  x[i] = (float)(mom[i] * inv_scale);
}

// s = exp(mean + sd * y) * wps * pass
__global__ void surrogate_weight_kernel(int64_t n, const float* __restrict__ y, double mean, double sd,
                                        const double* __restrict__ wps, const uint8_t* __restrict__ pass,
                                        double* __restrict__ s) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool ok = pass == nullptr || pass[i];
  s[i] = ok ? exp(mean + sd * (double)y[i]) * (wps ? wps[i] : 1.0) : 0.0;
}

// the same from a float32 phase-space weight (the float32 proposals of the first stage)
__global__ void surrogate_weight_f32_kernel(int64_t n, const float* __restrict__ y, double mean, double sd,
                                            const float* __restrict__ wps, const uint8_t* __restrict__ pass,
                                            double* __restrict__ s) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool ok = pass == nullptr || pass[i];
  // a proposal weight only has to be a positive function of the event (stage 2 divides it out), so
  // the exponential runs in float32 (one MUFU op instead of a float64 polynomial on GB300's slow
  // float64 pipe) wherever float32 holds it
  const float af = fmaf((float)sd, y[i], (float)mean);
  const float w = wps ? wps[i] : 1.0f;
  const double v = fabsf(af) < 80.0f ? (double)(__expf(af) * w) : exp(mean + sd * (double)y[i]) * (double)w;
  s[i] = ok ? v : 0.0;
}

// exact weight w = me * wps * pass
__global__ void exact_weight_kernel(int64_t n, const double* __restrict__ me, const double* __restrict__ wps,
                                    const uint8_t* __restrict__ pass, double* __restrict__ w) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool ok = pass == nullptr || pass[i];
  w[i] = ok ? me[i] * (wps ? wps[i] : 1.0) : 0.0;
}

// ratio = w / wref (or w); keep when r * wmax < ratio; overweight = max(1, ratio / wmax)
__global__ void accept_kernel(int64_t n, const double* __restrict__ w, const double* __restrict__ wref, double wmax,
                              const double* __restrict__ r, uint8_t* __restrict__ keep, double* __restrict__ over) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double ratio = w[i];
  if (wref) ratio = wref[i] > 0.0 ? w[i] / wref[i] : 0.0;
  keep[i] = (ratio > 0.0 && r[i] * wmax < ratio) ? 1 : 0;
  if (over) over[i] = fmax(1.0, ratio / wmax);
}

// --- deterministic compaction: per-block counts, one-block scan of the counts, scatter
__global__ void count_kernel(int64_t n, const uint8_t* __restrict__ keep, int32_t* __restrict__ counts) {
  __shared__ int warp_sums[kBlock / 32];
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  const int v = (i < n && keep[i]) ? 1 : 0;
  const int ws = __popc(__ballot_sync(0xffffffffu, v));
  if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = ws;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int k = 0; k < kBlock / 32; ++k) t += warp_sums[k];
    counts[blockIdx.x] = t;
  }
}

__global__ void scan_counts_kernel(int nblocks, int32_t* __restrict__ counts, int32_t* __restrict__ total) {
  // single block: exclusive scan in place, in chunks of kBlock
  __shared__ int32_t buf[kBlock];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nblocks; base += kBlock) {
    const int i = base + threadIdx.x;
    const int v = i < nblocks ? counts[i] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < kBlock; off <<= 1) {
      const int t = threadIdx.x >= off ? buf[threadIdx.x - off] : 0;
      __syncthreads();
      buf[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nblocks) counts[i] = carry + buf[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == kBlock - 1) carry += buf[kBlock - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void scatter_kernel(int64_t n, const uint8_t* __restrict__ keep, const int32_t* __restrict__ offsets,
                               int32_t* __restrict__ index) {
  __shared__ int warp_base[kBlock / 32];
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  const int v = (i < n && keep[i]) ? 1 : 0;
  const unsigned mask = __ballot_sync(0xffffffffu, v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_base[warp] = __popc(mask);
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int k = 0; k < kBlock / 32; ++k) {
      const int c = warp_base[k];
      warp_base[k] = t;
      t += c;
    }
  }
  __syncthreads();
  if (v) index[offsets[blockIdx.x] + warp_base[warp] + __popc(mask & ((1u << lane) - 1))] = (int32_t)i;
}

__global__ void gather_kernel(int64_t m, const int32_t* __restrict__ index, int row, const double* __restrict__ src,
                              double* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m * row) return;
  const int64_t r = i / row, c = i % row;
  dst[i] = src[(int64_t)index[r] * row + c];
}

// training targets: keep = pass && 0 < me < inf, logme = log(me) where kept (0 elsewhere)
__global__ void log_targets_kernel(int64_t n, const double* __restrict__ me, const uint8_t* __restrict__ pass,
                                   double* __restrict__ logme, uint8_t* __restrict__ keep) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double m = me[i];
  const bool k = (!pass || pass[i]) && m > 0.0 && m < INFINITY;
  keep[i] = k ? 1 : 0;
  logme[i] = k ? log(m) : 0.0;
}

// (sum y, sum y^2, max y) in float64, in two passes of fixed order (the same bits on every run):
// block b of MGX_MOMENTS_BLOCKS takes the contiguous range [b c, (b+1) c) of c = ceil(n / blocks)
// values, its 256 threads stride through it in order and a fixed tree combines them into
// part[3 b .. 3 b + 2]; then one block combines the blocks' partials by the same tree.
__device__ void tree3(double& a, double& b, double& c) {
  __shared__ double s1[256], s2[256], s3[256];
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  s3[threadIdx.x] = c;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      s1[threadIdx.x] += s1[threadIdx.x + h];
      s2[threadIdx.x] += s2[threadIdx.x + h];
      s3[threadIdx.x] = fmax(s3[threadIdx.x], s3[threadIdx.x + h]);
    }
    __syncthreads();
  }
  a = s1[0];
  b = s2[0];
  c = s3[0];
}

__global__ void __launch_bounds__(256) moments_part_kernel(int64_t n, const double* __restrict__ y,
                                                            double* __restrict__ part) {
  const int64_t chunk = (n + MGX_MOMENTS_BLOCKS - 1) / MGX_MOMENTS_BLOCKS;
  const int64_t lo = (int64_t)blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
  double a = 0.0, b = 0.0, c = -INFINITY;
  for (int64_t i = lo + threadIdx.x; i < hi; i += 256) {
    const double v = y[i];
    a += v;
    b = fma(v, v, b);
    c = fmax(c, v);
  }
  tree3(a, b, c);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = a;
    part[3 * blockIdx.x + 1] = b;
    part[3 * blockIdx.x + 2] = c;
  }
}

__global__ void __launch_bounds__(256) moments_final_kernel(const double* __restrict__ part, double* __restrict__ out) {
  double a = 0.0, b = 0.0, c = -INFINITY;
  if (threadIdx.x < MGX_MOMENTS_BLOCKS) {
    a = part[3 * threadIdx.x];
    b = part[3 * threadIdx.x + 1];
    c = part[3 * threadIdx.x + 2];
  }
  tree3(a, b, c);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
    out[2] = c;
  }
}

__global__ void standardize_kernel(int64_t n, const double* __restrict__ y, double mean, double sd,
                                   float* __restrict__ t) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  t[i] = (float)((y[i] - mean) / sd);
}

// unweighted events: j-th kept event of the last stage is idx2[j]; with a first stage, its event
// is idx1[idx2[j]] and its weight over1[idx1[idx2[j]]] x over2[idx2[j]]
__global__ void unweighted_out_kernel(int64_t m, const int32_t* __restrict__ idx2, const int32_t* __restrict__ idx1,
                                      const double* __restrict__ over1, const double* __restrict__ over2,
                                      int64_t first, double* __restrict__ weight, int64_t* __restrict__ index) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const int32_t i2 = idx2[j];
  const int32_t i1 = idx1 ? idx1[i2] : i2;
  weight[j] = over2 ? over1[i1] * over2[i2] : over1[i1];
  index[j] = first + i1;
}

unsigned grid(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

// q-quantile of v (linear interpolation between order statistics, positions q (n - 1)); v reordered
double quantile(std::vector<double>& v, double q) {
  if (v.empty()) return 0.0;
  if (q >= 1.0) return *std::max_element(v.begin(), v.end());
  const double pos = q * (double)(v.size() - 1);
  const size_t lo = (size_t)pos;
  std::nth_element(v.begin(), v.begin() + lo, v.end());
  const double a = v[lo];
  if (lo + 1 >= v.size()) return a;
  const double b = *std::min_element(v.begin() + lo + 1, v.end());
  return a + (b - a) * (pos - (double)lo);
}

}  // namespace

extern "C" {

int mgx_features(int64_t n, int ncomp, const double* momenta, double scale, float* x, void* stream) {
  if (n < 0 || ncomp <= 0 || !(scale > 0.0) || (n > 0 && (!momenta || !x))) return MGX_ERR_INVALID_ARGUMENT;
  if (n == 0) return MGX_OK;
  features_kernel<<<grid(n * ncomp), kBlock, 0, (cudaStream_t)stream>>>(n, ncomp, momenta, 1.0 / scale, x);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

int mgx_surrogate_weight(int64_t n, const float* y, double mean, double sd, const double* wps, const uint8_t* pass,
                         double* s, void* stream) {
  if (n < 0 || (n > 0 && (!y || !s))) return MGX_ERR_INVALID_ARGUMENT;
  if (n == 0) return MGX_OK;
  surrogate_weight_kernel<<<grid(n), kBlock, 0, (cudaStream_t)stream>>>(n, y, mean, sd, wps, pass, s);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

int mgx_surrogate_weight_f32(int64_t n, const float* y, double mean, double sd, const float* wps, const uint8_t* pass,
                             double* s, void* stream) {
  if (n < 0 || (n > 0 && (!y || !s))) return MGX_ERR_INVALID_ARGUMENT;
  if (n == 0) return MGX_OK;
  surrogate_weight_f32_kernel<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, (cudaStream_t)stream>>>(
      n, y, mean, sd, wps, pass, s);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

int mgx_exact_weight(int64_t n, const double* me, const double* wps, const uint8_t* pass, double* w, void* stream) {
  if (n < 0 || (n > 0 && (!me || !w))) return MGX_ERR_INVALID_ARGUMENT;
  if (n == 0) return MGX_OK;
  exact_weight_kernel<<<grid(n), kBlock, 0, (cudaStream_t)stream>>>(n, me, wps, pass, w);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

int mgx_accept(int64_t n, const double* w, const double* wref, double wmax, const double* r, uint8_t* keep,
               double* overweight, void* stream) {
  if (n < 0 || !(wmax > 0.0) || (n > 0 && (!w || !r || !keep))) return MGX_ERR_INVALID_ARGUMENT;
  if (n == 0) return MGX_OK;
  accept_kernel<<<grid(n), kBlock, 0, (cudaStream_t)stream>>>(n, w, wref, wmax, r, keep, overweight);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

int mgx_compact_workspace_bytes(int64_t n, size_t* bytes) {
  if (n < 0 || !bytes) return MGX_ERR_INVALID_ARGUMENT;
  *bytes = ((size_t)grid(n) + 64) * sizeof(int32_t);
  return MGX_OK;
}

// index[0 .. count) = positions i with keep[i] != 0, ascending; count written to count_dev
int mgx_compact(int64_t n, const uint8_t* keep, int32_t* index, int32_t* count_dev, void* ws, size_t wsb,
                void* stream) {
  if (n < 0 || n > 0x7fffffff || !count_dev || (n > 0 && (!keep || !index))) return MGX_ERR_INVALID_ARGUMENT;
  cudaStream_t st = (cudaStream_t)stream;
  if (n == 0) return cudaMemsetAsync(count_dev, 0, sizeof(int32_t), st) == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
  size_t need = 0;
  mgx_compact_workspace_bytes(n, &need);
  if (!ws || wsb < need) return MGX_ERR_WORKSPACE_TOO_SMALL;
  int32_t* counts = (int32_t*)ws;
  const unsigned nb = grid(n);
  count_kernel<<<nb, kBlock, 0, st>>>(n, keep, counts);
  scan_counts_kernel<<<1, kBlock, 0, st>>>((int)nb, counts, count_dev);
  scatter_kernel<<<nb, kBlock, 0, st>>>(n, keep, counts, index);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

int mgx_gather(int64_t m, const int32_t* index, int row, const double* src, double* dst, void* stream) {
  if (m < 0 || row <= 0 || (m > 0 && (!index || !src || !dst))) return MGX_ERR_INVALID_ARGUMENT;
  if (m == 0) return MGX_OK;
  gather_kernel<<<grid(m * row), kBlock, 0, (cudaStream_t)stream>>>(m, index, row, src, dst);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

int mgx_log_targets(int64_t n, const double* me, const uint8_t* pass, double* logme, uint8_t* keep, void* stream) {
  if (n < 0 || (n > 0 && (!me || !logme || !keep))) return MGX_ERR_INVALID_ARGUMENT;
  if (n == 0) return MGX_OK;
  log_targets_kernel<<<grid(n), kBlock, 0, (cudaStream_t)stream>>>(n, me, pass, logme, keep);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

int mgx_moments(int64_t n, const double* y, double* sums, void* stream) {
  if (n < 0 || !sums || (n > 0 && !y)) return MGX_ERR_INVALID_ARGUMENT;
  static_assert(MGX_MOMENTS_BLOCKS <= 256, "one thread per partial in the final pass");
  moments_part_kernel<<<MGX_MOMENTS_BLOCKS, 256, 0, (cudaStream_t)stream>>>(n, y, sums + 3);
  moments_final_kernel<<<1, 256, 0, (cudaStream_t)stream>>>(sums + 3, sums);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

int mgx_standardize_f32(int64_t n, const double* y, double mean, double sd, float* t, void* stream) {
  if (n < 0 || !(sd > 0.0) || (n > 0 && (!y || !t))) return MGX_ERR_INVALID_ARGUMENT;
  if (n == 0) return MGX_OK;
  standardize_kernel<<<grid(n), kBlock, 0, (cudaStream_t)stream>>>(n, y, mean, sd, t);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

int mgx_unweighted_out(int64_t m, const int32_t* idx2, const int32_t* idx1, const double* over1, const double* over2,
                       int64_t first, double* weight, int64_t* index, void* stream) {
  if (m < 0 || first < 0 || (m > 0 && (!idx2 || !over1 || !weight || !index))) return MGX_ERR_INVALID_ARGUMENT;
  if (m == 0) return MGX_OK;
  unweighted_out_kernel<<<grid(m), kBlock, 0, (cudaStream_t)stream>>>(m, idx2, idx1, over1, over2, first, weight,
                                                                     index);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

int mgx_unweighting_maxima(int64_t n, const double* w, const double* s, double q, double* maxima, void* stream) {
  if (n < 0 || !maxima || !(q > 0.0) || q > 1.0 || (n > 0 && (!w || !s))) return MGX_ERR_INVALID_ARGUMENT;
  std::vector<double> hw((size_t)n), hs((size_t)n);
  cudaStream_t st = (cudaStream_t)stream;
  if (n > 0 && (cudaMemcpyAsync(hw.data(), w, n * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaMemcpyAsync(hs.data(), s, n * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess))
    return MGX_ERR_CUDA;
  std::vector<double> pw, ps, pr;
  for (int64_t i = 0; i < n; ++i)
    if (hw[i] > 0.0 && hs[i] > 0.0) {
      pw.push_back(hw[i]);
      ps.push_back(hs[i]);
      pr.push_back(hw[i] / hs[i]);
    }
  maxima[0] = quantile(pw, q);
  maxima[1] = quantile(ps, q);
  maxima[2] = quantile(pr, q);
  return MGX_OK;
}

}  // extern "C"
