// MLP surrogate of log|M|^2 over phase space, trained and evaluated by hand-written kernels.
//
// Network: x[24] -> 4 hidden layers of width 256 with SiLU -> scalar.  Weights are kept in
// float32 (master copy, Adam moments) and used in bfloat16 by the tensor cores with float32
// accumulation in tensor memory (tcgen05.mma kind::f16).  The three dense contractions of a
// training step are one generic GEMM C[128 x NT] = A[128 x K] B[NT x K]^T with fused epilogues:
//   forward   Z = X W^T + b, H = silu(Z)                 (A = X, B = W)
//   backward  dZ_prev = (dZ W) * silu'(Z_prev)          (A = dZ, B = W^T)
//   weights   dW = dZ^T X                                (A = dZ^T, B = X^T; contraction over the batch)
// The output layer (256 -> 1), the loss, bias gradients and Adam are plain SIMT kernels.
// The two-stage unweighting that uses the surrogate (Danziger, Janssen, Schumann, Siegert,
// arXiv:2109.11964) is in unweight.cu.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "mgx.h"
#include "umma.cuh"

using namespace mgx;

namespace {

constexpr int kRows = 128;   // batch rows per tile (tcgen05 M)
constexpr int kKc = 64;      // contraction chunk staged in shared memory
constexpr int kWidth = 256;
constexpr int kNin = 24;
constexpr int kK0 = 32;      // input features padded to the bf16 k-step
constexpr int kDepth = 4;    // hidden layers

__device__ __forceinline__ float sigmoidf(float z) { return 1.0f / (1.0f + __expf(-z)); }
__device__ __forceinline__ float siluf(float z) { return z * sigmoidf(z); }
__device__ __forceinline__ float silu_grad(float z) {
  const float s = sigmoidf(z);
  return s * (1.0f + z * (1.0f - s));
}

enum { EPI_FWD = 0, EPI_BWD = 1, EPI_DW = 2 };

struct GemmArgs {
  const __nv_bfloat16* A;  // [M][lda]
  int lda;
  const __nv_bfloat16* B;  // [N][ldb]
  int ldb;
  int M, N, K;             // C is M x N, contraction K (multiple of 16; of kKc when K > kKc)
  int epi;
  // forward: Z fp32 [M][N], H bf16 [M][N], HT bf16 [N][ldt], bias [N]
  // backward: zprev fp32 [M][N] (silu' source), out bf16 [M][N], outT bf16 [N][ldt]
  // weights: dW fp32 [M][N]
  const float* bias;
  const float* zprev;
  float* zout;
  __nv_bfloat16* hout;
  __nv_bfloat16* houtT;
  int ldt;
  float* wout;
  int* err;                // device error counter: +1 per tile whose tensor-core wait ran out
  int skip_mma;            // test hook: issue no MMA, so that the waits run out
  unsigned long long wait_ns;
  int ksplit;              // weights: the contraction is cut into ksplit slices (grid z), slice z writing
                           // its partial product to wout + z M N (summed afterwards in slice order)
};

// One CTA computes C[m0 .. m0+127][n0 .. n0+NT) with NT = min(N - n0, 256) (multiple of 32).
__global__ void __launch_bounds__(kRows) gemm_bf16_kernel(const GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int NT = min(g.N, kWidth);
  const int kc = min(g.K, kKc);
  unsigned char* sa = sm;                                  // 128 x kc bf16
  unsigned char* sb = sa + (size_t)kRows * kc * 2;         // NT x kc bf16
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sb + (size_t)NT * kc * 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.x * kRows, n0 = blockIdx.y * NT;
  uint32_t tcols = 32;
  while ((int)tcols < NT) tcols <<= 1;
  if (tid == 0) umma::mbar_init(mbar, 1);
  if (warp == 0) umma::tmem_alloc_once(tslot, tcols);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t sbo = (uint32_t)(kc / 8) * 128;
  const uint32_t id = umma::idesc(umma::FMT_BF16, kRows, (uint32_t)NT);
  const uint32_t saddr = umma::smem_u32(sa), sbaddr = umma::smem_u32(sb);
  uint32_t phase = 0;
  bool ok = true;
  // this CTA's slice of the contraction (the whole of it unless the weight gradient is split)
  const int nslice = g.ksplit > 1 ? g.ksplit : 1;
  const int chunks = (g.K + kc - 1) / kc, per = (chunks + nslice - 1) / nslice;
  const int kbeg = (int)blockIdx.z * per * kc, kend = min(g.K, kbeg + per * kc);
  float* wout = g.wout ? g.wout + (size_t)blockIdx.z * g.M * g.N : nullptr;
  for (int k0 = kbeg; k0 < kend; k0 += kc) {
    // stage A rows (row tid) and B rows; 16-byte pieces = one core-matrix row each
    const int row = m0 + tid;
    for (int c = 0; c < kc / 8; ++c) {
      uint4 v = make_uint4(0, 0, 0, 0);
      if (row < g.M) v = __ldg(reinterpret_cast<const uint4*>(g.A + (size_t)row * g.lda + k0 + 8 * c));
      *reinterpret_cast<uint4*>(sa + umma::kmajor_offset(tid, 8 * c, kc, 2)) = v;
    }
    for (int r = tid; r < NT; r += kRows) {
      const int nrow = n0 + r;
      for (int c = 0; c < kc / 8; ++c) {
        uint4 v = make_uint4(0, 0, 0, 0);
        if (nrow < g.N) v = __ldg(reinterpret_cast<const uint4*>(g.B + (size_t)nrow * g.ldb + k0 + 8 * c));
        *reinterpret_cast<uint4*>(sb + umma::kmajor_offset(r, 8 * c, kc, 2)) = v;
      }
    }
    umma::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      umma::fence_after_sync();
      if (!g.skip_mma) {
        for (int ks = 0; ks < kc / 16; ++ks)
          umma::mma_f16(tmem, umma::smem_desc(saddr + ks * 256, 128, sbo),
                        umma::smem_desc(sbaddr + ks * 256, 128, sbo), id, (k0 > kbeg || ks > 0) ? 1u : 0u);
        umma::mma_commit(mbar);
      }
    }
    const bool done = umma::mbar_wait(mbar, phase, g.wait_ns);
    phase ^= 1;
    if (!__syncthreads_and(done)) {
      ok = false;
      break;
    }
    umma::fence_after_sync();
  }
  if (ok) {
    // epilogue: TMEM lane tid = row m0 + tid
    const int m = m0 + tid;
    for (int c0 = 0; c0 < NT; c0 += 8) {
      float acc[8];
      umma::tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, acc);
      umma::tmem_wait_ld();
      if (m >= g.M) continue;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int n = n0 + c0 + j;
        if (n >= g.N) continue;
        if (g.epi == EPI_FWD) {
          const float z = acc[j] + g.bias[n];
          const __nv_bfloat16 h = __float2bfloat16_rn(siluf(z));
          g.zout[(size_t)m * g.N + n] = z;
          g.hout[(size_t)m * g.N + n] = h;
          g.houtT[(size_t)n * g.ldt + m] = h;
        } else if (g.epi == EPI_BWD) {
          const __nv_bfloat16 d = __float2bfloat16_rn(acc[j] * silu_grad(g.zprev[(size_t)m * g.N + n]));
          g.hout[(size_t)m * g.N + n] = d;
          g.houtT[(size_t)n * g.ldt + m] = d;
        } else {
          wout[(size_t)m * g.N + n] = kbeg < kend ? acc[j] : 0.0f;   // an empty slice contributes 0
        }
      }
    }
  } else {
    // the tile's outputs become NaN (never stale values), the error is counted, and the block waits
    // (bounded) for MMAs still in flight before it frees its tensor memory
    if (tid == 0 && g.err) atomicAdd(g.err, 1);
    const int m = m0 + tid;
    const float nan = __int_as_float(0x7fc00000);
    if (m < g.M)
      for (int c = 0; c < NT; ++c) {
        const int n = n0 + c;
        if (n >= g.N) break;
        if (g.epi == EPI_FWD) {
          g.zout[(size_t)m * g.N + n] = nan;
          g.hout[(size_t)m * g.N + n] = __float2bfloat16_rn(nan);
          g.houtT[(size_t)n * g.ldt + m] = __float2bfloat16_rn(nan);
        } else if (g.epi == EPI_BWD) {
          g.hout[(size_t)m * g.N + n] = __float2bfloat16_rn(nan);
          g.houtT[(size_t)n * g.ldt + m] = __float2bfloat16_rn(nan);
        } else {
          wout[(size_t)m * g.N + n] = nan;
        }
      }
    umma::mbar_wait(mbar, phase ^ 1, g.wait_ns);
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  if (warp == 0) {
    umma::tmem_dealloc(tmem, tcols);
  }
}

size_t gemm_smem(const GemmArgs& g) {
  const int NT = std::min(g.N, kWidth), kc = std::min(g.K, kKc);
  return (size_t)kRows * kc * 2 + (size_t)NT * kc * 2 + 64;
}

int gemm(const GemmArgs& g, cudaStream_t st) {
  const size_t smem = gemm_smem(g);
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024) != cudaSuccess)
      return MGX_ERR_CUDA;
    attr = true;
  }
  const int NT = std::min(g.N, kWidth);
  dim3 grid((g.M + kRows - 1) / kRows, (g.N + NT - 1) / NT, g.ksplit > 1 ? g.ksplit : 1);
  gemm_bf16_kernel<<<grid, kRows, smem, st>>>(g);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

// ---------------------------------------------------------------- SIMT kernels
// inputs: x fp32 [n][24] -> bf16 [n][32] (zero padded) and its transpose [32][ldt]
__global__ void pack_input_kernel(int n, const float* __restrict__ x, __nv_bfloat16* __restrict__ xb,
                                  __nv_bfloat16* __restrict__ xbT, int ldt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * kK0) return;
  const int r = i / kK0, c = i % kK0;
  const __nv_bfloat16 v = __float2bfloat16_rn(c < kNin ? x[(size_t)r * kNin + c] : 0.0f);
  xb[i] = v;
  if (xbT) xbT[(size_t)c * ldt + r] = v;
}

// output layer y = w4 . h4 + b4 (one warp per row)
__global__ void output_kernel(int n, const __nv_bfloat16* __restrict__ h, const float* __restrict__ w4,
                              const float* __restrict__ b4, float* __restrict__ y) {
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
  if (row >= n) return;
  float acc = 0.0f;
  for (int k = lane; k < kWidth; k += 32) acc = fmaf(__bfloat162float(h[(size_t)row * kWidth + k]), w4[k], acc);
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) y[row] = acc + b4[0];
}

// dy = 2 (y - t)/n, loss partial sums; dZ4 = dy w4 * silu'(Z4) (bf16, row-major and transposed)
__global__ void output_backward_kernel(int n, const float* __restrict__ y, const float* __restrict__ t,
                                       const float* __restrict__ w4, const float* __restrict__ z4,
                                       float* __restrict__ dy, __nv_bfloat16* __restrict__ dz,
                                       __nv_bfloat16* __restrict__ dzT, int ldt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * kWidth) return;
  const int r = i / kWidth, c = i % kWidth;
  const float d = 2.0f * (y[r] - t[r]) / (float)n;
  if (c == 0) dy[r] = d;
  const __nv_bfloat16 v = __float2bfloat16_rn(d * w4[c] * silu_grad(z4[i]));
  dz[i] = v;
  dzT[(size_t)c * ldt + r] = v;
}

// out[i] = sum over slices z (in order) of part[z][i]: the split weight gradient, deterministically
__global__ void slice_sum_kernel(int n, int nslice, const float* __restrict__ part, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float acc = 0.0f;
  for (int z = 0; z < nslice; ++z) acc += part[(size_t)z * n + i];
  out[i] = acc;
}

// column sums over rows of a transposed bf16 matrix [ncol][ld] (bias gradients), one warp per column
__global__ void colsum_kernel(int ncol, int n, const __nv_bfloat16* __restrict__ mT, int ld, float* __restrict__ out) {
  const int c = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
  if (c >= ncol) return;
  float acc = 0.0f;
  for (int r = lane; r < n; r += 32) acc += __bfloat162float(mT[(size_t)c * ld + r]);
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[c] = acc;
}

// output-layer gradients: dw4[k] = sum_r dy[r] h4[r][k], db4 = sum_r dy[r]; loss = mean (y - t)^2
__global__ void output_grad_kernel(int n, const float* __restrict__ dy, const __nv_bfloat16* __restrict__ h4T, int ld,
                                   const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dw4,
                                   float* __restrict__ db4, float* __restrict__ loss) {
  const int c = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
  if (c > kWidth) return;
  float acc = 0.0f;
  for (int r = lane; r < n; r += 32) {
    if (c < kWidth) acc = fmaf(dy[r], __bfloat162float(h4T[(size_t)c * ld + r]), acc);
    else acc += dy[r];
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    if (c < kWidth) dw4[c] = acc;
    else db4[0] = acc;
  }
  if (c == kWidth && loss) {
    float l = 0.0f;
    for (int r = lane; r < n; r += 32) l += (y[r] - t[r]) * (y[r] - t[r]);
    for (int o = 16; o; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if (lane == 0) loss[0] = l / (float)n;
  }
}

// Adam on the flat float32 parameter vector; refreshes the bf16 weight copies (row-major and
// transposed) of the hidden layers
struct ParamLayout {
  int off_w[kDepth], off_b[kDepth], kin[kDepth];
  int off_w4, off_b4, total;
};

__global__ void adam_kernel(int total, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float eps, float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

__global__ void refresh_bf16_kernel(const float* __restrict__ p, ParamLayout L, __nv_bfloat16* __restrict__ wb,
                                    __nv_bfloat16* __restrict__ wbT, __nv_bfloat16* __restrict__ wc) {
  // wb/wbT: per layer blocks of kWidth * kin[l] in the same order as the float weights; wc: the same
  // blocks in the canonical K-major layout [256][kin] that the inference kernel reads from shared memory
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int base = 0;
  for (int l = 0; l < kDepth; ++l) {
    const int sz = kWidth * L.kin[l];
    if (i >= base && i < base + sz) {
      const int j = i - base, r = j / L.kin[l], c = j % L.kin[l];
      const __nv_bfloat16 v = __float2bfloat16_rn(p[L.off_w[l] + j]);
      wb[base + j] = v;
      wbT[base + (size_t)c * kWidth + r] = v;
      wc[base + umma::kmajor_offset(r, c, L.kin[l], 2) / 2] = v;
      return;
    }
    base += sz;
  }
}

// ---------------------------------------------------------------- inference
// Activations between layers live in HBM as canonical K-major tiles: tile t (128 rows) of a K-wide
// activation is K/kc chunks (kc = min(K, 64)) of 128 x kc bf16, each chunk contiguous in exactly the
// layout tcgen05 reads from shared memory, so every operand load is one bulk copy.
constexpr int kInfThreads = 192;   // warps 0-3: epilogue (tensor-memory lanes 0-127); 4: loads; 5: MMAs
constexpr int kInfStages = 4;      // operand chunks in flight
constexpr int64_t kInferRows = 1 << 22;   // rows per pass of the layer kernels (workspace ~1.1 KB / row)

// x tiles [tile][128 x 32] (canonical, K = 32, columns 24..31 zero) from float32 rows x [n][24] times
// inv_scale (in float32) or from float64 momenta [n][24] times inv_scale (rounded to float32 first,
// then to bf16)
__global__ void pack_tiles_kernel(int64_t n, int64_t ntiles, const float* __restrict__ x, const double* __restrict__ mom,
                                  double inv_scale, __nv_bfloat16* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntiles * kRows * (kK0 / 8)) return;
  const int64_t row = i / (kK0 / 8);
  const int grp = (int)(i % (kK0 / 8));
  const int64_t tile = row / kRows;
  const int r = (int)(row % kRows);
  __align__(16) __nv_bfloat16 v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int c = grp * 8 + q;
    float f = 0.0f;
    if (row < n && c < kNin) f = mom ? (float)(mom[row * kNin + c] * inv_scale) : x[row * kNin + c] * (float)inv_scale;
    v[q] = __float2bfloat16_rn(f);
  }
  *reinterpret_cast<uint4*>(out + tile * kRows * kK0 + umma::kmajor_offset(r, grp * 8, kK0, 2) / 2) =
      *reinterpret_cast<const uint4*>(v);
}

struct InferArgs {
  const __nv_bfloat16* a;   // input tiles (K columns)
  const __nv_bfloat16* w;   // this layer's weights, canonical [256][K]
  const float* bias;        // [256]
  int K;                    // 32 or 256
  int64_t ntiles, nrows;
  __nv_bfloat16* h;         // middle layers: output tiles (256 columns); nullptr for the last layer
  const float* w4;          // last layer: the output layer's weights [256] and bias
  const float* b4;
  float* y;                 // last layer: y [nrows]
  int* err;                 // device error counter: +1 per block whose wait ran out
  int skip_mma;             // test hook: issue no MMA, so that the waits run out
  unsigned long long wait_ns;
};

size_t infer_smem(int K) {
  const int kc = K < 64 ? K : 64;
  return (size_t)kWidth * K * 2 + (size_t)kInfStages * kRows * kc * 2 + 2 * kWidth * 4 + 16 * 8 + 16;
}

// One hidden layer (+ the output layer when h == nullptr) over all tiles: a persistent block keeps
// the layer's weights in shared memory, streams the input tiles through a ring of kInfStages chunk
// buffers (bulk copies, warp 4), accumulates each tile's 128 x 256 product into one of two
// tensor-memory accumulators (tcgen05.mma issued by warp 5), and its four epilogue warps apply bias
// and SiLU to the other accumulator meanwhile and write the bf16 activations (or the scalar output).
// Every wait is bounded; a wait that runs out sets the block's abort flag, the remaining outputs of
// the block become NaN and the error is counted.
__global__ void __launch_bounds__(kInfThreads, 1) mlp_infer_kernel(const InferArgs g) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int K = g.K, kc = K < 64 ? K : 64, nch = K / kc;
  const uint32_t wbytes = (uint32_t)kWidth * K * 2, cbytes = (uint32_t)kRows * kc * 2;
  unsigned char* sw = sm;
  unsigned char* sa = sm + wbytes;
  float* sbias = reinterpret_cast<float*>(sa + kInfStages * cbytes);
  float* sw4 = sbias + kWidth;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sw4 + kWidth);
  uint64_t *full = bar, *empty = bar + kInfStages, *accf = bar + 2 * kInfStages, *acce = accf + 2;
  uint64_t *wfull = acce + 2, *drain = wfull + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  if (t == 0) {
    for (int i = 0; i < kInfStages; ++i) {
      umma::mbar_init(full + i, 1);
      umma::mbar_init(empty + i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      umma::mbar_init(accf + i, 1);
      umma::mbar_init(acce + i, 4 * 32);
    }
    umma::mbar_init(wfull, 1);
    umma::mbar_init(drain, 1);
    *abort_flag = 0;
  }
  for (int i = t; i < kWidth; i += kInfThreads) {
    sbias[i] = g.bias[i];
    sw4[i] = g.w4 ? g.w4[i] : 0.0f;
  }
  if (warp == 0) umma::tmem_alloc_once(tslot, 512);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *tslot;
  if (warp == 4) {
    if (lane == 0) {
      // the layer's weights once, then the input tiles' chunks through the ring
      umma::mbar_arrive_expect_tx(wfull, wbytes);
      for (uint32_t o = 0; o < wbytes; o += 16384)
        umma::bulk_g2s(sw + o, reinterpret_cast<const unsigned char*>(g.w) + o, min(16384u, wbytes - o), wfull);
      uint32_t it = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < g.ntiles && ok; tile += gridDim.x)
        for (int c = 0; c < nch; ++c, ++it) {
          const int s = (int)(it % kInfStages);
          if (!umma::mbar_wait(empty + s, ((it / kInfStages) & 1) ^ 1, g.wait_ns) || *abort_flag) {
            ok = false;
            *abort_flag = 1;
            break;
          }
          umma::mbar_arrive_expect_tx(full + s, cbytes);
          umma::bulk_g2s(sa + s * cbytes,
                         reinterpret_cast<const unsigned char*>(g.a) + ((size_t)tile * nch + c) * cbytes, cbytes,
                         full + s);
        }
      // copies still in flight land before the block can exit
      for (uint32_t j = it > kInfStages ? it - kInfStages : 0; j < it; ++j)
        umma::mbar_wait(full + j % kInfStages, (j / kInfStages) & 1, g.wait_ns);
      umma::mbar_wait(wfull, 0, g.wait_ns);
    }
  } else if (warp == 5) {
    if (lane == 0) {
      bool ok = umma::mbar_wait(wfull, 0, g.wait_ns);
      if (!ok) *abort_flag = 1;
      const uint32_t id = umma::idesc(umma::FMT_BF16, kRows, kWidth);
      const uint32_t sbo_a = (uint32_t)(kc * 2 / 16) * 128, sbo_w = (uint32_t)(K * 2 / 16) * 128;
      const uint32_t sa_u = umma::smem_u32(sa), sw_u = umma::smem_u32(sw);
      uint32_t it = 0, lt = 0;
      for (int64_t tile = blockIdx.x; tile < g.ntiles && ok; tile += gridDim.x, ++lt) {
        const uint32_t b = lt & 1;
        if (!umma::mbar_wait(acce + b, ((lt >> 1) & 1) ^ 1, g.wait_ns) || *abort_flag) {
          ok = false;
          break;
        }
        umma::fence_after_sync();
        for (int c = 0; c < nch; ++c, ++it) {
          const int s = (int)(it % kInfStages);
          if (!umma::mbar_wait(full + s, (it / kInfStages) & 1, g.wait_ns) || *abort_flag) {
            ok = false;
            break;
          }
          umma::fence_after_sync();
          if (!g.skip_mma) {
            for (int ks = 0; ks < kc / 16; ++ks)
              umma::mma_f16(tmem + b * kWidth, umma::smem_desc(sa_u + s * cbytes + ks * 256, 128, sbo_a),
                            umma::smem_desc(sw_u + (uint32_t)(c * kc + ks * 16) * 16, 128, sbo_w), id,
                            (c > 0 || ks > 0) ? 1u : 0u);
            umma::mma_commit(empty + s);
          }
        }
        if (!ok) break;
        if (!g.skip_mma) umma::mma_commit(accf + b);
      }
      if (!ok) *abort_flag = 1;
      // every MMA issued has completed before the tensor memory is freed
      if (!g.skip_mma) {
        umma::mma_commit(drain);
        umma::mbar_wait(drain, 0, g.wait_ns);
      }
    }
  } else {
    // epilogue: thread t owns row t of each tile (tensor-memory lane t)
    const float nan = __int_as_float(0x7fc00000);
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    bool ok = true;
    uint32_t lt = 0;
    for (int64_t tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x, ++lt) {
      const uint32_t b = lt & 1;
      if (ok) {
        bool done = umma::mbar_wait(accf + b, (lt >> 1) & 1, g.wait_ns) && !*abort_flag;
        done = __all_sync(0xffffffffu, done);
        if (!done) {
          ok = false;
          *abort_flag = 1;
        }
      }
      umma::fence_after_sync();
      const int64_t row = tile * kRows + t;
      float y = 0.0f;
      unsigned char* out = g.h ? reinterpret_cast<unsigned char*>(g.h) + (size_t)tile * kRows * kWidth * 2 : nullptr;
      for (int n0 = 0; n0 < kWidth; n0 += 32) {
        float v[32];
        if (ok) {
          umma::tmem_ld32(tmem + b * kWidth + lane_base + (uint32_t)n0, v);
          umma::tmem_wait_ld();
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) v[q] = nan;
        }
        if (out) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            __align__(16) __nv_bfloat16 hv[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const float z = v[8 * j + q] + sbias[n0 + 8 * j + q];
              hv[q] = __float2bfloat16_rn(z * __fdividef(1.0f, 1.0f + __expf(-z)));
            }
            const int n = n0 + 8 * j;
            *reinterpret_cast<uint4*>(out + (n / 64) * (kRows * 64 * 2) + umma::kmajor_offset(t, n % 64, 64, 2)) =
                *reinterpret_cast<const uint4*>(hv);
          }
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const float z = v[q] + sbias[n0 + q];
            const float h = __bfloat162float(__float2bfloat16_rn(z * __fdividef(1.0f, 1.0f + __expf(-z))));
            y = fmaf(h, sw4[n0 + q], y);
          }
        }
      }
      if (!out && row < g.nrows) g.y[row] = ok ? y + g.b4[0] : nan;
      umma::fence_before_sync();
      if (ok) umma::mbar_arrive(acce + b);
    }
  }
  __syncthreads();
  if (t == 0 && *abort_flag && g.err) atomicAdd(g.err, 1);
  umma::fence_after_sync();
  if (warp == 0) {
    umma::tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------- host state
ParamLayout layout() {
  ParamLayout L;
  int o = 0;
  for (int l = 0; l < kDepth; ++l) {
    L.kin[l] = l == 0 ? kK0 : kWidth;
    L.off_w[l] = o;
    o += kWidth * L.kin[l];
    L.off_b[l] = o;
    o += kWidth;
  }
  L.off_w4 = o;
  o += kWidth;
  L.off_b4 = o;
  o += 1;
  L.total = o;
  return L;
}

int wb_size(const ParamLayout& L) {
  int s = 0;
  for (int l = 0; l < kDepth; ++l) s += kWidth * L.kin[l];
  return s;
}

}  // namespace

struct mgx_mlp {
  int device = 0;
  ParamLayout L{};
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *wb = nullptr, *wbT = nullptr;
  int step = 0;
  __nv_bfloat16* wc = nullptr;                     // hidden-layer weights in the canonical layout (inference)
  int* d_status = nullptr;                         // device error counter of the GEMM waits
  int skip_mma = 0;                                // test hook
  unsigned long long wait_ns = 1000000000ull;      // time limit of one tensor-core wait
};

namespace {

int wb_offset(const ParamLayout& L, int l) {
  int s = 0;
  for (int j = 0; j < l; ++j) s += kWidth * L.kin[j];
  return s;
}

// workspace for n rows (n padded to a multiple of 128 for the transposed buffers)
constexpr int kDwSlices = 32;   // slices of the batch contraction of a weight gradient (grid z)

struct MlpWs {
  __nv_bfloat16 *x, *xT, *h[kDepth], *hT[kDepth], *dz[2], *dzT[2];
  float *z[kDepth], *y, *dy, *loss;
  float* part;            // [kDwSlices][256][256] partial weight gradients
  int* err;
  int ldt;
  size_t bytes;
};

MlpWs ws_layout(char* base, int n) {
  MlpWs w{};
  const int ldt = (n + kRows - 1) / kRows * kRows;
  w.ldt = ldt;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += (bytes + 255) / 256 * 256;
    return p;
  };
  w.x = (__nv_bfloat16*)take((size_t)ldt * kK0 * 2);
  w.xT = (__nv_bfloat16*)take((size_t)ldt * kK0 * 2);
  for (int l = 0; l < kDepth; ++l) {
    w.h[l] = (__nv_bfloat16*)take((size_t)ldt * kWidth * 2);
    w.hT[l] = (__nv_bfloat16*)take((size_t)ldt * kWidth * 2);
    w.z[l] = (float*)take((size_t)ldt * kWidth * 4);
  }
  for (int j = 0; j < 2; ++j) {
    w.dz[j] = (__nv_bfloat16*)take((size_t)ldt * kWidth * 2);
    w.dzT[j] = (__nv_bfloat16*)take((size_t)ldt * kWidth * 2);
  }
  w.y = (float*)take((size_t)ldt * 4);
  w.dy = (float*)take((size_t)ldt * 4);
  w.loss = (float*)take(256);
  w.part = (float*)take((size_t)kDwSlices * kWidth * kWidth * 4);
  w.err = (int*)take(256);
  w.bytes = off;
  return w;
}

int forward(mgx_mlp* net, int n, const float* x, const MlpWs& w, cudaStream_t st, bool keep_transposes) {
  const ParamLayout& L = net->L;
  pack_input_kernel<<<(n * kK0 + 255) / 256, 256, 0, st>>>(n, x, w.x, keep_transposes ? w.xT : nullptr, w.ldt);
  const __nv_bfloat16* in = w.x;
  int kin = kK0;
  for (int l = 0; l < kDepth; ++l) {
    GemmArgs g{};
    g.A = in; g.lda = kin;
    g.B = net->wb + wb_offset(L, l); g.ldb = kin;
    g.M = n; g.N = kWidth; g.K = kin; g.epi = EPI_FWD;
    g.bias = net->p + L.off_b[l];
    g.zout = w.z[l]; g.hout = w.h[l]; g.houtT = w.hT[l]; g.ldt = w.ldt;
    g.err = net->d_status; g.skip_mma = net->skip_mma; g.wait_ns = net->wait_ns;
    const int rc = gemm(g, st);
    if (rc != MGX_OK) return rc;
    in = w.h[l];
    kin = kWidth;
  }
  output_kernel<<<(n + 7) / 8, 256, 0, st>>>(n, w.h[kDepth - 1], net->p + L.off_w4, net->p + L.off_b4, w.y);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

// gradients of the mean squared error into net->g
int backward(mgx_mlp* net, int n, const float* t, const MlpWs& w, cudaStream_t st) {
  const ParamLayout& L = net->L;
  output_grad_kernel<<<(kWidth + 1 + 7) / 8, 256, 0, st>>>(n, w.dy, w.hT[kDepth - 1], w.ldt, w.y, t, net->g + L.off_w4,
                                                          net->g + L.off_b4, w.loss);
  int cur = 0;
  for (int l = kDepth - 1; l >= 0; --l) {
    const int kin = L.kin[l];
    // dW_l = dZ_l^T X_l (contraction over the batch, padded to ldt rows of zeros)
    GemmArgs gw{};
    gw.A = w.dzT[cur]; gw.lda = w.ldt;
    gw.B = l == 0 ? w.xT : w.hT[l - 1]; gw.ldb = w.ldt;
    gw.M = kWidth; gw.N = kin; gw.K = w.ldt; gw.epi = EPI_DW;
    // the contraction over the batch is cut into slices (more CTAs than the 2 row tiles of dW), each
    // writing a partial product; the slices are summed in order (deterministic)
    const int chunks = (w.ldt + kKc - 1) / kKc;
    gw.ksplit = std::min(kDwSlices, chunks);
    gw.wout = gw.ksplit > 1 ? w.part : net->g + L.off_w[l];
    gw.err = net->d_status; gw.skip_mma = net->skip_mma; gw.wait_ns = net->wait_ns;
    int rc = gemm(gw, st);
    if (rc != MGX_OK) return rc;
    if (gw.ksplit > 1) {
      const int nw = kWidth * kin;
      slice_sum_kernel<<<(nw + 255) / 256, 256, 0, st>>>(nw, gw.ksplit, w.part, net->g + L.off_w[l]);
    }
    colsum_kernel<<<(kWidth + 7) / 8, 256, 0, st>>>(kWidth, n, w.dzT[cur], w.ldt, net->g + L.off_b[l]);
    if (l == 0) break;
    // dZ_{l-1} = (dZ_l W_l) * silu'(Z_{l-1})
    GemmArgs gb{};
    gb.A = w.dz[cur]; gb.lda = kWidth;
    gb.B = net->wbT + wb_offset(L, l); gb.ldb = kWidth;
    gb.M = n; gb.N = kin; gb.K = kWidth; gb.epi = EPI_BWD;
    gb.zprev = w.z[l - 1]; gb.hout = w.dz[cur ^ 1]; gb.houtT = w.dzT[cur ^ 1]; gb.ldt = w.ldt;
    gb.err = net->d_status; gb.skip_mma = net->skip_mma; gb.wait_ns = net->wait_ns;
    rc = gemm(gb, st);
    if (rc != MGX_OK) return rc;
    cur ^= 1;
  }
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

int refresh(mgx_mlp* net, cudaStream_t st) {
  const int n = wb_size(net->L);
  refresh_bf16_kernel<<<(n + 255) / 256, 256, 0, st>>>(net->p, net->L, net->wb, net->wbT, net->wc);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

// inference workspace for passes of `rows` rows: x tiles (K = 32) and two activation tile buffers
struct InferWs {
  __nv_bfloat16 *x, *h0, *h1;
  size_t bytes;
};
InferWs infer_layout(char* base, int64_t rows) {
  const int64_t tiles = (rows + kRows - 1) / kRows;
  InferWs w{};
  const size_t xb = (size_t)tiles * kRows * kK0 * 2, hb = (size_t)tiles * kRows * kWidth * 2;
  w.x = (__nv_bfloat16*)base;
  w.h0 = (__nv_bfloat16*)(base ? base + xb : nullptr);
  w.h1 = (__nv_bfloat16*)(base ? base + xb + hb : nullptr);
  w.bytes = xb + 2 * hb;
  return w;
}

// y[n] = network(rows) for rows given as float32 x [n][24] or float64 momenta [n][24] / scale
int infer(mgx_mlp* net, int64_t n, const float* x, const double* mom, double scale, float* y, void* ws, size_t wsb,
          cudaStream_t st) {
  const int64_t chunk = std::min<int64_t>(n, kInferRows);
  const InferWs w = infer_layout((char*)ws, chunk);
  if (!ws || wsb < w.bytes) return MGX_ERR_WORKSPACE_TOO_SMALL;
  const size_t smem = infer_smem(kWidth);     // the largest: also keeps one block (512 tensor-memory columns) per SM
  static int attr_dev = -1;
  if (attr_dev != net->device) {
    if (cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return MGX_ERR_CUDA;
    attr_dev = net->device;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, net->device);
  const ParamLayout& L = net->L;
  for (int64_t r0 = 0; r0 < n; r0 += chunk) {
    const int64_t m = std::min(chunk, n - r0), tiles = (m + kRows - 1) / kRows;
    const int64_t packs = tiles * kRows * (kK0 / 8);
    pack_tiles_kernel<<<(unsigned)((packs + 255) / 256), 256, 0, st>>>(
        m, tiles, x ? x + r0 * kNin : nullptr, mom ? mom + r0 * kNin : nullptr, 1.0 / scale, w.x);
    const __nv_bfloat16* in = w.x;
    for (int l = 0; l < kDepth; ++l) {
      InferArgs a{};
      a.a = in;
      a.w = net->wc + wb_offset(L, l);
      a.bias = net->p + L.off_b[l];
      a.K = L.kin[l];
      a.ntiles = tiles;
      a.nrows = m;
      const bool last = l == kDepth - 1;
      a.h = last ? nullptr : (l % 2 == 0 ? w.h0 : w.h1);
      a.w4 = net->p + L.off_w4;
      a.b4 = net->p + L.off_b4;
      a.y = y + r0;
      a.err = net->d_status;
      a.skip_mma = net->skip_mma;
      a.wait_ns = net->wait_ns;
      mlp_infer_kernel<<<(unsigned)std::min<int64_t>(tiles, sms), kInfThreads, smem, st>>>(a);
      in = a.h;
    }
    if (cudaGetLastError() != cudaSuccess) return MGX_ERR_CUDA;
  }
  return MGX_OK;
}

}  // namespace

extern "C" {

int mgx_mlp_num_params(void) { return layout().total; }

int mgx_mlp_create(int device, uint64_t seed, mgx_mlp** out) {
  if (!out) return MGX_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cudaSetDevice(device) != cudaSuccess) return MGX_ERR_INVALID_ARGUMENT;
  mgx_mlp* net = new mgx_mlp();
  net->device = device;
  net->L = layout();
  const int total = net->L.total, nwb = wb_size(net->L);
  bool ok = cudaMalloc(&net->p, sizeof(float) * total) == cudaSuccess &&
            cudaMalloc(&net->g, sizeof(float) * total) == cudaSuccess &&
            cudaMalloc(&net->m, sizeof(float) * total) == cudaSuccess &&
            cudaMalloc(&net->v, sizeof(float) * total) == cudaSuccess &&
            cudaMalloc(&net->wb, sizeof(__nv_bfloat16) * nwb) == cudaSuccess &&
            cudaMalloc(&net->wbT, sizeof(__nv_bfloat16) * nwb) == cudaSuccess &&
            cudaMalloc(&net->wc, sizeof(__nv_bfloat16) * nwb) == cudaSuccess &&
            cudaMalloc(&net->d_status, 256) == cudaSuccess && cudaMemset(net->d_status, 0, 256) == cudaSuccess;
  // He-uniform initialisation from a seeded 64-bit LCG (weights of padded input columns zero)
  std::vector<float> h(total, 0.0f);
  uint64_t s = seed * 6364136223846793005ull + 1442695040888963407ull;
  auto uni = [&]() {
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(s >> 11) * (1.0 / 9007199254740992.0);
  };
  for (int l = 0; l < kDepth; ++l) {
    const int fan = l == 0 ? kNin : kWidth;
    const double a = std::sqrt(6.0 / fan);
    for (int r = 0; r < kWidth; ++r)
      for (int c = 0; c < net->L.kin[l]; ++c)
        h[net->L.off_w[l] + r * net->L.kin[l] + c] = c < fan ? (float)((2.0 * uni() - 1.0) * a) : 0.0f;
  }
  const double a4 = std::sqrt(3.0 / kWidth);
  for (int c = 0; c < kWidth; ++c) h[net->L.off_w4 + c] = (float)((2.0 * uni() - 1.0) * a4);
  ok = ok && cudaMemcpy(net->p, h.data(), sizeof(float) * total, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemset(net->m, 0, sizeof(float) * total) == cudaSuccess &&
       cudaMemset(net->v, 0, sizeof(float) * total) == cudaSuccess &&
       cudaMemset(net->g, 0, sizeof(float) * total) == cudaSuccess;
  ok = ok && refresh(net, 0) == MGX_OK && cudaDeviceSynchronize() == cudaSuccess;
  cudaSetDevice(cur);
  if (!ok) {
    mgx_mlp_destroy(net);
    return MGX_ERR_CUDA;
  }
  *out = net;
  return MGX_OK;
}

void mgx_mlp_destroy(mgx_mlp* net) {
  if (!net) return;
  cudaFree(net->p); cudaFree(net->g); cudaFree(net->m); cudaFree(net->v);
  cudaFree(net->wb); cudaFree(net->wbT); cudaFree(net->wc); cudaFree(net->d_status);
  delete net;
}


int mgx_mlp_workspace_bytes(int64_t n, int training, size_t* bytes) {
  if (!bytes || n < 0 || (training && n > (1 << 24))) return MGX_ERR_INVALID_ARGUMENT;
  if (training) {
    *bytes = ws_layout(nullptr, (int)std::max<int64_t>(n, 1)).bytes;
    return MGX_OK;
  }
  *bytes = infer_layout(nullptr, std::min<int64_t>(std::max<int64_t>(n, 1), kInferRows)).bytes;
  return MGX_OK;
}

int mgx_mlp_get_params(const mgx_mlp* net, float* host) {
  if (!net || !host) return MGX_ERR_INVALID_ARGUMENT;
  return cudaMemcpy(host, net->p, sizeof(float) * net->L.total, cudaMemcpyDeviceToHost) == cudaSuccess ? MGX_OK
                                                                                                     : MGX_ERR_CUDA;
}

int mgx_mlp_set_params(mgx_mlp* net, const float* host) {
  if (!net || !host) return MGX_ERR_INVALID_ARGUMENT;
  if (cudaMemcpy(net->p, host, sizeof(float) * net->L.total, cudaMemcpyHostToDevice) != cudaSuccess) return MGX_ERR_CUDA;
  if (refresh(net, 0) != MGX_OK) return MGX_ERR_CUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

int mgx_mlp_forward(mgx_mlp* net, int64_t n, const float* x, float* y, void* ws, size_t wsb, void* stream) {
  if (!net || n < 0 || (n > 0 && (!x || !y))) return MGX_ERR_INVALID_ARGUMENT;
  if (n == 0) return MGX_OK;
  return infer(net, n, x, nullptr, 1.0, y, ws, wsb, (cudaStream_t)stream);
}

int mgx_mlp_forward_momenta_f32(mgx_mlp* net, int64_t n, const float* momenta, double scale, float* y, void* ws,
                                size_t wsb, void* stream) {
  if (!net || n < 0 || (n > 0 && (!momenta || !y)) || !(scale > 0.0)) return MGX_ERR_INVALID_ARGUMENT;
  if (n == 0) return MGX_OK;
  return infer(net, n, momenta, nullptr, scale, y, ws, wsb, (cudaStream_t)stream);
}

int mgx_mlp_forward_momenta(mgx_mlp* net, int64_t n, const double* momenta, double scale, float* y, void* ws,
                            size_t wsb, void* stream) {
  if (!net || n < 0 || (n > 0 && (!momenta || !y)) || !(scale > 0.0)) return MGX_ERR_INVALID_ARGUMENT;
  if (n == 0) return MGX_OK;
  return infer(net, n, nullptr, momenta, scale, y, ws, wsb, (cudaStream_t)stream);
}

// gradients of the mean squared error for one batch, into grad (DEVICE, num_params floats)
int mgx_mlp_gradients(mgx_mlp* net, int n, const float* x, const float* t, float* grad, float* loss, void* ws,
                      size_t wsb, void* stream) {
  if (!net || n <= 0 || n > (1 << 24) || !x || !t) return MGX_ERR_INVALID_ARGUMENT;
  MlpWs w = ws_layout((char*)ws, n);
  if (!ws || wsb < w.bytes) return MGX_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = (cudaStream_t)stream;
  // zero the padded rows of the transposed buffers (they enter the batch contractions)
  if (cudaMemsetAsync(ws, 0, w.bytes, st) != cudaSuccess) return MGX_ERR_CUDA;
  int rc = forward(net, n, x, w, st, true);
  if (rc != MGX_OK) return rc;
  output_backward_kernel<<<(n * kWidth + 255) / 256, 256, 0, st>>>(n, w.y, t, net->p + net->L.off_w4, w.z[kDepth - 1],
                                                                  w.dy, w.dz[0], w.dzT[0], w.ldt);
  rc = backward(net, n, t, w, st);
  if (rc != MGX_OK) return rc;
  if (grad && cudaMemcpyAsync(grad, net->g, sizeof(float) * net->L.total, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return MGX_ERR_CUDA;
  if (loss && cudaMemcpyAsync(loss, w.loss, sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return MGX_ERR_CUDA;
  return MGX_OK;
}

namespace {
// one Adam step on gradient g (DEVICE, num_params floats), then the bf16 copies
int adam_step(mgx_mlp* net, const float* g, float lr, cudaStream_t st) {
  net->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.0f - std::pow(b1, (float)net->step), bc2 = 1.0f - std::pow(b2, (float)net->step);
  adam_kernel<<<(net->L.total + 255) / 256, 256, 0, st>>>(net->L.total, net->p, g, net->m, net->v, lr, b1, b2, 1e-8f,
                                                          bc1, bc2);
  if (cudaGetLastError() != cudaSuccess) return MGX_ERR_CUDA;
  return refresh(net, st);
}
}  // namespace

int mgx_mlp_train_step(mgx_mlp* net, int n, const float* x, const float* t, float lr, float* loss, void* ws, size_t wsb,
                       void* stream) {
  const int rc = mgx_mlp_gradients(net, n, x, t, nullptr, loss, ws, wsb, stream);
  if (rc != MGX_OK) return rc;
  return adam_step(net, net->g, lr, (cudaStream_t)stream);
}

int mgx_mlp_device_errors(mgx_mlp* net, int* count, int reset) {
  if (!net || !count) return MGX_ERR_INVALID_ARGUMENT;
  if (cudaMemcpy(count, net->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return MGX_ERR_CUDA;
  if (reset && cudaMemset(net->d_status, 0, sizeof(int)) != cudaSuccess) return MGX_ERR_CUDA;
  return MGX_OK;
}

int mgx_mlp_set_wait_test(mgx_mlp* net, int skip_mma, double wait_ms) {
  if (!net || wait_ms <= 0.0 || wait_ms > 10000.0) return MGX_ERR_INVALID_ARGUMENT;
  net->skip_mma = skip_mma ? 1 : 0;
  net->wait_ns = (unsigned long long)(wait_ms * 1e6);
  return MGX_OK;
}

int mgx_mlp_adam_step(mgx_mlp* net, const float* grad, float lr, void* stream) {
  if (!net || !grad) return MGX_ERR_INVALID_ARGUMENT;
  return adam_step(net, grad, lr, (cudaStream_t)stream);
}

}  // extern "C"
