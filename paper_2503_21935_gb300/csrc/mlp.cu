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
#include "philox.cuh"
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
  int M, N, K;             // C is M x N (N a multiple of 32), contraction K (a multiple of min(K, kKc) and of 16)
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
  int nt;                  // columns per tile (64, 128 or 256; set by gemm())
};

constexpr int kGemmStages = 2;   // shared-memory stages of the contraction (copy of chunk k+1 during MMA k)

// 16-byte asynchronous global -> shared copy (zero-filled when !valid; src must still be a mapped address)
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// One CTA computes C[m0 .. m0+127][n0 .. n0+nt).  The contraction runs in chunks of kc = min(K, 64)
// through two shared-memory stages: the 16-byte cp.async copies of chunk k+1 (canonical K-major
// layout, rows past M or N zero-filled) are in flight while the tensor cores run chunk k; each
// stage's MMAs commit to their own mbarrier, waited on before the stage is refilled.  The epilogue
// reads 32 accumulator columns at a time (TMEM lane = row) and stores them with 16-byte stores.
__global__ void __launch_bounds__(kRows) gemm_bf16_kernel(const GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int NT = g.nt;
  const int kc = min(g.K, kKc);
  const size_t a_bytes = (size_t)kRows * kc * 2, stage_bytes = a_bytes + (size_t)NT * kc * 2;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + kGemmStages * stage_bytes);   // one per stage
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + kGemmStages);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.x * kRows, n0 = blockIdx.y * NT;
  uint32_t tcols = 32;
  while ((int)tcols < NT) tcols <<= 1;
  if (tid == 0)
    for (int s = 0; s < kGemmStages; ++s) umma::mbar_init(&mbar[s], 1);
  if (warp == 0) umma::tmem_alloc_once(tslot, tcols);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t sbo = (uint32_t)(kc / 8) * 128;
  const uint32_t id = umma::idesc(umma::FMT_BF16, kRows, (uint32_t)NT);
  // this CTA's slice of the contraction (the whole of it unless the weight gradient is split)
  const int nslice = g.ksplit > 1 ? g.ksplit : 1;
  const int chunks = (g.K + kc - 1) / kc, per = (chunks + nslice - 1) / nslice;
  const int kbeg = (int)blockIdx.z * per * kc, kend = min(g.K, kbeg + per * kc);
  const int nk = kbeg < kend ? (kend - kbeg) / kc : 0;
  float* wout = g.wout ? g.wout + (size_t)blockIdx.z * g.M * g.N : nullptr;

  auto issue = [&](int k) {   // copies of chunk k into stage k % 2
    const int k0 = kbeg + k * kc;
    unsigned char* sa = sm + (size_t)(k % kGemmStages) * stage_bytes;
    unsigned char* sb = sa + a_bytes;
    const int row = m0 + tid;
    const bool va = row < g.M;
    const __nv_bfloat16* ar = g.A + (size_t)(va ? row : 0) * g.lda + k0;
    for (int c = 0; c < kc / 8; ++c) cp_async16(umma::smem_u32(sa + umma::kmajor_offset(tid, 8 * c, kc, 2)), ar + 8 * c, va);
    for (int r = tid; r < NT; r += kRows) {
      const int nrow = n0 + r;
      const bool vb = nrow < g.N;
      const __nv_bfloat16* br = g.B + (size_t)(vb ? nrow : 0) * g.ldb + k0;
      for (int c = 0; c < kc / 8; ++c) cp_async16(umma::smem_u32(sb + umma::kmajor_offset(r, 8 * c, kc, 2)), br + 8 * c, vb);
    }
    cp_async_commit();
  };
  // chunk j's MMAs commit to mbarrier j % 2 as its (j / 2)-th phase; a stage is refilled only after
  // the chunk that last read it was waited on, so no mbarrier completes twice unobserved
  auto wait_one = [&](int j) {
    return umma::mbar_wait(&mbar[j % kGemmStages], (uint32_t)((j / kGemmStages) & 1), g.wait_ns);
  };
  bool ok = true;
  int waited = 0, issued = 0, failed = -1;   // chunks known complete / whose MMA step ran / timed out
  if (nk > 0) issue(0);
  for (int k = 0; k < nk; ++k) {
    if (k + 1 < nk) {
      // stage (k+1) % 2 was last read by the MMAs of chunk k-1
      if (k >= 1) {
        if (!__syncthreads_and(wait_one(k - 1))) {
          ok = false;
          failed = k - 1;
          break;
        }
        waited = k;
      }
      issue(k + 1);
      cp_async_wait<1>();   // this thread's copies of chunk k have landed
    } else {
      cp_async_wait<0>();
    }
    umma::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0 && !g.skip_mma) {
      umma::fence_after_sync();
      const uint32_t sa = umma::smem_u32(sm + (size_t)(k % kGemmStages) * stage_bytes);
      const uint32_t sb = sa + (uint32_t)a_bytes;
      for (int ks = 0; ks < kc / 16; ++ks)
        umma::mma_f16(tmem, umma::smem_desc(sa + ks * 256, 128, sbo), umma::smem_desc(sb + ks * 256, 128, sbo), id,
                      (k > 0 || ks > 0) ? 1u : 0u);
      umma::mma_commit(&mbar[k % kGemmStages]);
    }
    issued = k + 1;
  }
  for (int j = waited; ok && j < issued; ++j) {
    if (!__syncthreads_and(wait_one(j))) {
      ok = false;
      failed = j;
    } else {
      waited = j + 1;
    }
  }
  cp_async_wait<0>();   // no copy of this block in flight past this point
  umma::fence_after_sync();
  const int m = m0 + tid;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  if (ok) {
    for (int c0 = 0; c0 < NT; c0 += 32) {
      float acc[32];
      umma::tmem_ld32(tmem + lane_base + (uint32_t)c0, acc);
      umma::tmem_wait_ld();
      const int nb = n0 + c0;
      if (m >= g.M || nb >= g.N) continue;
      if (g.epi == EPI_FWD) {
        const float4* b4 = reinterpret_cast<const float4*>(g.bias + nb);
        float4* z4 = reinterpret_cast<float4*>(g.zout + (size_t)m * g.N + nb);
        uint4* h4 = reinterpret_cast<uint4*>(g.hout + (size_t)m * g.N + nb);
        float bv[32];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 t = __ldg(b4 + q);
          bv[4 * q] = t.x; bv[4 * q + 1] = t.y; bv[4 * q + 2] = t.z; bv[4 * q + 3] = t.w;
        }
        uint32_t hp[16];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] += bv[j];
#pragma unroll
        for (int j = 0; j < 16; ++j) hp[j] = pack_bf16x2(siluf(acc[2 * j]), siluf(acc[2 * j + 1]));
#pragma unroll
        for (int q = 0; q < 8; ++q) z4[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
#pragma unroll
        for (int q = 0; q < 4; ++q) h4[q] = make_uint4(hp[4 * q], hp[4 * q + 1], hp[4 * q + 2], hp[4 * q + 3]);
        const __nv_bfloat16* hb = reinterpret_cast<const __nv_bfloat16*>(hp);
#pragma unroll
        for (int j = 0; j < 32; ++j) g.houtT[(size_t)(nb + j) * g.ldt + m] = hb[j];
      } else if (g.epi == EPI_BWD) {
        const float4* zp = reinterpret_cast<const float4*>(g.zprev + (size_t)m * g.N + nb);
        float zv[32];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 t = __ldg(zp + q);
          zv[4 * q] = t.x; zv[4 * q + 1] = t.y; zv[4 * q + 2] = t.z; zv[4 * q + 3] = t.w;
        }
        uint32_t dp[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
          dp[j] = pack_bf16x2(acc[2 * j] * silu_grad(zv[2 * j]), acc[2 * j + 1] * silu_grad(zv[2 * j + 1]));
        uint4* d4 = reinterpret_cast<uint4*>(g.hout + (size_t)m * g.N + nb);
#pragma unroll
        for (int q = 0; q < 4; ++q) d4[q] = make_uint4(dp[4 * q], dp[4 * q + 1], dp[4 * q + 2], dp[4 * q + 3]);
        const __nv_bfloat16* db = reinterpret_cast<const __nv_bfloat16*>(dp);
#pragma unroll
        for (int j = 0; j < 32; ++j) g.houtT[(size_t)(nb + j) * g.ldt + m] = db[j];
      } else {
        float4* w4 = reinterpret_cast<float4*>(wout + (size_t)m * g.N + nb);
        const bool any = nk > 0;   // an empty slice contributes 0
#pragma unroll
        for (int q = 0; q < 8; ++q)
          w4[q] = any ? make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3])
                      : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      }
    }
  } else {
    // the tile's outputs become NaN (never stale values), the error is counted, and the block waits
    // (bounded) for MMAs still in flight before it frees its tensor memory
    if (tid == 0 && g.err) atomicAdd(g.err, 1);
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
    // MMAs really committed and not seen complete: the chunk that timed out, once more, and later ones
    if (!g.skip_mma)
      for (int j = failed; j >= 0 && j < issued; ++j) wait_one(j);
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  if (warp == 0) {
    umma::tmem_dealloc(tmem, tcols);
  }
}

constexpr int kMaxDevices = 64;

int current_device() {
  int dev = 0;
  return cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kMaxDevices ? dev : -1;
}

// SM count of the current device (cached per device)
int sm_count_cached() {
  static int n[kMaxDevices] = {};
  const int dev = current_device();
  if (dev < 0) return 148;
  if (n[dev] <= 0 && (cudaDeviceGetAttribute(&n[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n[dev] <= 0))
    n[dev] = 148;
  return n[dev];
}

size_t gemm_smem(const GemmArgs& g) {
  const int kc = std::min(g.K, kKc);
  return (size_t)kGemmStages * ((size_t)kRows * kc * 2 + (size_t)g.nt * kc * 2) + 64;
}

int gemm(GemmArgs g, cudaStream_t st) {
  const int kc = std::min(g.K, kKc);
  if (g.M <= 0 || g.N <= 0 || g.N % 32 != 0 || g.K <= 0 || g.K % 16 != 0 || g.K % kc != 0)
    return MGX_ERR_INVALID_ARGUMENT;
  // the widest tile (256, 128 or 64 columns) that still gives every SM 3 CTAs: the kernel is bound by
  // the latency of its copies, MMA round trips and epilogue stores, which more resident warps hide
  const int zs = g.ksplit > 1 ? g.ksplit : 1;
  const int64_t mtiles = (int64_t)((g.M + kRows - 1) / kRows) * zs;
  g.nt = std::min(g.N, kWidth);
  while (g.nt > 64 && g.N % (g.nt / 2) == 0 && mtiles * ((g.N + g.nt - 1) / g.nt) < 3 * sm_count_cached()) g.nt /= 2;
  const size_t smem = gemm_smem(g);
  static bool attr[kMaxDevices] = {};   // the attribute is set once per device
  const int dev = current_device();
  if (dev < 0 || !attr[dev]) {
    if (cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024) != cudaSuccess)
      return MGX_ERR_CUDA;
    if (dev >= 0) attr[dev] = true;
  }
  dim3 grid((g.M + kRows - 1) / kRows, (g.N + g.nt - 1) / g.nt, zs);
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

// dy = 2 (y - t)/n; dZ4 = dy w4 * silu'(Z4) (bf16, row-major and transposed).  Block (32, 8) per
// 32 x 32 tile: rows are read and written along the lanes, the transposed copy goes through shared
// memory so that its stores run along the rows too.
__global__ void output_backward_kernel(int n, const float* __restrict__ y, const float* __restrict__ t,
                                       const float* __restrict__ w4, const float* __restrict__ z4,
                                       float* __restrict__ dy, __nv_bfloat16* __restrict__ dz,
                                       __nv_bfloat16* __restrict__ dzT, int ldt) {
  __shared__ __nv_bfloat16 tile[32][34];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32, tx = threadIdx.x, ty = threadIdx.y;
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + tx;
    if (r < n) {
      const float d = 2.0f * (y[r] - t[r]) / (float)n;
      if (c == 0) dy[r] = d;
      const __nv_bfloat16 v = __float2bfloat16_rn(d * w4[c] * silu_grad(z4[(size_t)r * kWidth + c]));
      dz[(size_t)r * kWidth + c] = v;
      tile[i][tx] = v;
    }
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + tx, c = c0 + i;
    if (r < n) dzT[(size_t)c * ldt + r] = tile[tx][i];
  }
}

// sum of one value per thread over a block of 256 threads, in a fixed order (deterministic)
__device__ float block_sum256(float v) {
  __shared__ float part[8];
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  float s = 0.0f;
  if (threadIdx.x == 0)
    for (int w = 0; w < 8; ++w) s += part[w];
  return s;   // valid in thread 0
}

// out[i] = sum over slices z (in order) of part[z][i]: the split weight gradient, deterministically
__global__ void slice_sum_kernel(int n, int nslice, const float* __restrict__ part, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float acc = 0.0f;
  for (int z = 0; z < nslice; ++z) acc += part[(size_t)z * n + i];
  out[i] = acc;
}

// column sums over rows of a transposed bf16 matrix [ncol][ld] (bias gradients), one block of 256
// threads per column
__global__ void colsum_kernel(int ncol, int n, const __nv_bfloat16* __restrict__ mT, int ld, float* __restrict__ out) {
  const int c = blockIdx.x;
  const __nv_bfloat16* row = mT + (size_t)c * ld;   // ld is a multiple of 128: rows are 16-byte aligned
  const int n8 = n / 8;
  float acc = 0.0f;
#pragma unroll 4
  for (int i = threadIdx.x; i < n8; i += 256) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(row) + i);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 f = __bfloat1622float2(h[q]);
      acc += f.x + f.y;
    }
  }
  for (int r = 8 * n8 + threadIdx.x; r < n; r += 256) acc += __bfloat162float(row[r]);
  acc = block_sum256(acc);
  if (threadIdx.x == 0) out[c] = acc;
}

// output-layer gradients, one block of 256 threads per result: dw4[k] = sum_r dy[r] h4[r][k] (blocks
// k < 256), db4 = sum_r dy[r] (block 256), loss = mean (y - t)^2 (block 257)
__global__ void output_grad_kernel(int n, const float* __restrict__ dy, const __nv_bfloat16* __restrict__ h4T, int ld,
                                   const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dw4,
                                   float* __restrict__ db4, float* __restrict__ loss) {
  const int c = blockIdx.x;
  const int n8 = n / 8;   // rows in groups of 8: 16-byte loads (dy, y: workspace rows; t: the caller's
                          // targets, read with 4-byte loads as its alignment is not known)
  float acc = 0.0f;
  if (c < kWidth) {
    const uint4* hr = reinterpret_cast<const uint4*>(h4T + (size_t)c * ld);
    const float4* d4 = reinterpret_cast<const float4*>(dy);
#pragma unroll 4
    for (int i = threadIdx.x; i < n8; i += 256) {
      const uint4 v = __ldg(hr + i);
      const float4 a = __ldg(d4 + 2 * i), b = __ldg(d4 + 2 * i + 1);
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
      const float2 h0 = __bfloat1622float2(h[0]), h1 = __bfloat1622float2(h[1]), h2 = __bfloat1622float2(h[2]),
                   h3 = __bfloat1622float2(h[3]);
      acc = fmaf(a.x, h0.x, acc); acc = fmaf(a.y, h0.y, acc); acc = fmaf(a.z, h1.x, acc); acc = fmaf(a.w, h1.y, acc);
      acc = fmaf(b.x, h2.x, acc); acc = fmaf(b.y, h2.y, acc); acc = fmaf(b.z, h3.x, acc); acc = fmaf(b.w, h3.y, acc);
    }
    for (int r = 8 * n8 + threadIdx.x; r < n; r += 256) acc = fmaf(dy[r], __bfloat162float(h4T[(size_t)c * ld + r]), acc);
  } else if (c == kWidth) {
    const float4* d4 = reinterpret_cast<const float4*>(dy);
#pragma unroll 4
    for (int i = threadIdx.x; i < 2 * n8; i += 256) {
      const float4 a = __ldg(d4 + i);
      acc += (a.x + a.y) + (a.z + a.w);
    }
    for (int r = 8 * n8 + threadIdx.x; r < n; r += 256) acc += dy[r];
  } else {
#pragma unroll 8
    for (int r = threadIdx.x; r < n; r += 256) {
      const float e = y[r] - __ldg(t + r);
      acc = fmaf(e, e, acc);
    }
  }
  acc = block_sum256(acc);
  if (threadIdx.x == 0) {
    if (c < kWidth) dw4[c] = acc;
    else if (c == kWidth) db4[0] = acc;
    else if (loss) loss[0] = acc / (float)n;
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

// A training batch drawn with replacement from ntotal examples: batch row r takes example
// j = floor(u ntotal), u = (first word of the Philox-4x32-10 block with counter (r, step,
// kSampleStream, 0) under key seed) / 2^32, computed as (word x ntotal) >> 32.
constexpr uint32_t kSampleStream = 0x4D4C5053u;

__global__ void sample_rows_kernel(int batch, int ntotal, const float* __restrict__ x, const float* __restrict__ t,
                                   uint64_t seed, uint32_t step, float* __restrict__ xs, float* __restrict__ ts) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= batch) return;
  uint32_t w[4];
  philox_block(seed, kSampleStream, (uint64_t)r, step, w);
  const int j = (int)(((uint64_t)w[0] * (uint64_t)ntotal) >> 32);
#pragma unroll
  for (int c = 0; c < kNin; ++c) xs[(size_t)r * kNin + c] = x[(size_t)j * kNin + c];
  ts[r] = t[j];
}

// ---------------------------------------------------------------- inference
// Activations between layers live in HBM as canonical K-major tiles: tile t (128 rows) of a K-wide
// activation is K/kc chunks (kc = min(K, 64)) of 128 x kc bf16, each chunk contiguous in exactly the
// layout tcgen05 reads from shared memory, so every operand load is one bulk copy.
constexpr int kInfThreads = 320;   // warps 0-7: epilogue (warp w: tensor-memory lanes 32 (w % 4) .. +31,
                                   // columns 128 (w / 4) .. +127); 8: loads; 9: MMAs
constexpr int kInfEpi = 256;       // epilogue threads
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
  return (size_t)kWidth * K * 2 + (size_t)kInfStages * kRows * kc * 2 + 2 * kWidth * 4 + 2 * 2 * kRows * 4 + 16 * 8 +
         16;
}

// One hidden layer (+ the output layer when h == nullptr) over all tiles: a persistent block keeps
// the layer's weights in shared memory, streams the input tiles through a ring of kInfStages chunk
// buffers (bulk copies, warp 8), accumulates each tile's 128 x 256 product into one of two
// tensor-memory accumulators (tcgen05.mma issued by warp 9), and its eight epilogue warps (two per
// tensor-memory lane quarter, one per half of the columns) apply bias and SiLU to the other
// accumulator meanwhile and write the bf16 activations; in the last layer each half forms its part
// of the 256 -> 1 output, and the two parts are added in shared memory (one named barrier per tile).
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
  float* ypart = sw4 + kWidth;   // [tile parity][column half][row] partial outputs of the last layer
  uint64_t* bar = reinterpret_cast<uint64_t*>(ypart + 2 * 2 * kRows);
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
      umma::mbar_init(acce + i, kInfEpi);
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
  if (warp == 8) {
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
  } else if (warp == 9) {
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
    // epilogue: warp w owns rows 32 (w % 4) .. +31 of each tile (its tensor-memory lane quarter) and
    // columns 128 (w / 4) .. +127
    const float nan = __int_as_float(0x7fc00000);
    const int quarter = warp & 3, half = warp >> 2, r = quarter * 32 + lane;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    const int c_lo = half * (kWidth / 2);
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
      const int64_t row = tile * kRows + r;
      float y = 0.0f;
      unsigned char* out = g.h ? reinterpret_cast<unsigned char*>(g.h) + (size_t)tile * kRows * kWidth * 2 : nullptr;
      for (int n0 = c_lo; n0 < c_lo + kWidth / 2; n0 += 32) {
        float v[32];
        if (ok) {
          umma::tmem_ld32(tmem + b * kWidth + lane_base + (uint32_t)n0, v);
          umma::tmem_wait_ld();
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) v[q] = nan;
        }
        float bv[32];   // this chunk's bias (shared memory, 16-byte loads)
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 f = reinterpret_cast<const float4*>(sbias + n0)[q];
          bv[4 * q] = f.x; bv[4 * q + 1] = f.y; bv[4 * q + 2] = f.z; bv[4 * q + 3] = f.w;
        }
        if (out) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            __align__(16) __nv_bfloat16 hv[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const float z = v[8 * j + q] + bv[8 * j + q];
              hv[q] = __float2bfloat16_rn(z * __fdividef(1.0f, 1.0f + __expf(-z)));
            }
            const int n = n0 + 8 * j;
            *reinterpret_cast<uint4*>(out + (n / 64) * (kRows * 64 * 2) + umma::kmajor_offset(r, n % 64, 64, 2)) =
                *reinterpret_cast<const uint4*>(hv);
          }
        } else {
          float wv[32];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 f = reinterpret_cast<const float4*>(sw4 + n0)[q];
            wv[4 * q] = f.x; wv[4 * q + 1] = f.y; wv[4 * q + 2] = f.z; wv[4 * q + 3] = f.w;
          }
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const float z = v[q] + bv[q];
            const float h = __bfloat162float(__float2bfloat16_rn(z * __fdividef(1.0f, 1.0f + __expf(-z))));
            y = fmaf(h, wv[q], y);
          }
        }
      }
      if (!out) {
        // y = (columns 0..127 part) + (columns 128..255 part) + b4, the same order for every row
        float* yp = ypart + (lt & 1) * 2 * kRows;
        yp[half * kRows + r] = y;
        asm volatile("bar.sync 1, %0;" ::"n"(kInfEpi) : "memory");
        if (half == 0 && row < g.nrows) g.y[row] = ok ? (yp[r] + yp[kRows + r]) + g.b4[0] : nan;
      }
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
  float *xs, *ts;         // a sampled training batch: inputs [n][24] and targets [n]
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
  w.xs = (float*)take((size_t)ldt * kNin * 4);
  w.ts = (float*)take((size_t)ldt * 4);
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
  output_grad_kernel<<<kWidth + 2, 256, 0, st>>>(n, w.dy, w.hT[kDepth - 1], w.ldt, w.y, t, net->g + L.off_w4,
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
    colsum_kernel<<<kWidth, 256, 0, st>>>(kWidth, n, w.dzT[cur], w.ldt, net->g + L.off_b[l]);
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
  // zero the padded batch columns [n, ldt) of the transposed buffers (they enter the batch
  // contractions); every other element the step reads is written first
  if (w.ldt > n) {
    const size_t pitch = (size_t)w.ldt * 2, width = (size_t)(w.ldt - n) * 2;
    auto pad = [&](__nv_bfloat16* buf, int rows) {
      return cudaMemset2DAsync(buf + n, pitch, 0, width, rows, st) == cudaSuccess;
    };
    bool okz = pad(w.xT, kK0);
    for (int l = 0; l < kDepth; ++l) okz = okz && pad(w.hT[l], kWidth);
    for (int j = 0; j < 2; ++j) okz = okz && pad(w.dzT[j], kWidth);
    if (!okz) return MGX_ERR_CUDA;
  }
  int rc = forward(net, n, x, w, st, true);
  if (rc != MGX_OK) return rc;
  output_backward_kernel<<<dim3((n + 31) / 32, kWidth / 32), dim3(32, 8), 0, st>>>(
      n, w.y, t, net->p + net->L.off_w4, w.z[kDepth - 1], w.dy, w.dz[0], w.dzT[0], w.ldt);
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

int mgx_mlp_gradients_sampled(mgx_mlp* net, int ntotal, const float* x, const float* t, int batch, uint64_t seed,
                              uint64_t step, float* grad, float* loss, void* ws, size_t wsb, void* stream) {
  if (!net || ntotal <= 0 || batch <= 0 || batch > (1 << 24) || !x || !t) return MGX_ERR_INVALID_ARGUMENT;
  MlpWs w = ws_layout((char*)ws, batch);
  if (!ws || wsb < w.bytes) return MGX_ERR_WORKSPACE_TOO_SMALL;
  sample_rows_kernel<<<(batch + 255) / 256, 256, 0, (cudaStream_t)stream>>>(batch, ntotal, x, t, seed, (uint32_t)step,
                                                                             w.xs, w.ts);
  if (cudaGetLastError() != cudaSuccess) return MGX_ERR_CUDA;
  return mgx_mlp_gradients(net, batch, w.xs, w.ts, grad, loss, ws, wsb, stream);
}

int mgx_mlp_train_step_sampled(mgx_mlp* net, int ntotal, const float* x, const float* t, int batch, uint64_t seed,
                               uint64_t step, float lr, float* loss, void* ws, size_t wsb, void* stream) {
  const int rc = mgx_mlp_gradients_sampled(net, ntotal, x, t, batch, seed, step, nullptr, loss, ws, wsb, stream);
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
