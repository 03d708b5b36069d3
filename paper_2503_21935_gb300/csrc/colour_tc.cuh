// Tensor-core colour sum (modes MGX_MIXED_TF32 and MGX_MIXED_BF16X3), the one dense
// contraction of the path.
//
// The jamps of a batch (rounded to float32) form a real matrix X with one row per (event, good
// helicity, Re/Im):
// row r = 2 (e ngood + ih) + part, K = ncol.  With the colour matrix scaled to integers,
// Cs = den C, Y = X Cs is a tcgen05.mma tile of M = 128 rows (f32 accumulate in tensor memory)
// and |M_h|^2 = (x_Re . y_Re + x_Im . y_Im) / den.  Both operands are split into sums of
// low-precision parts and the partial products are accumulated into the same tile:
//   tf32:   X = X0 + X1 (two tf32 terms, ~22 bits of X); Cs exact in tf32 (one part);
//           products X0 Cs + X1 Cs.
//   bf16x3: X = X0 + X1 + X2 (three bf16 terms, ~24 bits), Cs = C0 + C1 (two bf16 terms, exact
//           for integers below 2^16); products X_i C_j with i + j < 3 (the dropped X2 C1 and
//           X1 C1 ... terms lie below 2^-24 relative).
#pragma once
#include <cuda_bf16.h>

#include "umma.cuh"

namespace mgx {

constexpr int kTcRows = 128;

struct TcTf32 {
  static constexpr uint32_t kFmt = umma::FMT_TF32;
  static constexpr int kElem = 4, kKStep = 8, kAParts = 2, kBParts = 1;
  __device__ static void split(float x, unsigned char* dst[], uint32_t off) {
    const float hi = umma::to_tf32(x);
    *reinterpret_cast<float*>(dst[0] + off) = hi;
    *reinterpret_cast<float*>(dst[1] + off) = umma::to_tf32(x - hi);
  }
  __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    umma::mma_tf32(d, a, b, id, acc);
  }
};

struct TcBf16x3 {
  static constexpr uint32_t kFmt = umma::FMT_BF16;
  static constexpr int kElem = 2, kKStep = 16, kAParts = 3, kBParts = 2;
  __device__ static void split(float x, unsigned char* dst[], uint32_t off) {
    const __nv_bfloat16 p0 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(p0);           // exact
    const __nv_bfloat16 p1 = __float2bfloat16_rn(r1);
    const __nv_bfloat16 p2 = __float2bfloat16_rn(r1 - __bfloat162float(p1));
    *reinterpret_cast<__nv_bfloat16*>(dst[0] + off) = p0;
    *reinterpret_cast<__nv_bfloat16*>(dst[1] + off) = p1;
    *reinterpret_cast<__nv_bfloat16*>(dst[2] + off) = p2;
  }
  __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    umma::mma_f16(d, a, b, id, acc);   // kind::f16 with A and B both bf16
  }
};

// shared memory: A parts (128 x kpad each, canonical K-major), B parts (npad x kpad each),
// mbarrier, TMEM slot
template <class F>
__host__ __device__ inline size_t colour_tc_smem(int kpad, int npad) {
  return (size_t)F::kAParts * kTcRows * kpad * F::kElem + (size_t)F::kBParts * npad * kpad * F::kElem + 64;
}

template <class F>
__global__ void __launch_bounds__(kTcRows)
    colour_tc_kernel(const float* __restrict__ jamps, int64_t nrows, int ncol, int kpad, int npad,
                     uint32_t tmem_cols, const unsigned char* __restrict__ bcanon, double inv_den,
                     double* __restrict__ mh, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const size_t a_bytes = (size_t)kTcRows * kpad * F::kElem, b_bytes = (size_t)npad * kpad * F::kElem;
  unsigned char* a[F::kAParts];
#pragma unroll
  for (int p = 0; p < F::kAParts; ++p) a[p] = smem_raw + p * a_bytes;
  unsigned char* b = smem_raw + F::kAParts * a_bytes;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(b + F::kBParts * b_bytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  // B parts (already in canonical layout) into shared memory
  {
    const uint4* src = reinterpret_cast<const uint4*>(bcanon);
    uint4* dst = reinterpret_cast<uint4*>(b);
    for (int i = tid; i < (int)(F::kBParts * b_bytes / 16); i += kTcRows) dst[i] = __ldg(src + i);
  }
  if (tid == 0) umma::mbar_init(mbar, 1);
  if (warp == 0) umma::tmem_alloc(tslot, tmem_cols);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t sbo = (uint32_t)(kpad * F::kElem / 16) * 128;
  const uint32_t id = umma::idesc(F::kFmt, kTcRows, (uint32_t)npad);
  const uint32_t sb = umma::smem_u32(b);
  uint32_t phase = 0;
  bool ok = true;
  for (int64_t tile = blockIdx.x; tile * kTcRows < nrows; tile += gridDim.x) {
    const int64_t r = tile * kTcRows + tid;
    const bool valid = r < nrows;
    const float* xr = jamps + (r >> 1) * 2 * ncol + (r & 1);
    for (int k = 0; k < kpad; ++k) {
      const float x = (valid && k < ncol) ? __ldg(xr + 2 * k) : 0.0f;
      F::split(x, a, umma::kmajor_offset((uint32_t)tid, (uint32_t)k, (uint32_t)kpad, F::kElem));
    }
    umma::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      umma::fence_after_sync();
      bool first = true;
      for (int pa = 0; pa < F::kAParts; ++pa)
        for (int pb = 0; pb < F::kBParts && pa + pb < F::kAParts; ++pb) {
          const uint32_t sa = umma::smem_u32(a[pa]), sbp = sb + (uint32_t)(pb * b_bytes);
          for (int ks = 0; ks < kpad / F::kKStep; ++ks) {
            F::mma(tmem, umma::smem_desc(sa + ks * 256, 128, sbo), umma::smem_desc(sbp + ks * 256, 128, sbo), id,
                   first ? 0u : 1u);
            first = false;
          }
        }
      umma::mma_commit(mbar);
    }
    const bool done = umma::mbar_wait(mbar, phase);
    phase ^= 1;
    if (!__syncthreads_and(done)) {
      ok = false;
      break;
    }
    umma::fence_after_sync();
    // epilogue: this thread's row of Y (TMEM lane = row), dotted with its row of X
    float acc = 0.0f;
    for (int c0 = 0; c0 < npad; c0 += 8) {
      float y[8];
      umma::tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, y);
      umma::tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k = c0 + j;
        if (valid && k < ncol) acc = fmaf(__ldg(xr + 2 * k), y[j], acc);
      }
    }
    const float other = __shfl_xor_sync(0xffffffffu, acc, 1);
    if (valid && (r & 1) == 0) mh[r >> 1] = (double)(acc + other) * inv_den;
    umma::fence_before_sync();
    __syncthreads();
  }
  if (!ok) {
    if (tid == 0 && err) atomicExch(err, 1);
    umma::mbar_wait(mbar, phase ^ 1);   // bounded second wait for the MMAs still in flight
  }
  __syncthreads();
  umma::fence_after_sync();
  if (warp == 0) {
    umma::tmem_dealloc(tmem, tmem_cols);
    umma::tmem_relinquish();
  }
}

}  // namespace mgx
