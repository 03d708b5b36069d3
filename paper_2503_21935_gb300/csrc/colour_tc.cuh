// Tensor-core colour sum (mode MGX_MIXED_TF32), the one dense contraction of the path.
//
// The jamps of a batch form a real matrix X with one row per (event, good helicity, Re/Im):
// row r = 2 (e ngood + ih) + part, K = ncol.  With the colour matrix scaled to integers,
// Cs = den C (exact in tf32), Y = X Cs is one tcgen05.mma tile of M = 128 rows per k-step
// (kind::tf32, f32 accumulate in tensor memory), X split as X_hi + X_lo (two tf32 terms, so the
// product keeps ~22 bits of X), and |M_h|^2 = (x_Re . y_Re + x_Im . y_Im) / den.
#pragma once
#include "umma.cuh"

namespace mgx {

constexpr int kTcRows = 128;

// shared memory: A_hi, A_lo (128 x kpad f32, canonical K-major), B (npad x kpad), mbarrier, TMEM slot
__host__ __device__ inline size_t colour_tc_smem(int kpad, int npad) {
  return (size_t)2 * kTcRows * kpad * 4 + (size_t)npad * kpad * 4 + 64;
}

__global__ void __launch_bounds__(kTcRows)
    colour_tc_kernel(const double* __restrict__ jamps, int64_t nrows, int ncol, int kpad, int npad,
                     uint32_t tmem_cols, const float* __restrict__ bcanon, double inv_den,
                     double* __restrict__ mh, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* a_hi = smem_raw;
  unsigned char* a_lo = a_hi + (size_t)kTcRows * kpad * 4;
  unsigned char* b = a_lo + (size_t)kTcRows * kpad * 4;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(b + (size_t)npad * kpad * 4);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  // B tile (already in canonical layout) into shared memory
  const float* bsrc = bcanon;
  float* bdst = reinterpret_cast<float*>(b);
  for (int i = tid; i < npad * kpad; i += kTcRows) bdst[i] = __ldg(bsrc + i);
  if (tid == 0) umma::mbar_init(mbar, 1);
  if (warp == 0) umma::tmem_alloc(tslot, tmem_cols);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t sbo = (uint32_t)(kpad / 4) * 128;
  const uint32_t id = umma::idesc(umma::FMT_TF32, kTcRows, (uint32_t)npad);
  const uint32_t sa_hi = umma::smem_u32(a_hi), sa_lo = umma::smem_u32(a_lo), sb = umma::smem_u32(b);
  uint32_t phase = 0;
  bool ok = true;
  for (int64_t tile = blockIdx.x; tile * kTcRows < nrows; tile += gridDim.x) {
    const int64_t r = tile * kTcRows + tid;
    const bool valid = r < nrows;
    const double* xr = jamps + (r >> 1) * 2 * ncol + (r & 1);
    for (int k = 0; k < kpad; ++k) {
      const float x = (valid && k < ncol) ? (float)__ldg(xr + 2 * k) : 0.0f;
      const float hi = umma::to_tf32(x);
      const float lo = umma::to_tf32(x - hi);
      const uint32_t off = umma::kmajor_offset((uint32_t)tid, (uint32_t)k, (uint32_t)kpad, 4);
      *reinterpret_cast<float*>(a_hi + off) = hi;
      *reinterpret_cast<float*>(a_lo + off) = lo;
    }
    umma::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      umma::fence_after_sync();
      for (int ks = 0; ks < kpad / 8; ++ks)
        umma::mma_tf32(tmem, umma::smem_desc(sa_hi + ks * 256, 128, sbo), umma::smem_desc(sb + ks * 256, 128, sbo), id,
                       ks > 0);
      for (int ks = 0; ks < kpad / 8; ++ks)
        umma::mma_tf32(tmem, umma::smem_desc(sa_lo + ks * 256, 128, sbo), umma::smem_desc(sb + ks * 256, 128, sbo), id,
                       1);
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
        if (valid && k < ncol) acc = fmaf((float)__ldg(xr + 2 * k), y[j], acc);
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
