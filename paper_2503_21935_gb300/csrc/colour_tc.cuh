// Tensor-core colour sum (modes MGX_MIXED_TF32 and MGX_MIXED_BF16X3), the one dense contraction of
// the path, fused into the thread-per-event amplitude kernel.
//
// After the 128 threads of a block have run the op table for their 128 events, the jamps of one good
// helicity h form a real matrix X_h = [128 events x ncol] per part (Re, Im).  With the colour matrix
// scaled to integers, Cs = den C, Y = X_h Cs is one tcgen05.mma tile (M = 128 rows, N = ncol padded
// to 16, f32 accumulation in tensor memory) and |M_h|^2 = (x_Re . y_Re + x_Im . y_Im) / den, the dot
// taken by each thread with its own row.  Both operands are split into sums of low-precision parts
// and the partial products accumulate into the same tile:
//   tf32:   x = x0 + x1 (two tf32 terms, ~22 bits of the float32 jamp); Cs exact in tf32 (one part);
//           products x0 Cs + x1 Cs.
//   bf16x3: x = x0 + x1 + x2 (three bf16 terms, ~24 bits), Cs = C0 + C1 (two bf16 terms, exact for
//           integers below 2^16); products x_i C_j with i + j < 3 (the dropped terms lie below 2^-24
//           relative).
// The contraction runs over K = ncol in chunks of at most 32 columns (one shared-memory stage each),
// so a process with many flows needs no more shared memory than one with few.  One thread issues the
// MMAs; tcgen05.commit arrives on an mbarrier that every thread waits on, with a time limit: a wait
// that runs out makes the call return false (the kernel then marks the block's events NaN, counts the
// error and stops using the tensor cores).
#pragma once
#include <cuda_bf16.h>

#include "umma.cuh"

namespace mgx {

constexpr int kTcRows = 128;   // events per tile = threads per block of the fused kernel
constexpr int kTcKc = 32;      // contraction columns per shared-memory stage

struct TcTf32 {
  static constexpr uint32_t kFmt = umma::FMT_TF32;
  static constexpr int kElem = 4, kKStep = 8, kAParts = 2, kBParts = 1;
  __device__ static void split(float x, unsigned char* const dst[], uint32_t off) {
    const float hi = umma::to_tf32(x);
    *reinterpret_cast<float*>(dst[0] + off) = hi;
    *reinterpret_cast<float*>(dst[1] + off) = umma::to_tf32(x - hi);
  }
  __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    umma::mma_tf32(d, a, b, id, acc);
  }
  // four consecutive columns of a row -> one 16-byte piece per part, and back (the sum of the parts)
  __device__ static void split_piece(const float* x, uint4* out) {
    float hi[4], lo[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      hi[q] = umma::to_tf32(x[q]);
      lo[q] = umma::to_tf32(x[q] - hi[q]);
    }
    out[0] = *reinterpret_cast<const uint4*>(hi);
    out[1] = *reinterpret_cast<const uint4*>(lo);
  }
  __device__ static void join_piece(const uint4* in, float* x) {
    const float* hi = reinterpret_cast<const float*>(&in[0]);
    const float* lo = reinterpret_cast<const float*>(&in[1]);
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = hi[q] + lo[q];
  }
};

struct TcBf16x3 {
  static constexpr uint32_t kFmt = umma::FMT_BF16;
  static constexpr int kElem = 2, kKStep = 16, kAParts = 3, kBParts = 2;
  __device__ static void split(float x, unsigned char* const dst[], uint32_t off) {
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
  // eight consecutive columns of a row -> one 16-byte piece per part, and back (the sum of the parts)
  __device__ static void split_piece(const float* x, uint4* out) {
    __align__(16) __nv_bfloat16 p0[8], p1[8], p2[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      p0[q] = __float2bfloat16_rn(x[q]);
      const float r1 = x[q] - __bfloat162float(p0[q]);
      p1[q] = __float2bfloat16_rn(r1);
      p2[q] = __float2bfloat16_rn(r1 - __bfloat162float(p1[q]));
    }
    out[0] = *reinterpret_cast<const uint4*>(p0);
    out[1] = *reinterpret_cast<const uint4*>(p1);
    out[2] = *reinterpret_cast<const uint4*>(p2);
  }
  __device__ static void join_piece(const uint4* in, float* x) {
    const __nv_bfloat16* p0 = reinterpret_cast<const __nv_bfloat16*>(&in[0]);
    const __nv_bfloat16* p1 = reinterpret_cast<const __nv_bfloat16*>(&in[1]);
    const __nv_bfloat16* p2 = reinterpret_cast<const __nv_bfloat16*>(&in[2]);
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = (__bfloat162float(p0[q]) + __bfloat162float(p1[q])) + __bfloat162float(p2[q]);
  }
};

// Colour matrix and launch constants of the fused colour sum (kernel parameter, by value).
struct TcArgs {
  const unsigned char* bchunks;  // integer-scaled colour matrix: per K chunk c, kBParts canonical
                                 // K-major tiles [npad][kc_c] (kc_c = min(32, kpad - 32 c)), contiguous
  int ncol, npad, kpad, nchunk;  // kpad: ncol rounded up to the k-step; nchunk = ceil(kpad / 32)
  uint32_t tcols;                // tensor-memory columns held by each block (power of 2, >= npad)
  double inv_den;                // 1 / den
  int* status;                   // device error counter (one increment per block whose wait ran out)
  int skip_mma;                  // test hook: issue no MMA, so that the waits run out
  unsigned long long wait_ns;    // time limit of one mbarrier wait
};

// shared-memory bytes of the colour-sum stage: A parts (128 x kc) and B parts (npad x kc) of one chunk,
// or, when the contraction is one chunk, the A parts of both Re and Im
template <class F>
__host__ __device__ inline size_t tc_stage_bytes(int kpad, int npad) {
  if (kpad <= kTcKc)   // one stage: Re and Im parts of the whole row (paired rounds) and the colour matrix
    return (size_t)2 * F::kAParts * kTcRows * kpad * F::kElem + (size_t)F::kBParts * npad * kpad * F::kElem;
  const int kc = kTcKc;
  return (size_t)F::kAParts * kTcRows * kc * F::kElem + (size_t)F::kBParts * npad * kc * F::kElem;
}

// The colour sums when the contraction is one stage (kpad <= 32, i.e. ncol <= 32): one round per
// helicity.  The colour matrix is copied into shared memory once per call; each thread stages its Re
// and Im rows together as 16-byte pieces per part; one thread issues both MMA groups, Re into
// tensor-memory columns [0, npad) and Im into [npad, 2 npad), under one commit; after the bounded
// wait each thread dots its two accumulator rows with its row rebuilt from the staged parts (the
// operand the MMAs used), so no jamp is held in registers across the wait.
template <class F, class JW>
__device__ bool tc_colour_sums_paired(const KParams& P, const TcArgs& A, const JW& W, bool valid, int64_t e,
                                      double scale, double* __restrict__ mh_out, unsigned char* stage,
                                      uint64_t* mbar, uint32_t tmem, uint32_t& phase) {
  constexpr int kPer = 16 / F::kElem;   // columns per 16-byte piece: 4 tf32, 8 bf16
  const int t = threadIdx.x, warp = t >> 5;
  const int kc = A.kpad, ncol = A.ncol, npad = A.npad, npiece = kc / kPer;
  const uint32_t a_bytes = (uint32_t)(kTcRows * kc * F::kElem);
  const uint32_t sbo = (uint32_t)(kc * F::kElem / 16) * 128;
  unsigned char* b = stage + 2 * F::kAParts * a_bytes;
  {
    const int nv = F::kBParts * npad * kc * F::kElem / 16;
    const uint4* src = reinterpret_cast<const uint4*>(A.bchunks);
    for (int i = t; i < nv; i += kTcRows) reinterpret_cast<uint4*>(b)[i] = __ldg(src + i);
  }
  // piece j of part p of row t (ri = 0: Re, 1: Im) in the canonical K-major layout
  unsigned char* const row = stage + (t / 8) * sbo + (t % 8) * 16;
  auto piece = [&](int ri, int p, int j) { return reinterpret_cast<uint4*>(row + (ri * F::kAParts + p) * a_bytes + j * 128); };
  const uint32_t id = umma::idesc(F::kFmt, kTcRows, (uint32_t)npad);
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  for (int ih = 0; ih < P.ngood; ++ih) {
    const int jb = P.jamp_off + 2 * ncol * ih;
    for (int j = 0; j < npiece; ++j) {
      double v[2 * kPer];   // (Re, Im) of kPer columns, every load issued before the conversions
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int k = j * kPer + q;
        const bool in = valid && k < ncol;
        v[2 * q] = in ? W[jb + 2 * k] : 0.0;
        v[2 * q + 1] = in ? W[jb + 2 * k + 1] : 0.0;
      }
#pragma unroll
      for (int ri = 0; ri < 2; ++ri) {
        float x[kPer];
#pragma unroll
        for (int q = 0; q < kPer; ++q) x[q] = __double2float_rn(v[2 * q + ri]);
        uint4 pc[F::kAParts];
        F::split_piece(x, pc);
#pragma unroll
        for (int p = 0; p < F::kAParts; ++p) *piece(ri, p, j) = pc[p];
      }
    }
    umma::fence_proxy_async_smem();
    umma::fence_before_sync();
    __syncthreads();
    if (t == 0) {
      umma::fence_after_sync();
      if (!A.skip_mma) {
        const uint32_t b_part = (uint32_t)(npad * kc * F::kElem);
        for (int ri = 0; ri < 2; ++ri) {
          bool first = true;
          for (int pa = 0; pa < F::kAParts; ++pa)
            for (int pb = 0; pb < F::kBParts && pa + pb < F::kAParts; ++pb) {
              const uint32_t sa = umma::smem_u32(stage + (ri * F::kAParts + pa) * a_bytes);
              const uint32_t sb = umma::smem_u32(b) + pb * b_part;
              for (int ks = 0; ks < kc / F::kKStep; ++ks) {
                F::mma(tmem + (uint32_t)(ri * npad), umma::smem_desc(sa + ks * 256, 128, sbo),
                       umma::smem_desc(sb + ks * 256, 128, sbo), id, first ? 0u : 1u);
                first = false;
              }
            }
        }
        umma::mma_commit(mbar);
      }
    }
    const bool done = umma::mbar_wait(mbar, phase, A.wait_ns);
    phase ^= 1;
    if (!__syncthreads_and(done)) return false;
    umma::fence_after_sync();
    float acc = 0.0f;
#pragma unroll 1
    for (int ri = 0; ri < 2; ++ri) {
#pragma unroll 1
      for (int n0 = 0; n0 < npad; n0 += 16) {
        float y[16];
        umma::tmem_ld16(tmem + lane_base + (uint32_t)(ri * npad + n0), y);
        umma::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16 / kPer; ++j) {
          const int jj = n0 / kPer + j;
          if (jj < npiece) {   // columns kc .. npad - 1 of Y are zero and have no staged x
            uint4 pc[F::kAParts];
#pragma unroll
            for (int p = 0; p < F::kAParts; ++p) pc[p] = *piece(ri, p, jj);
            float x[kPer];
            F::join_piece(pc, x);
#pragma unroll
            for (int q = 0; q < kPer; ++q) acc = fmaf(x[q], y[j * kPer + q], acc);
          }
        }
      }
    }
    umma::fence_before_sync();   // tensor-memory reads done before the next round's MMAs
    if (valid) {
      const double mh = scale * ((double)acc * A.inv_den);
      W[P.mh_off + ih] = mh;
      if (mh_out) mh_out[e * P.ngood + ih] = mh;
    }
  }
  return true;
}

// Colour sums of every good helicity for the block's 128 events (thread t owns event e, `valid` when
// e < nevt; the jamps [ngood][ncol][Re, Im] are in the thread's workspace view W).  Writes
// W[mh_off + ih] = scale |M_h|^2 (and mh_out) for valid events.  Every thread of the block must
// call it.  Returns false when an mbarrier wait ran out.
template <class F, class JW>
__device__ bool tc_colour_sums(const KParams& P, const TcArgs& A, const JW& W, bool valid, int64_t e, double scale,
                               double* __restrict__ mh_out, unsigned char* stage, uint64_t* mbar, uint32_t tmem,
                               uint32_t& phase) {
  if (A.nchunk == 1) return tc_colour_sums_paired<F>(P, A, W, valid, e, scale, mh_out, stage, mbar, tmem, phase);
  const int t = threadIdx.x, warp = t >> 5;
  const int kc_max = A.kpad < kTcKc ? A.kpad : kTcKc;
  const size_t a_bytes = (size_t)kTcRows * kc_max * F::kElem;
  unsigned char* a[F::kAParts];
#pragma unroll
  for (int p = 0; p < F::kAParts; ++p) a[p] = stage + p * a_bytes;
  unsigned char* b = stage + F::kAParts * a_bytes;
  const uint32_t id = umma::idesc(F::kFmt, kTcRows, (uint32_t)A.npad);
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const int ncol = A.ncol;
  for (int ih = 0; ih < P.ngood; ++ih) {
    float acc = 0.0f;
#pragma unroll 1
    for (int part = 0; part < 2; ++part) {
      const int jb = P.jamp_off + 2 * ncol * ih + part;
      size_t boff = 0;
      float xv[kTcKc];   // the last staged chunk of this thread's row (all of it for ncol <= 32)
      for (int c = 0; c < A.nchunk; ++c) {
        const int k0 = c * kTcKc;
        const int kc = A.kpad - k0 < kTcKc ? A.kpad - k0 : kTcKc;
        const size_t bbytes = (size_t)F::kBParts * A.npad * kc * F::kElem;
        // the colour matrix's chunk (already in canonical layout; at most 16 KB = 8 pieces a thread)
        {
          const uint4* src = reinterpret_cast<const uint4*>(A.bchunks + boff);
          uint4* dst = reinterpret_cast<uint4*>(b);
          const int nv = (int)(bbytes / 16);
          for (int q0 = 0; q0 < 8; q0 += 4) {
            uint4 v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (t + (q0 + q) * kTcRows < nv) v[q] = __ldg(src + t + (q0 + q) * kTcRows);
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (t + (q0 + q) * kTcRows < nv) dst[t + (q0 + q) * kTcRows] = v[q];
          }
        }
        // this thread's row of the chunk, rounded to float32: every load issued before any store, so
        // their latencies overlap; then split into parts
#pragma unroll
        for (int k = 0; k < kTcKc; ++k) {
          const int kk = k0 + k;
          xv[k] = (valid && k < kc && kk < ncol) ? __double2float_rn(W[jb + 2 * kk]) : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < kTcKc; ++k)
          if (k < kc) F::split(xv[k], a, umma::kmajor_offset((uint32_t)t, (uint32_t)k, (uint32_t)kc, F::kElem));
        umma::fence_proxy_async_smem();
        umma::fence_before_sync();
        __syncthreads();
        if (t == 0) {
          umma::fence_after_sync();
          if (!A.skip_mma) {
            const uint32_t sbo = (uint32_t)(kc * F::kElem / 16) * 128;
            const uint32_t b_part = (uint32_t)((size_t)A.npad * kc * F::kElem);
            bool first = c == 0;
            for (int pa = 0; pa < F::kAParts; ++pa)
              for (int pb = 0; pb < F::kBParts && pa + pb < F::kAParts; ++pb) {
                const uint32_t sa = umma::smem_u32(a[pa]), sb = umma::smem_u32(b) + pb * b_part;
                for (int ks = 0; ks < kc / F::kKStep; ++ks) {
                  F::mma(tmem, umma::smem_desc(sa + ks * 256, 128, sbo), umma::smem_desc(sb + ks * 256, 128, sbo), id,
                         first ? 0u : 1u);
                  first = false;
                }
              }
            umma::mma_commit(mbar);
          }
        }
        const bool done = umma::mbar_wait(mbar, phase, A.wait_ns);
        phase ^= 1;
        if (!__syncthreads_and(done)) return false;
        umma::fence_after_sync();
        boff += bbytes;
      }
      // epilogue: this thread's row of Y (tensor-memory lane t), dotted with its float32 jamps: those
      // still in registers when the contraction was one chunk (npad <= 32), else reloaded 16 at a time
      // (loads issued together)
      if (A.nchunk == 1) {
#pragma unroll
        for (int n0 = 0; n0 < kTcKc; n0 += 16) {
          if (n0 < A.npad) {
            float y[16];
            umma::tmem_ld16(tmem + lane_base + (uint32_t)n0, y);
            umma::tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 16; ++q)
              if (n0 + q < ncol) acc = fmaf(xv[n0 + q], y[q], acc);
          }
        }
      } else {
        for (int n0 = 0; n0 < A.npad; n0 += 16) {
          float xe[16];
#pragma unroll
          for (int q = 0; q < 16; ++q)
            xe[q] = (valid && n0 + q < ncol) ? __double2float_rn(W[jb + 2 * (n0 + q)]) : 0.0f;
          float y[16];
          umma::tmem_ld16(tmem + lane_base + (uint32_t)n0, y);
          umma::tmem_wait_ld();
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (n0 + q < ncol) acc = fmaf(xe[q], y[q], acc);
        }
      }
      umma::fence_before_sync();   // tensor-memory reads done before the next round's MMAs
    }
    if (valid) {
      const double mh = scale * ((double)acc * A.inv_den);
      W[P.mh_off + ih] = mh;
      if (mh_out) mh_out[e * P.ngood + ih] = mh;
    }
  }
  return true;
}

}  // namespace mgx
