// mgx: C-ABI library for batched tree-level |M|^2 on one GB300 (sm_103a).
// Host API, helicity filter and the launch of the event-parallel kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cctype>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "mgx.h"
#include "mgx_ops.cuh"
#include "colour_tc.cuh"

namespace {

struct mgx_program_desc {
  const char* name;
  int npar, nin, root, nops;
  const int32_t* ops;
  int nflows;
  const int32_t* flows;
  int nterms_tab;
  const int32_t* terms;  // 8 ints per diagram term of the AMP groups
  int ncol;
  const double* colour;
  int ncoupl;
  const double* coupl;   // (boson id, Q, T3) per entry
  int nmass;
  const int32_t* mass;   // (mass param, width param) per entry
  const int32_t* extmass;
  int ws_doubles, ndiag, nterm, avg_den;
  int gs_power;          // power of g_s of every amplitude (vertices are evaluated with g_s = 1)
  int col_den;           // common denominator of the colour matrix
  int jamp_zero;         // some flow is never updated: zero the jamps first
  int counts[17];        // variants: ffv_f, ffv_fb, ffv_v, vvv, vvvv, bil, rbil; current ops; amp terms, flows,
                         // groups, runs (terms sharing one bilinear within a group); sum-current
                         // 4-vector adds (variants x (summands - 1)); VVV header child dots; VVVV
                         // header pair dots; header slash blocks (vector variants of f f V vertices);
                         // those of them scaled by a fermion propagator prefactor
  struct {
    int nops;
    const int32_t* ops;
    int nflows;
    const int32_t* flows;
    int nterms;
    const int32_t* terms;
    int nitems;
    const int32_t* items;  // (op row << 8) | variant, variant 255 = header
    int nsteps;
    const int32_t* steps;  // (kind 0 = wave of items / 1 = amplitude rows, start, count)
    int store;             // doubles of shared memory for one event's currents
    int chunk;             // terms per chunk
  } cta;
  struct {
    int nparts;            // parts of the diagram split into (at most) 2, 4, 8
    const int32_t* ops;    // op positions of every part, in program order, parts concatenated
    const int32_t* start;  // [nparts + 1] offsets into ops
  } split[3];
};

#include "generated/programs.inc"

}  // namespace

using namespace mgx;

// ------------------------------------------------------------------ kernel
namespace {

constexpr int kThreads = 128;        // thread-per-event kernel
constexpr int kMaxColCta = 32;       // jamps per helicity held by one thread in the CTA kernel
constexpr int kMaxColFp32 = 120;     // colour flows of the largest built-in process

// g_s^(2p) = (4 pi alpha_s)^p: every amplitude carries g_s^p, the vertices use g_s = 1
__device__ __forceinline__ double coupling_scale(const KParams& P, double alpha_s) {
  const double g2 = 4.0 * M_PI * alpha_s;
  double s = 1.0;
  for (int k = 0; k < P.gs_power; ++k) s *= g2;
  return s;
}

// |M_h|^2 = J^dagger C J with C given as C_ii on the diagonal and 2 C_ij above it.
template <class JV>
__device__ __forceinline__ double quad_form(const JV& J, const double* csym, const float* csym_f, int n, int mode) {
  if (mode == MGX_MIXED_FP32) {
    // one float64 -> float32 rounding per jamp component (conversions use the FP64 pipe)
    float jf[2 * kMaxColFp32];
    for (int k = 0; k < 2 * n; ++k) jf[k] = (float)J(k);
    float acc = 0.0f;
    for (int i = 0; i < n; ++i) {
      const float ri = jf[2 * i], ii = jf[2 * i + 1];
      const float* crow = csym_f + i * n;
      float zr = __ldg(crow + i) * ri, zi = __ldg(crow + i) * ii;
      for (int j = i + 1; j < n; ++j) {
        const float c = __ldg(crow + j);
        zr = fmaf(c, jf[2 * j], zr);
        zi = fmaf(c, jf[2 * j + 1], zi);
      }
      acc = fmaf(ri, zr, fmaf(ii, zi, acc));
    }
    return (double)acc;
  }
  double acc = 0.0;
  for (int i = 0; i < n; ++i) {
    const double ri = J(2 * i), ii = J(2 * i + 1);
    const double* crow = csym + i * n;
    double zr = __ldg(crow + i) * ri, zi = __ldg(crow + i) * ii;
    for (int j = i + 1; j < n; ++j) {
      const double c = __ldg(crow + j);
      zr = fma(c, J(2 * j), zr);
      zi = fma(c, J(2 * j + 1), zi);
    }
    acc = fma(ri, zr, fma(ii, zi, acc));
  }
  return acc;
}

// |M_h|^2 / g_s^(2p) of one helicity from jamps J(k) of real type R: float64 (or the mixed
// float32 form above), or float32 throughout
template <class R, class JV>
__device__ __forceinline__ double colour_sum(const KParams& P, const JV& J, int n, int mode) {
  if constexpr (std::is_same<R, double>::value) {
    return quad_form(J, P.colsym, P.colsym_f, n, mode);
  } else {
    float acc = 0.0f;
    for (int i = 0; i < n; ++i) {
      const float ri = J(2 * i), ii = J(2 * i + 1);
      const float* crow = P.colsym_f + i * n;
      float zr = __ldg(crow + i) * ri, zi = __ldg(crow + i) * ii;
      for (int j = i + 1; j < n; ++j) {
        const float c = __ldg(crow + j);
        zr = fmaf(c, J(2 * j), zr);
        zi = fmaf(c, J(2 * j + 1), zi);
      }
      acc = fmaf(ri, zr, fmaf(ii, zi, acc));
    }
    return (double)acc;
  }
}

// helicity sum (float64, canonical order), me and the two selections from per-helicity
// weights mh[ngood] and colour weights colw[ncol] (any indexable storage)
template <class A, class B>
__device__ inline void finish_event(const KParams& P, int64_t e, const A& mh, const B& colw, const double* rhel,
                                    const double* rcol, double* me, int32_t* selhel, int32_t* selcol) {
  double tot = 0.0;
  for (int ih = 0; ih < P.ngood; ++ih) tot += mh(ih);
  me[e] = tot * P.avg;
  if (selhel) {
    const double target = rhel[e] * tot;
    double acc = 0.0;
    int sel = P.good[P.ngood - 1];
    for (int ih = 0; ih < P.ngood; ++ih) {
      acc += mh(ih);
      if (acc > target) { sel = P.good[ih]; break; }
    }
    selhel[e] = sel;
  }
  if (selcol) {
    double wt = 0.0;
    for (int i = 0; i < P.ncol; ++i) wt += colw(i);
    const double target = rcol[e] * wt;
    double acc = 0.0;
    int sel = P.ncol - 1;
    for (int i = 0; i < P.ncol; ++i) {
      acc += colw(i);
      if (acc > target) { sel = i; break; }
    }
    selcol[e] = sel;
  }
}

// ---------------------------------------------------------------- thread-per-event kernel
// Each thread owns one event at a time; current variants and jamps live in a per-thread
// global workspace (offset-major so a warp's accesses coalesce).  Used for processes whose
// per-event store does not fit in shared memory.
// The op table of one event, evaluated by one thread into the workspace view W: every current
// variant, then the jamps [ngood][ncol][Re, Im] at W[jamp_off].  Currents and jamps are of real type R.
// kSplit: only the ops list[0 .. nlist) (one part of a diagram split, in program order) into partial
// jamps that start at zero and to which every flow update adds.
template <class R, class H = AllHel, bool kSplit = false>
__device__ inline void eval_amplitudes(const KParams& P, const double* pe, const WST<R>& W, const H& hs = H(),
                                       const int* __restrict__ list = nullptr, int nlist = 0) {
  using T = Real<R>;
  const double gs = 1.0;                                   // g_s^(2p) applied to |M|^2 later
  if (kSplit || P.jamp_zero)
    for (int ih = 0; ih < P.ngood; ++ih) {
      if (!hs.ok(P.good[ih])) continue;                 // only the helicities this thread computes
      for (int i = 0; i < 2 * P.ncol; ++i) W[P.jamp_off + 2 * P.ncol * ih + i] = T::from(0.0);
    }
  const int nloop = kSplit ? nlist : P.nops;
  for (int li = 0; li < nloop; ++li) {
    const int iop = kSplit ? __ldg(list + li) : li;
    const Op o = load_op(P.ops, iop);
    if (o.code == OP_AMP) {
      const int2* fl = P.flows + o.cpl;
      if (o.aux2 == 1) {
        // one term X . Y: the helicities run as (bilinear variant, other variant) pairs so that
        // each bilinear variant is loaded once; the term's phase rotates the product
        const int4 a = __ldg(P.terms + 2 * o.aux);
        const int4 b = __ldg(P.terms + 2 * o.aux + 1);
        for (int ux = 0; ux < hs.count(a.y); ++ux) {
          const int ix = hs.var(ux, a.y);
          cxT<R> X[4];
          W.load4(a.x + 8 * ix, X);
          const int hx = pdep(ix, a.y);
          for (int uy = 0; uy < hs.count(a.w); ++uy) {
            const int iy = hs.var(uy, a.w);
            const int ih = P.hidx[hx | pdep(iy, a.w)];
            if (ih < 0) continue;
            cxT<R> Y[4];
            W.load4(a.z + 8 * iy, Y);
            cxT<R> amp;
            if (b.y == 0) {
              amp = mdot(X, Y);
            } else {
              amp = cmul(X[0], Y[0]);
              amp = cfma(X[1], Y[1], amp);
              amp = cfma(X[2], Y[2], amp);
              amp = cfma(X[3], Y[3], amp);
            }
            amp = rot_phase(b.x, amp);
            const int jb = P.jamp_off + 2 * P.ncol * ih;
            for (int f = 0; f < o.mass; ++f) {
              const int2 q = __ldg(fl + f);
              const int off = jb + 2 * q.x;
              cxT<R> j = rot_phase(q.y & 3, amp);
              if (kSplit || !(q.y & 4)) j = cxT<R>{W[off], W[off + 1]} + j;
              W[off] = j.r;
              W[off + 1] = j.i;
            }
          }
        }
        continue;
      }
      for (int ih = 0; ih < P.ngood; ++ih) {
        if (!hs.ok(P.good[ih])) continue;
        const cxT<R> amp = group_amp<R>(P.terms, o, P.good[ih], W);
        const int jb = P.jamp_off + 2 * P.ncol * ih;
        // phase rotation by sign-bit and swap selects (no branch per flow), then one add each;
        // the first update of a flow in program order (code bit 2) writes
        for (int f = 0; f < o.mass; ++f) {
          const int2 q = __ldg(fl + f);
          const int off = jb + 2 * q.x;
          cxT<R> j = rot_phase(q.y & 3, amp);
          if (kSplit || !(q.y & 4)) j = cxT<R>{W[off], W[off + 1]} + j;
          W[off] = j.r;
          W[off + 1] = j.i;
        }
      }
      continue;
    }
    op_header<R>(P, o, gs, pe, W, hs);
    op_variants<R>(P, o, gs, pe, W, hs);
  }
}

// SIMT colour sums: W[mh_off + ih] = scale |M_h|^2 for every good helicity (float64, the mixed
// float32 form, or float32 throughout)
template <class R>
__device__ inline void simt_colour_sums(const KParams& P, int64_t e, const WST<R>& W, double scale,
                                        double* __restrict__ mh_out, int mode) {
  using T = Real<R>;
  for (int ih = 0; ih < P.ngood; ++ih) {
    const int jb = P.jamp_off + 2 * P.ncol * ih;
    const double mh = scale * colour_sum<R>(P, [&](int k) { return W[jb + k]; }, P.ncol, mode);
    W[P.mh_off + ih] = T::from(mh);
    if (mh_out) mh_out[e * P.ngood + ih] = mh;
  }
}

// colour weights w_s = scale sum_h |J_s(h)|^2 from the jamps, then the helicity sum and the
// selections from W[mh_off ..]
template <class R>
__device__ inline void finish_from_workspace(const KParams& P, int64_t e, const WST<R>& W, double scale,
                                             const double* __restrict__ rhel, const double* __restrict__ rcol,
                                             double* __restrict__ me, int32_t* __restrict__ selhel,
                                             int32_t* __restrict__ selcol, double* __restrict__ colw_out) {
  using T = Real<R>;
  if (selcol || colw_out) {
    for (int i = 0; i < P.ncol; ++i) {
      R w = T::from(0.0);
      for (int ih = 0; ih < P.ngood; ++ih) {
        const int jb = P.jamp_off + 2 * P.ncol * ih + 2 * i;
        w = fma(W[jb], W[jb], fma(W[jb + 1], W[jb + 1], w));
      }
      const double wd = T::to_double(w) * scale;
      W[P.colw_off + i] = T::from(wd);
      if (colw_out) colw_out[e * P.ncol + i] = wd;
    }
  }
  finish_event(P, e, [&](int ih) { return T::to_double(W[P.mh_off + ih]); },
               [&](int i) { return T::to_double(W[P.colw_off + i]); }, rhel, rcol, me, selhel, selcol);
}

// One event, evaluated by one thread: the op table, the colour sum, helicity sum and selections.
template <class R>
__device__ inline void eval_event(const KParams& P, int64_t e, const double* pe, const WST<R>& W,
                                  const double* __restrict__ alphas, const double* __restrict__ rhel,
                                  const double* __restrict__ rcol, double* __restrict__ me,
                                  int32_t* __restrict__ selhel, int32_t* __restrict__ selcol,
                                  double* __restrict__ mh_out, double* __restrict__ colw_out, int mode) {
  eval_amplitudes<R>(P, pe, W);
  const double scale = coupling_scale(P, alphas[e]);
  simt_colour_sums<R>(P, e, W, scale, mh_out, mode);
  finish_from_workspace<R>(P, e, W, scale, rhel, rcol, me, selhel, selcol, colw_out);
}

// stage the momenta of events [base, base + nb) (contiguous [events][npar][4]) through shared memory
__device__ __forceinline__ void stage_momenta(const double* __restrict__ mom, int64_t base, int64_t nb, int npar4,
                                              double* smem) {
  const double2* src = reinterpret_cast<const double2*>(mom + base * npar4);
  double2* dst = reinterpret_cast<double2*>(smem);
  __syncthreads();
  for (int i = threadIdx.x; i < (int)(nb * npar4 / 2); i += blockDim.x) dst[i] = __ldg(src + i);
  __syncthreads();
}

// 4 resident blocks per SM for float64 (128 registers), 8 for float (64 registers): the float
// path is latency-bound on its workspace and gains from the extra warps.  With kSmemWs the
// per-event workspace lives in shared memory after the staged momenta (small processes in
// latency-bound batches, kSmemThreads threads per block, one block per SM).
template <class R, bool kSmemWs>
__global__ void __launch_bounds__(kThreads, kSmemWs ? 1 : (std::is_same<R, float>::value ? 8 : 4))
    me_kernel(const KParams P, int64_t nevt, const double* __restrict__ mom, const double* __restrict__ alphas,
              const double* __restrict__ rhel, const double* __restrict__ rcol, double* __restrict__ me,
              int32_t* __restrict__ selhel, int32_t* __restrict__ selcol, double* __restrict__ mh_out,
              double* __restrict__ colw_out, double* __restrict__ ws, int64_t nthreads, int mode) {
  extern __shared__ double smem[];
  const int npar4 = 4 * P.npar;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const WST<R> W = kSmemWs ? WST<R>{reinterpret_cast<R*>(smem + blockDim.x * npar4) + threadIdx.x, blockDim.x}
                           : WST<R>{reinterpret_cast<R*>(ws) + tid, nthreads};
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nevt; base += nthreads) {
    stage_momenta(mom, base, min((int64_t)blockDim.x, nevt - base), npar4, smem);
    const int64_t e = base + threadIdx.x;
    if (e >= nevt) continue;
    eval_event<R>(P, e, smem + threadIdx.x * npar4, W, alphas, rhel, rcol, me, selhel, selcol, mh_out, colw_out,
                  mode);
  }
}

// The thread-per-event kernel with the colour sum on the tensor cores (float64 amplitudes): after the
// block's 128 threads have run the op table for their events, the block forms every helicity's
// colour sum with tcgen05.mma (tc_colour_sums), then each thread finishes its event.  The colour-sum
// stage reuses the shared memory of the staged momenta; the mbarrier and the tensor-memory address
// sit after it.  If a tensor-core wait runs out, the block counts the error, marks its events NaN
// (me) and -1 (selections) from then on, and stops using the tensor cores.
template <class F>
__global__ void __launch_bounds__(kThreads, 4)
    me_tc_kernel(const KParams P, const TcArgs A, int64_t nevt, const double* __restrict__ mom,
                 const double* __restrict__ alphas, const double* __restrict__ rhel, const double* __restrict__ rcol,
                 double* __restrict__ me, int32_t* __restrict__ selhel, int32_t* __restrict__ selcol,
                 double* __restrict__ mh_out, double* __restrict__ colw_out, double* __restrict__ ws,
                 int64_t nthreads, size_t bar_off) {
  extern __shared__ __align__(1024) double smem[];
  unsigned char* raw = reinterpret_cast<unsigned char*>(smem);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(raw + bar_off);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int npar4 = 4 * P.npar;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const WS W{ws + tid, nthreads};
  if (threadIdx.x == 0) umma::mbar_init(mbar, 1);
  if (threadIdx.x < 32) umma::tmem_alloc_once(tslot, A.tcols);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  // Nothing but the loop position stays live across the op table (the tensor-memory address is read
  // back from shared memory and the mbarrier phase restarts at 0 every pass: a pass completes an even
  // number of phases, two parts per helicity and chunk), so the op table keeps the registers of the
  // plain thread kernel.
  int64_t base = (int64_t)blockIdx.x * blockDim.x;
  bool healthy = true;
  uint32_t fail_phase = 0;
  for (; base < nevt; base += nthreads) {
    const int64_t e = base + threadIdx.x;
    const bool valid = e < nevt;
    stage_momenta(mom, base, min((int64_t)blockDim.x, nevt - base), npar4, smem);
    if (valid) eval_amplitudes<double>(P, smem + threadIdx.x * npar4, W);
    const double scale = valid ? coupling_scale(P, alphas[e]) : 0.0;
    __syncthreads();                      // the staged momenta are dead: the stage reuses them
    uint32_t phase = 0;
    if (!tc_colour_sums<F>(P, A, W, valid, e, scale, mh_out, raw, mbar, *tslot, phase)) {
      healthy = false;
      fail_phase = phase;
      break;
    }
    if (valid) finish_from_workspace<double>(P, e, W, scale, rhel, rcol, me, selhel, selcol, colw_out);
  }
  if (!healthy) {
    if (threadIdx.x == 0 && A.status) atomicAdd(A.status, 1);
    for (; base < nevt; base += nthreads) {   // this pass and every later one: NaN and -1
      const int64_t e = base + threadIdx.x;
      if (e >= nevt) continue;
      me[e] = __longlong_as_double(0x7ff8000000000000ll);
      if (selhel) selhel[e] = -1;
      if (selcol) selcol[e] = -1;
    }
    umma::mbar_wait(mbar, fail_phase ^ 1, A.wait_ns);   // bounded wait for MMAs still in flight
  }
  const uint32_t tmem = *tslot;
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  if (threadIdx.x < 32) {
    umma::tmem_dealloc(tmem, A.tcols);
  }
}

// ---------------------------------------------------------------- helicity-parallel kernel
// For batches too small to fill the thread-per-event grid (Sec. 2: processing different helicity
// combinations of one event in parallel lets far fewer events keep the GPU busy).  The helicities
// of an event are split into G = 2^|fix| groups by their bits on the fixed legs `fix`; item
// (e, g) = thread computes the current variants and amplitudes that group g's helicities use (the
// variants of currents without a fixed leg are computed by every group), their colour sums into
// mh_buf [nevt][ngood] and the group's share of the colour weights into cw_buf [nevt][G][ncol].
// finish_hel_kernel then sums each event's helicities in canonical order and selects.  One launch
// covers every group (a grid dimension rather than one CUDA stream per helicity).
template <class R>
__global__ void __launch_bounds__(kThreads, std::is_same<R, float>::value ? 8 : 4)
    me_hel_kernel(const KParams P, int64_t nevt, int gshift, int fix, const double* __restrict__ mom,
                  const double* __restrict__ alphas, double* __restrict__ mh_buf, double* __restrict__ cw_buf,
                  double* __restrict__ ws, int64_t nthreads, int mode) {
  using T = Real<R>;
  extern __shared__ double smem[];
  const int npar4 = 4 * P.npar;
  const int G = 1 << gshift;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const WST<R> W{reinterpret_cast<R*>(ws) + tid, nthreads};
  // items are numbered group-major over the events padded to whole blocks, so a block (and every
  // warp) runs one group for consecutive events: the same variants, coalesced workspace accesses
  const int64_t npad = (nevt + blockDim.x - 1) / blockDim.x * blockDim.x;
  const int64_t nitems = npad << gshift;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nitems; base += nthreads) {
    const int g = (int)(base / npad);
    const int64_t e0 = base % npad;
    if (e0 >= nevt) continue;                                 // the whole block is padding
    stage_momenta(mom, e0, min((int64_t)blockDim.x, nevt - e0), npar4, smem);
    const int64_t e = e0 + threadIdx.x;
    if (e >= nevt) continue;
    const GroupHel hs{fix, pdep(g, fix)};
    eval_amplitudes<R>(P, smem + threadIdx.x * npar4, W, hs);
    const double scale = coupling_scale(P, alphas[e]);
    for (int ih = 0; ih < P.ngood; ++ih) {
      if (!hs.ok(P.good[ih])) continue;
      const int jb = P.jamp_off + 2 * P.ncol * ih;
      mh_buf[e * P.ngood + ih] = scale * colour_sum<R>(P, [&](int k) { return W[jb + k]; }, P.ncol, mode);
    }
    double* cw = cw_buf + (e * G + g) * P.ncol;
    for (int i = 0; i < P.ncol; ++i) {
      R w = T::from(0.0);
      for (int ih = 0; ih < P.ngood; ++ih) {
        if (!hs.ok(P.good[ih])) continue;
        const int jb = P.jamp_off + 2 * P.ncol * ih + 2 * i;
        w = fma(W[jb], W[jb], fma(W[jb + 1], W[jb + 1], w));
      }
      cw[i] = T::to_double(w) * scale;
    }
  }
}

// helicity sum (canonical order), colour weights (groups summed in group order) and selections
__global__ void __launch_bounds__(kThreads)
    finish_hel_kernel(const KParams P, int64_t nevt, int G, const double* __restrict__ mh_buf,
                      const double* __restrict__ cw_buf, const double* __restrict__ rhel,
                      const double* __restrict__ rcol, double* __restrict__ me, int32_t* __restrict__ selhel,
                      int32_t* __restrict__ selcol, double* __restrict__ mh_out, double* __restrict__ colw_out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nevt) return;
  const double* m = mh_buf + e * P.ngood;
  const double* cw = cw_buf + e * G * P.ncol;
  auto colw = [&](int i) {
    double w = 0.0;
    for (int g = 0; g < G; ++g) w += cw[g * P.ncol + i];
    return w;
  };
  if (mh_out)
    for (int ih = 0; ih < P.ngood; ++ih) mh_out[e * P.ngood + ih] = m[ih];
  if (colw_out)
    for (int i = 0; i < P.ncol; ++i) colw_out[e * P.ncol + i] = colw(i);
  finish_event(P, e, [&](int ih) { return m[ih]; }, colw, rhel, rcol, me, selhel, selcol);
}

// ---------------------------------------------------------------- diagram-split kernels
// The amplitude groups of a process are cut into D parts (process compiler: contiguous segments of
// the program, each with every current op its terms need); item (e, g, d) = one thread runs part d
// of event e restricted to helicity group g (as in the helicity-parallel kernel; one group when
// fix = 0) into zeroed partial jamps and writes them to pj [nevt][D][ngood][ncol][Re, Im].
// split_combine_kernel then sums each (event, helicity)'s D partial jamp vectors, forms the colour
// sum and the helicity's colour-weight terms, and finish_hel_kernel (with one "group" per
// helicity) sums the helicities in canonical order and selects.
template <class R>
__global__ void __launch_bounds__(kThreads, std::is_same<R, float>::value ? 8 : 4)
    me_split_kernel(const KParams P, int64_t nevt, int gshift, int fix, int nparts, const int* __restrict__ part_ops,
                    const int* __restrict__ part_start, const double* __restrict__ mom, R* __restrict__ pj,
                    double* __restrict__ ws, int64_t nthreads) {
  extern __shared__ double smem[];
  const int npar4 = 4 * P.npar;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const WST<R> W{reinterpret_cast<R*>(ws) + tid, nthreads};
  // items are numbered (group, part)-major over the events padded to whole blocks, so a block (and
  // every warp) runs one part's op list for one group over consecutive events: no divergence,
  // coalesced workspace accesses
  const int64_t npad = (nevt + blockDim.x - 1) / blockDim.x * blockDim.x;
  const int64_t nitems = (npad * nparts) << gshift;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nitems; base += nthreads) {
    const int gd = (int)(base / npad);
    const int d = gd % nparts, g = gd / nparts;
    const int64_t e0 = base % npad;
    if (e0 >= nevt) continue;                                 // the whole block is padding
    stage_momenta(mom, e0, min((int64_t)blockDim.x, nevt - e0), npar4, smem);
    const int64_t e = e0 + threadIdx.x;
    if (e >= nevt) continue;
    const GroupHel hs{fix, pdep(g, fix)};
    const int s0 = __ldg(part_start + d), s1 = __ldg(part_start + d + 1);
    eval_amplitudes<R, GroupHel, true>(P, smem + threadIdx.x * npar4, W, hs, part_ops + s0, s1 - s0);
    const int nj = 2 * P.ncol;
    R* out = pj + (e * nparts + d) * (int64_t)P.ngood * nj;
    for (int ih = 0; ih < P.ngood; ++ih) {
      if (!hs.ok(P.good[ih])) continue;
      // 8 loads issued before their stores (a store between loads would serialise their latencies)
      for (int k0 = 0; k0 < nj; k0 += 8) {
        R v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (k0 + q < nj) v[q] = W[P.jamp_off + ih * nj + k0 + q];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (k0 + q < nj) out[ih * nj + k0 + q] = v[q];
      }
    }
  }
}

// one thread per (event, good helicity): J = sum of the D partial jamps, then |M_h|^2 (colour sum of
// the mode) into mh_buf [nevt][ngood] and |J_i|^2 into cwh [nevt][ngood][ncol], both times the
// event's coupling factor
template <class R>
__global__ void __launch_bounds__(kThreads)
    split_combine_kernel(const KParams P, int64_t nevt, int nparts, const R* __restrict__ pj,
                         const double* __restrict__ alphas, double* __restrict__ mh_buf, double* __restrict__ cwh,
                         int mode) {
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= nevt * P.ngood) return;
  const int64_t e = item / P.ngood;
  const int ih = (int)(item % P.ngood);
  const int nj = 2 * P.ncol;
  R J[2 * kMaxColFp32];
  const R* src = pj + (e * nparts * (int64_t)P.ngood + ih) * nj;
  for (int k = 0; k < nj; ++k) J[k] = src[k];
  for (int d = 1; d < nparts; ++d)
    for (int k = 0; k < nj; ++k) J[k] = J[k] + src[(int64_t)d * P.ngood * nj + k];
  const double scale = coupling_scale(P, alphas[e]);
  mh_buf[item] = scale * colour_sum<R>(P, [&](int k) { return J[k]; }, P.ncol, mode);
  for (int i = 0; i < P.ncol; ++i)
    cwh[item * P.ncol + i] = scale * Real<R>::to_double(fma(J[2 * i], J[2 * i], J[2 * i + 1] * J[2 * i + 1]));
}

// ---------------------------------------------------------------- batched multi-process kernel
// One persistent launch over several processes with uneven event counts.  Work items are
// ranges of `events_per_item` events of one process, numbered process after process; CTAs
// take items from a device counter (atomicAdd: no waits), so the load balances across processes.
struct BatchIO {
  int64_t nevt;
  const double* mom;
  const double* alphas;
  const double* rhel;
  const double* rcol;
  double* me;
  int32_t* selhel;
  int32_t* selcol;
};

constexpr int kMaxBatch = 16;

// Everything the batch kernel reads per process, passed by value (about 17 KB of kernel
// parameters): the process parameters then sit in the constant bank like the single-process
// kernel's, instead of being loaded from global memory on every use.
struct BatchParams {
  KParams kp[kMaxBatch];
  BatchIO io[kMaxBatch];
};

struct BatchDesc {
  int nproc, max_npar4;
  int epi[kMaxBatch];    // events per work item, per process
  int64_t item_start[kMaxBatch + 1];
};

// (register budget of 4 resident blocks per SM, as the thread-per-event kernel gets by default:
// occupancy hides the workspace latency better than the few registers more would)
__global__ void __launch_bounds__(kThreads, 4)
    batch_kernel(const __grid_constant__ BatchParams BP, const BatchDesc D,
                 unsigned long long* __restrict__ counter, double* __restrict__ ws, int64_t nthreads, int mode) {
  extern __shared__ double smem[];
  __shared__ long long s_item;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const WS W{ws + tid, nthreads};
  const int64_t nitems = D.item_start[D.nproc];
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= nitems) break;
    int p = 0;
    while (item >= D.item_start[p + 1]) ++p;
    const KParams& P = BP.kp[p];
    const BatchIO& b = BP.io[p];
    const int npar4 = 4 * P.npar;
    const int64_t first = (item - D.item_start[p]) * D.epi[p];
    const int64_t last = min(first + (int64_t)D.epi[p], b.nevt);
    for (int64_t base = first; base < last; base += blockDim.x) {
      stage_momenta(b.mom, base, min((int64_t)blockDim.x, last - base), npar4, smem);
      const int64_t e = base + threadIdx.x;
      if (e < last)
        eval_event<double>(P, e, smem + threadIdx.x * npar4, W, b.alphas, b.rhel, b.rcol, b.me, b.selhel, b.selcol, nullptr,
                   nullptr, mode);
    }
  }
}

// ---------------------------------------------------------------- CTA-per-event kernel
// One CTA evaluates one event at a time with the event's current store in shared memory.
// Current waves: threads take (current, helicity-variant) items; amplitude steps: thread t
// closes every diagram term of the step for good helicity t and keeps that helicity's
// jamps in its own local array; then each thread forms its |M_h|^2.
struct CtaTab {
  const int4* ops;
  const int2* flows;
  const int4* terms;
  const int* items;
  const int3* steps;
  int nsteps, store;
};

constexpr int kCtaThreads = 128;

// Threads are (term lane g, helicity slot hl): hl = t % ngp, g = t / ngp, ngp the good-helicity
// count rounded up to 32.  In an amplitude step lane g closes groups g, g+G, ... for helicity hl;
// lanes > 0 hand their partial jamps to lane 0 through shared memory at the end.
__global__ void __launch_bounds__(kCtaThreads)
    me_cta_kernel(const KParams P, const CtaTab C, int64_t nevt, const double* __restrict__ mom,
                  const double* __restrict__ alphas, const double* __restrict__ rhel,
                  const double* __restrict__ rcol, double* __restrict__ me, int32_t* __restrict__ selhel,
                  int32_t* __restrict__ selcol, double* __restrict__ mh_out, double* __restrict__ colw_out,
                  int mode) {
  constexpr int T = kCtaThreads;
  extern __shared__ double sm[];
  double* store = sm;
  double* pe = sm + C.store;
  const SS W{store};
  const int tid = threadIdx.x;
  const int npar4 = 4 * P.npar;
  const int ngp = P.ngood <= 32 ? 32 : (P.ngood <= 64 ? 64 : 128);
  const int G = T / ngp;
  const int hl = tid % ngp, g = tid / ngp;
  const bool act = hl < P.ngood;
  const int h = act ? P.good[hl] : 0;
  const int ncol = P.ncol;
  for (int64_t e = blockIdx.x; e < nevt; e += gridDim.x) {
    for (int i = tid; i < npar4; i += T) pe[i] = __ldg(mom + e * npar4 + i);
    __syncthreads();
    const double gs = 1.0;                                   // g_s^(2p) applied to |M|^2 below
    const double scale = coupling_scale(P, __ldg(alphas + e));
    double J[2 * kMaxColCta];
#pragma unroll
    for (int i = 0; i < 2 * kMaxColCta; ++i) J[i] = 0.0;
    for (int s = 0; s < C.nsteps; ++s) {
      const int3 st = C.steps[s];
      if (st.x == 0) {
        for (int it = tid; it < st.z; it += T) {
          const int item = __ldg(C.items + st.y + it);
          const Op o = load_op(C.ops, item >> 8);
          const int v = item & 255;
          if (v == 255) op_header<double>(P, o, gs, pe, W);
          else op_variant<double>(P, o, v, gs, pe, W);
        }
      } else if (act) {
        for (int a = st.y + g; a < st.y + st.z; a += G) {
          const Op o = load_op(C.ops, a);
          const cx amp = group_amp<double>(C.terms, o, h, W);
          const int2* fl = C.flows + o.cpl;
          for (int f = 0; f < o.mass; ++f) {
            const int2 q = __ldg(fl + f);
            const cx r = rot_phase(q.y & 3, amp);
            J[2 * q.x] += r.r;
            J[2 * q.x + 1] += r.i;
          }
        }
      }
      __syncthreads();
    }
    // the store is dead now: partial jamps of lanes > 0, then per-helicity results
    double* part = store;                               // [G-1][ngood][2 ncol]
    if (act && g > 0)
      for (int k = 0; k < 2 * ncol; ++k) part[((g - 1) * P.ngood + hl) * 2 * ncol + k] = J[k];
    __syncthreads();
    if (act && g == 0)
      for (int gg = 1; gg < G; ++gg)
        for (int k = 0; k < 2 * ncol; ++k) J[k] += part[((gg - 1) * P.ngood + hl) * 2 * ncol + k];
    __syncthreads();
    double* mh_s = store;
    double* cwh_s = store + P.ngood;           // [ngood][ncol] |J_i(h)|^2
    double* colw_s = cwh_s + P.ngood * ncol;
    if (act && g == 0) {
      const double mh = scale * quad_form([&](int k) { return J[k]; }, P.colsym, P.colsym_f, ncol, mode);
      mh_s[hl] = mh;
      if (mh_out) mh_out[e * P.ngood + hl] = mh;
      for (int i = 0; i < ncol; ++i)
        cwh_s[hl * ncol + i] = scale * fma(J[2 * i], J[2 * i], J[2 * i + 1] * J[2 * i + 1]);
    }
    __syncthreads();
    for (int i = tid; i < ncol; i += T) {
      double w = 0.0;
      for (int ih = 0; ih < P.ngood; ++ih) w += cwh_s[ih * ncol + i];
      colw_s[i] = w;
      if (colw_out) colw_out[e * ncol + i] = w;
    }
    __syncthreads();
    if (tid == 0)
      finish_event(P, e, [&](int ih) { return mh_s[ih]; }, [&](int i) { return colw_s[i]; }, rhel, rcol, me, selhel,
                   selcol);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ host helpers
// Philox-4x32-10 (Salmon et al., SC'11) and RAMBO (Kleiss, Stirling, Ellis 1986) for the
// helicity-filter events.
void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0], p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t h0 = (uint32_t)(p0 >> 32), l0 = (uint32_t)p0, h1 = (uint32_t)(p1 >> 32), l1 = (uint32_t)p1;
    const uint32_t n0 = h1 ^ c[1] ^ k0, n2 = h0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = l1; c[2] = n2; c[3] = l0;
  }
}

double uniform_open(uint64_t seed, uint32_t stream, uint64_t evt, int idx) {
  uint32_t c[4] = {(uint32_t)evt, (uint32_t)(idx / 4), stream, (uint32_t)(evt >> 32)};
  philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  return ((double)c[idx % 4] + 0.5) * (1.0 / 4294967296.0);
}

// events [n][npar][4]: two beams along +-z, then RAMBO final state
void filter_events(int n, int npar, double sqrts, const std::vector<double>& masses, uint64_t seed,
                   std::vector<double>& out) {
  const int nf = npar - 2;
  out.assign((size_t)n * npar * 4, 0.0);
  for (int e = 0; e < n; ++e) {
    double* pe = out.data() + (size_t)e * npar * 4;
    pe[0] = 0.5 * sqrts; pe[3] = 0.5 * sqrts;
    pe[4] = 0.5 * sqrts; pe[7] = -0.5 * sqrts;
    std::vector<double> q((size_t)nf * 4), p((size_t)nf * 4);
    double Q[4] = {0, 0, 0, 0};
    for (int i = 0; i < nf; ++i) {
      const double r0 = uniform_open(seed, 0, e, 4 * i), r1 = uniform_open(seed, 0, e, 4 * i + 1),
                   r2 = uniform_open(seed, 0, e, 4 * i + 2), r3 = uniform_open(seed, 0, e, 4 * i + 3);
      const double c = 2.0 * r0 - 1.0, s = std::sqrt(std::max(0.0, 1.0 - c * c)), f = 2.0 * M_PI * r1;
      const double e0 = -std::log(r2 * r3);
      q[4 * i] = e0; q[4 * i + 1] = e0 * s * std::cos(f); q[4 * i + 2] = e0 * s * std::sin(f); q[4 * i + 3] = e0 * c;
      for (int j = 0; j < 4; ++j) Q[j] += q[4 * i + j];
    }
    const double M = std::sqrt(Q[0] * Q[0] - Q[1] * Q[1] - Q[2] * Q[2] - Q[3] * Q[3]);
    const double b[3] = {-Q[1] / M, -Q[2] / M, -Q[3] / M};
    const double g = Q[0] / M, a = 1.0 / (1.0 + g), x = sqrts / M;
    for (int i = 0; i < nf; ++i) {
      const double bq = b[0] * q[4 * i + 1] + b[1] * q[4 * i + 2] + b[2] * q[4 * i + 3];
      p[4 * i] = x * (g * q[4 * i] + bq);
      for (int j = 0; j < 3; ++j) p[4 * i + 1 + j] = x * (q[4 * i + 1 + j] + b[j] * q[4 * i] + a * bq * b[j]);
    }
    bool massive = false;
    for (double m : masses) massive |= m > 0.0;
    if (massive) {
      double msum = 0.0;
      for (double m : masses) msum += m;
      double xi = std::sqrt(1.0 - (msum / sqrts) * (msum / sqrts));
      for (int it = 0; it < 60; ++it) {
        double f = -sqrts, df = 0.0;
        for (int i = 0; i < nf; ++i) {
          const double en = std::sqrt(masses[i] * masses[i] + xi * xi * p[4 * i] * p[4 * i]);
          f += en;
          df += xi * p[4 * i] * p[4 * i] / en;
        }
        const double step = f / df;
        xi -= step;
        if (std::fabs(step) <= 1e-15 * xi) break;
      }
      for (int i = 0; i < nf; ++i) {
        const double e0 = p[4 * i];
        p[4 * i] = std::sqrt(masses[i] * masses[i] + xi * xi * e0 * e0);
        for (int j = 1; j < 4; ++j) p[4 * i + j] *= xi;
      }
    }
    for (int i = 0; i < nf; ++i)
      for (int j = 0; j < 4; ++j) pe[8 + 4 * i + j] = p[4 * i + j];
  }
}

std::string normalise(const char* s) {
  std::string out;
  bool sp = false;
  for (const char* c = s; *c; ++c) {
    if (std::isspace((unsigned char)*c)) { sp = !out.empty(); continue; }
    if (*c == '>') { if (!out.empty() && out.back() != ' ') out += ' '; out += "> "; sp = false; continue; }
    if (sp && !out.empty() && out.back() != ' ') out += ' ';
    sp = false;
    out += *c;
  }
  while (!out.empty() && out.back() == ' ') out.pop_back();
  return out;
}

double param_value(const mgx_params& p, int id) {
  switch (id) {
    case 1: return p.mt;
    case 2: return p.wt;
    case 3: return p.mz;
    case 4: return p.wz;
    case 5: return p.mta;
    default: return 0.0;
  }
}

// float -> bf16 bits, round to nearest even (finite inputs), and back
uint16_t bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
float bf16_value(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

int sm_count(int device) {
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device);
  return n > 0 ? n : 1;
}

}  // namespace

struct mgx_process {
  int device = 0;
  const mgx_program_desc* prog = nullptr;
  KParams kp{};
  int nhel = 0;
  std::vector<int> good;
  std::vector<double> colour;
  int4* d_ops = nullptr;
  int2* d_flows = nullptr;
  double* d_col = nullptr;
  float* d_colf = nullptr;
  int4* d_terms = nullptr;
  int4* d_cta_ops = nullptr;
  int2* d_cta_flows = nullptr;
  int4* d_cta_terms = nullptr;
  int* d_cta_items = nullptr;
  int3* d_cta_steps = nullptr;
  // integer-scaled colour matrix as canonical K-major tiles per 32-column K chunk: tf32 (one part)
  // and bf16 (two parts per chunk)
  unsigned char* d_tc_b32 = nullptr;
  unsigned char* d_tc_b16 = nullptr;
  int tc_kpad = 0, tc_kpad16 = 0, tc_npad = 0, tc_cols = 0;
  bool bf16_exact = false;    // every integer entry is the sum of its two bf16 parts
  int* d_status = nullptr;    // device error counter of the tensor-core waits
  int tc_skip_mma = 0;        // test hook: the tensor-core colour sum issues no MMA
  unsigned long long tc_wait_ns = 1000000000ull;   // time limit of one tensor-core wait
  int blocks_per_sm = 4;      // thread-per-event kernel
  int kernel = MGX_KERNEL_AUTO;
  // work model of the helicity-parallel and diagram-split plans (filled after the helicity filter)
  std::vector<int> most;                // [2^npar]: good helicities of the largest group, per fixed-leg set
  std::vector<double> cur_work[4];      // [part][2^npar]: current-variant work (whole program, splits 2/4/8)
  std::vector<double> amp_work[4];      // [part]: amplitude work per helicity
  int nparts[4] = {1, 1, 1, 1};
  int* d_split_ops[3] = {nullptr, nullptr, nullptr};
  int* d_split_start[3] = {nullptr, nullptr, nullptr};
};

namespace {

// the float kernel has half the registers of the float64 one (64 vs 128), so twice the blocks fit
int64_t grid_threads(const mgx_process* pr, int64_t nevt, int mode = MGX_FP64) {
  const int bps = mode == MGX_FLOAT ? 2 * pr->blocks_per_sm : pr->blocks_per_sm;
  const int64_t cap = (int64_t)sm_count(pr->device) * bps * kThreads;
  const int64_t need = ((nevt + kThreads - 1) / kThreads) * kThreads;
  return std::max<int64_t>(kThreads, std::min(cap, need));
}

// per-thread workspace bytes: one 8-byte slot per element, 4-byte in the float mode
size_t thread_ws_bytes(const KParams& kp, int mode) {
  return (size_t)kp.ws_doubles * (mode == MGX_FLOAT ? sizeof(float) : sizeof(double));
}

void set_layout(KParams& kp, int cur_doubles, int ngood, int ncol) {
  kp.cur_doubles = cur_doubles;
  kp.jamp_off = cur_doubles;
  kp.mh_off = kp.jamp_off + 2 * ncol * ngood;
  kp.colw_off = kp.mh_off + ngood;
  kp.ws_doubles = kp.colw_off + ncol;
}

bool mode_ok(int mode) {
  return mode == MGX_FP64 || mode == MGX_MIXED_FP32 || mode == MGX_MIXED_TF32 || mode == MGX_MIXED_BF16X3 ||
         mode == MGX_FLOAT;
}
bool mode_tc(int mode) { return mode == MGX_MIXED_TF32 || mode == MGX_MIXED_BF16X3; }
// modes whose whole path is the float64 amplitude code (CTA kernel, batch, fixed-scratch entry)
bool mode_f64(int mode) { return mode == MGX_FP64 || mode == MGX_MIXED_FP32; }

bool cta_usable(const mgx_process* pr, const KParams& kp) {
  return pr->prog->cta.nops > 0 && kp.ngood <= 128 && kp.ncol <= kMaxColCta;
}

bool use_cta(const mgx_process* pr, const KParams& kp) {
  return pr->kernel == MGX_KERNEL_CTA && cta_usable(pr, kp);
}

// shared-memory-workspace variant of the thread-per-event kernel
constexpr int kSmemThreads = 64;
constexpr size_t kSmemMax = 227u << 10;   // dynamic shared memory per block
size_t smem_ws_block_bytes(const KParams& kp, int mode) {
  return (size_t)kSmemThreads * (thread_ws_bytes(kp, mode) + 4 * kp.npar * sizeof(double));
}
bool smem_usable(const KParams& kp, int mode) {
  return (mode == MGX_FP64 || mode == MGX_MIXED_FP32 || mode == MGX_FLOAT) && smem_ws_block_bytes(kp, mode) <= kSmemMax;
}
// the thread kernel with its workspace in shared memory: chosen explicitly, or by AUTO when the
// whole batch fits one pass of a block per SM (a latency-bound batch of a small process)
bool use_smem_ws(const mgx_process* pr, const KParams& kp, int64_t nevt, int mode) {
  if (!smem_usable(kp, mode)) return false;
  if (pr->kernel == MGX_KERNEL_THREAD_SMEM) return true;
  return pr->kernel == MGX_KERNEL_AUTO && nevt <= (int64_t)kSmemThreads * sm_count(pr->device);
}

// AUTO on a batch too small to fill the thread kernel's grid: the launch then lasts as long as
// one thread takes for one event, and one block per event (the CTA kernel) takes a fraction of
// that.  Measured crossovers on GB300 in FP64: about 9.5k events (g g > t t~ g), 12k (g u~ >
// ta+ ta- g g u~) and 19k (g g > t t~ g g) against the thread kernel, about 2k against the
// shared-memory thread kernel of the small processes; against the helicity-parallel kernel the
// CTA kernel wins at 2048 events (g g > t t~ g g: 3.2 vs 3.5 ms) and loses at 8192 (12.4 vs 10.3 ms);
// the limits below stay under the crossovers.
bool use_cta_kernel(const mgx_process* pr, const KParams& kp, int64_t nevt, int mode) {
  if (!mode_f64(mode) || !cta_usable(pr, kp)) return false;
  if (pr->kernel == MGX_KERNEL_CTA) return true;
  const int64_t per_sm = smem_usable(kp, mode) ? 8 : 32;
  return pr->kernel == MGX_KERNEL_AUTO && nevt <= per_sm * sm_count(pr->device);
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// ---- plans for a batch: the whole-event thread kernel, the helicity-parallel kernel or the
// diagram-split kernel, chosen by a work model of the op table
struct HelPlan {
  int gshift = 0, fix = 0;   // G = 2^gshift helicity groups by the helicity bits on the legs in `fix`
  int split = 0;             // 0: no diagram split; 1, 2, 3: the split into at most 2, 4, 8 parts
  int nparts = 1;
};

int host_pdep(int v, int mask) {
  int r = 0, k = 0;
  for (int b = 0; b < 31; ++b)
    if (mask >> b & 1) {
      if (v >> k & 1) r |= 1 << b;
      ++k;
    }
  return r;
}

// float64 instructions per variant of each current kind (as in the roofline's work model); per
// helicity, an amplitude group costs one closing product per term and an add per flow
double op_variant_cost(const int32_t* o) {
  switch (o[0]) {
    case OP_EXT: return 24;
    case OP_FFV_F: case OP_FFV_FB: return 64;
    case OP_FFV_V: return 72;
    case OP_VVV: return 56;
    case OP_VVVV: return 32;
    case OP_BIL: return 56;
    case OP_RBIL: return 32;
    default: return 8.0 * std::max(0, o[12] - 1);   // OP_SUM: a 4-vector add per further summand
  }
}

// Work model of a process (after the helicity filter), for every set F of fixed legs: the largest
// helicity group's good-helicity count, and per part of the whole program (s = 0) and of each
// diagram split (s = 1..3) the current-variant work a thread does with legs F fixed and its
// amplitude work per helicity.
void build_work_model(mgx_process* pr) {
  const mgx_program_desc* prog = pr->prog;
  const int nf = 1 << prog->npar;
  pr->most.assign(nf, 0);
  for (int F = 0; F < nf; ++F) {
    const int k = __builtin_popcount((unsigned)F);
    for (int g = 0; g < (1 << k); ++g) {
      const int bits = host_pdep(g, F);
      int c = 0;
      for (int h : pr->good) c += (h & F) == bits;
      pr->most[F] = std::max(pr->most[F], c);
    }
  }
  for (int sidx = 0; sidx < 4; ++sidx) {
    const int np = sidx == 0 ? 1 : prog->split[sidx - 1].nparts;
    pr->nparts[sidx] = np;
    pr->cur_work[sidx].assign((size_t)np * nf, 0.0);
    pr->amp_work[sidx].assign(np, 0.0);
    for (int d = 0; d < np; ++d) {
      const int i0 = sidx == 0 ? 0 : prog->split[sidx - 1].start[d];
      const int i1 = sidx == 0 ? prog->nops : prog->split[sidx - 1].start[d + 1];
      for (int li = i0; li < i1; ++li) {
        const int32_t* o = prog->ops + 16 * (sidx == 0 ? li : prog->split[sidx - 1].ops[li]);
        if (o[0] == OP_AMP) {
          pr->amp_work[sidx][d] += 16.0 * o[12] + 2.0 * o[10];
          continue;
        }
        const double w = op_variant_cost(o);
        for (int F = 0; F < nf; ++F)
          pr->cur_work[sidx][(size_t)d * nf + F] += w * (double)(1 << __builtin_popcount((unsigned)(o[5] & ~F)));
      }
    }
  }
}

enum { PLAN_ANY = 0, PLAN_HEL = 1, PLAN_SPLIT = 2 };

// Time model of a plan on the GB300, from the float64 thread kernel's measured timings: a thread
// alone on an SM executes about one work unit (float64 instruction of the work model) per 60 ns,
// and the full grid about 5.2e11 units per second (152 SMs), scaled by the SM count.  A plan's time
// is the larger of its busiest thread's latency and its total work at the full-grid rate.
constexpr double kSecPerUnitLatency = 6.0e-8;
constexpr double kUnitsPerSecPerSm = 5.2e11 / 152;

// The plan of least estimated time (plus, for a diagram split, the combine step: one thread per
// event and helicity).  PLAN_ANY keeps the whole-event thread kernel unless another plan is
// estimated at least 1.1x faster; PLAN_HEL and PLAN_SPLIT return the best plan of that kind.
HelPlan best_plan(const mgx_process* pr, int64_t nevt, int mode, int kind) {
  const int nf = 1 << pr->prog->npar;
  const double n = pr->prog->ncol;
  const double colour = mode == MGX_FP64 ? n * n + 3 * n : 2 * n;
  const double ngood = (double)pr->good.size();
  const double rate = kUnitsPerSecPerSm * sm_count(pr->device) * (mode == MGX_FLOAT ? 2.0 : 1.0);
  auto time = [&](double wmax, double wtotal) { return std::max(wmax * kSecPerUnitLatency, wtotal / rate); };
  const double w1 = pr->cur_work[0][0] + (pr->amp_work[0][0] + colour) * ngood;
  const double t_thread = time(w1, w1 * (double)nevt);
  HelPlan best;
  double tb = -1.0;
  for (int sidx = 0; sidx < 4; ++sidx) {
    if ((kind == PLAN_HEL && sidx != 0) || (kind == PLAN_SPLIT && sidx == 0)) continue;
    const int np = pr->nparts[sidx];
    if (sidx > 0 && np < 2) continue;
    for (int F = sidx == 0 ? 1 : 0; F < nf; ++F) {
      const int k = __builtin_popcount((unsigned)F);
      // a split thread zeroes, updates and copies out the partial jamps of all its group's
      // helicities; measured, splits pay off only with at least 8 helicity groups
      if (k > 6 || (sidx > 0 && k < 3)) continue;
      const double groups = (double)(1 << k);
      double wmax = 0.0, wsum = 0.0;
      for (int d = 0; d < np; ++d) {
        const double cur = pr->cur_work[sidx][(size_t)d * nf + F];
        const double amp = pr->amp_work[sidx][d] + (sidx == 0 ? colour : 0.0);
        wmax = std::max(wmax, cur + amp * pr->most[F]);
        wsum += groups * cur + amp * ngood;
      }
      double t = time(wmax, wsum * (double)nevt);
      if (sidx > 0) {
        const double wc = colour + 2.0 * n * np;     // combine: one thread per (event, helicity)
        t += time(wc, wc * (double)nevt * ngood);
      }
      if (tb < 0.0 || t < tb) {
        tb = t;
        best = HelPlan{k, F, sidx, np};
      }
    }
  }
  if (kind == PLAN_ANY && !(tb >= 0.0 && tb < 0.9 * t_thread)) return HelPlan{};
  return best;
}

struct HelLayout {
  size_t ws, pj, mh, cw, total;
};
HelLayout hel_layout(const mgx_process* pr, const KParams& kp, const HelPlan& hp, int64_t nevt, int mode, int64_t nt) {
  HelLayout L;
  const size_t real = mode == MGX_FLOAT ? sizeof(float) : sizeof(double);
  L.ws = align256((size_t)nt * thread_ws_bytes(kp, mode));
  L.pj = hp.split ? align256((size_t)nevt * hp.nparts * kp.ngood * 2 * kp.ncol * real) : 0;
  L.mh = align256((size_t)nevt * kp.ngood * sizeof(double));
  // colour-weight terms: per (event, group) without a split, per (event, helicity) with one
  L.cw = align256((size_t)nevt * (hp.split ? (size_t)kp.ngood : ((size_t)1 << hp.gshift)) * kp.ncol * sizeof(double));
  L.total = L.ws + L.pj + L.mh + L.cw;
  return L;
}
// items of a plan: every (group, part) over the events padded to whole 128-thread blocks
int64_t plan_items(const HelPlan& hp, int64_t nevt) {
  return (((nevt + kThreads - 1) / kThreads * kThreads) * hp.nparts) << hp.gshift;
}

// the helicity-parallel or diagram-split kernels: chosen explicitly, or by AUTO for a batch that
// leaves the thread kernel's grid underfilled when the work model says a plan is clearly cheaper
// (float64, mixed float32 and float modes; the tensor-core modes run the fused thread kernel)
bool use_hel_kernel(const mgx_process* pr, const KParams& kp, int64_t nevt, int mode, HelPlan* plan) {
  if (!(mode_f64(mode) || mode == MGX_FLOAT) || pr->most.empty()) return false;
  if (pr->kernel == MGX_KERNEL_HELICITY || pr->kernel == MGX_KERNEL_SPLIT) {
    *plan = best_plan(pr, nevt, mode, pr->kernel == MGX_KERNEL_HELICITY ? PLAN_HEL : PLAN_SPLIT);
    return plan->gshift > 0 || plan->split > 0;
  }
  if (pr->kernel != MGX_KERNEL_AUTO || use_cta_kernel(pr, kp, nevt, mode) || use_smem_ws(pr, kp, nevt, mode))
    return false;
  *plan = best_plan(pr, nevt, mode, PLAN_ANY);
  return plan->gshift > 0 || plan->split > 0;
}

size_t cta_smem_bytes(const mgx_process* pr, const KParams& kp) {
  const int ngp = kp.ngood <= 32 ? 32 : (kp.ngood <= 64 ? 64 : 128);
  const int G = kCtaThreads / ngp;
  const int partials = (G - 1) * kp.ngood * 2 * kp.ncol;
  const int results = kp.ngood + kp.ngood * kp.ncol + kp.ncol;
  return (size_t)(std::max({pr->prog->cta.store, results, partials}) + 4 * kp.npar) * sizeof(double);
}

int launch_cta(mgx_process* pr, const KParams& kp, int64_t nevt, const double* mom, const double* as,
               const double* rh, const double* rc, double* me, int32_t* sh, int32_t* sc, double* mh, double* cw,
               int mode, cudaStream_t st) {
  const size_t smem = cta_smem_bytes(pr, kp);
  if (cudaFuncSetAttribute(me_cta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return MGX_ERR_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, me_cta_kernel, kCtaThreads, smem) != cudaSuccess ||
      per_sm < 1)
    return MGX_ERR_CUDA;
  const int64_t blocks = std::min<int64_t>(nevt, (int64_t)per_sm * sm_count(pr->device));
  CtaTab C{pr->d_cta_ops, pr->d_cta_flows, pr->d_cta_terms, pr->d_cta_items, pr->d_cta_steps,
           pr->prog->cta.nsteps, pr->prog->cta.store};
  me_cta_kernel<<<(unsigned)blocks, kCtaThreads, smem, st>>>(kp, C, nevt, mom, as, rh, rc, me, sh, sc, mh, cw, mode);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}


// Tensor-core colour-sum modes: the thread-per-event kernel with the fused tcgen05 colour sum; the
// workspace is that of the float64 thread kernel.
template <class F>
int launch_tc(mgx_process* pr, const KParams& kp, int64_t nevt, const double* mom, const double* as,
              const double* rh, const double* rc, double* me, int32_t* sh, int32_t* sc, double* mh, double* cw,
              void* ws, size_t wsb, cudaStream_t st) {
  static_assert(kThreads == kTcRows, "one tensor-core row per event of the block");
  const bool bf16 = F::kFmt == umma::FMT_BF16;
  if (bf16 && !pr->bf16_exact) return MGX_ERR_UNSUPPORTED_MODE;
  TcArgs A{};
  A.bchunks = bf16 ? pr->d_tc_b16 : pr->d_tc_b32;
  A.ncol = kp.ncol;
  A.npad = pr->tc_npad;
  A.kpad = bf16 ? pr->tc_kpad16 : pr->tc_kpad;
  A.nchunk = (A.kpad + kTcKc - 1) / kTcKc;
  A.tcols = (uint32_t)pr->tc_cols;
  A.inv_den = 1.0 / pr->prog->col_den;
  A.status = pr->d_status;
  A.skip_mma = pr->tc_skip_mma;
  A.wait_ns = pr->tc_wait_ns;
  const size_t stage = tc_stage_bytes<F>(A.kpad, A.npad);
  const size_t moms = (size_t)kThreads * 4 * kp.npar * sizeof(double);
  const size_t bar_off = align256(std::max(stage, moms));
  const size_t smem = bar_off + 16;
  if (cudaFuncSetAttribute(me_tc_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return MGX_ERR_CUDA;
  // the persistent grid, at most as many blocks per SM as the SM's tensor memory holds
  const int bps = std::min(pr->blocks_per_sm, 512 / pr->tc_cols);
  const int64_t cap = (int64_t)sm_count(pr->device) * std::max(1, bps) * kThreads;
  const int64_t nt = std::max<int64_t>(kThreads, std::min(cap, ((nevt + kThreads - 1) / kThreads) * kThreads));
  if (ws == nullptr || wsb < (size_t)nt * thread_ws_bytes(kp, MGX_FP64)) return MGX_ERR_WORKSPACE_TOO_SMALL;
  me_tc_kernel<F><<<(unsigned)(nt / kThreads), kThreads, smem, st>>>(kp, A, nevt, mom, as, rh, rc, me, sh, sc, mh, cw,
                                                                     (double*)ws, nt, bar_off);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

// the helicity-parallel kernel and its finish kernel, or the diagram-split kernel, its combine
// kernel and the finish kernel
int launch_hel(mgx_process* pr, const KParams& kp, const HelPlan& hp, int64_t nevt, const double* mom,
               const double* as, const double* rh, const double* rc, double* me, int32_t* sh, int32_t* sc, double* mh,
               double* cw, int mode, void* ws, size_t wsb, cudaStream_t st) {
  const int64_t nt = grid_threads(pr, plan_items(hp, nevt), mode);
  const HelLayout L = hel_layout(pr, kp, hp, nevt, mode, nt);
  if (ws == nullptr || wsb < L.total) return MGX_ERR_WORKSPACE_TOO_SMALL;
  char* p = (char*)ws;
  void* pj = p + L.ws;
  double* mh_buf = (double*)(p + L.ws + L.pj);
  double* cw_buf = (double*)(p + L.ws + L.pj + L.mh);
  const size_t shm = (size_t)kThreads * 4 * kp.npar * sizeof(double);
  const unsigned blocks = (unsigned)(nt / kThreads);
  const bool f32 = mode == MGX_FLOAT;
  if (hp.split == 0) {
    if (f32)
      me_hel_kernel<float><<<blocks, kThreads, shm, st>>>(kp, nevt, hp.gshift, hp.fix, mom, as, mh_buf, cw_buf,
                                                          (double*)ws, nt, mode);
    else
      me_hel_kernel<double><<<blocks, kThreads, shm, st>>>(kp, nevt, hp.gshift, hp.fix, mom, as, mh_buf, cw_buf,
                                                           (double*)ws, nt, mode);
    finish_hel_kernel<<<(unsigned)((nevt + kThreads - 1) / kThreads), kThreads, 0, st>>>(
        kp, nevt, 1 << hp.gshift, mh_buf, cw_buf, rh, rc, me, sh, sc, mh, cw);
    return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
  }
  const int* ops = pr->d_split_ops[hp.split - 1];
  const int* start = pr->d_split_start[hp.split - 1];
  const int64_t pairs = nevt * kp.ngood;
  const unsigned cblocks = (unsigned)((pairs + kThreads - 1) / kThreads);
  if (f32) {
    me_split_kernel<float><<<blocks, kThreads, shm, st>>>(kp, nevt, hp.gshift, hp.fix, hp.nparts, ops, start, mom,
                                                          (float*)pj, (double*)ws, nt);
    split_combine_kernel<float><<<cblocks, kThreads, 0, st>>>(kp, nevt, hp.nparts, (const float*)pj, as, mh_buf,
                                                              cw_buf, mode);
  } else {
    me_split_kernel<double><<<blocks, kThreads, shm, st>>>(kp, nevt, hp.gshift, hp.fix, hp.nparts, ops, start, mom,
                                                           (double*)pj, (double*)ws, nt);
    split_combine_kernel<double><<<cblocks, kThreads, 0, st>>>(kp, nevt, hp.nparts, (const double*)pj, as, mh_buf,
                                                               cw_buf, mode);
  }
  finish_hel_kernel<<<(unsigned)((nevt + kThreads - 1) / kThreads), kThreads, 0, st>>>(
      kp, nevt, kp.ngood, mh_buf, cw_buf, rh, rc, me, sh, sc, mh, cw);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

int launch(mgx_process* pr, const KParams& kp, int64_t nevt, const double* mom, const double* as,
           const double* rh, const double* rc, double* me, int32_t* sh, int32_t* sc, double* mh, double* cw,
           int mode, void* ws, size_t wsb, cudaStream_t st) {
  if (nevt == 0) return MGX_OK;
  if (mode == MGX_MIXED_TF32) return launch_tc<TcTf32>(pr, kp, nevt, mom, as, rh, rc, me, sh, sc, mh, cw, ws, wsb, st);
  if (mode == MGX_MIXED_BF16X3)
    return launch_tc<TcBf16x3>(pr, kp, nevt, mom, as, rh, rc, me, sh, sc, mh, cw, ws, wsb, st);
  if (use_cta_kernel(pr, kp, nevt, mode)) return launch_cta(pr, kp, nevt, mom, as, rh, rc, me, sh, sc, mh, cw, mode, st);
  HelPlan hp;
  if (use_hel_kernel(pr, kp, nevt, mode, &hp))
    return launch_hel(pr, kp, hp, nevt, mom, as, rh, rc, me, sh, sc, mh, cw, mode, ws, wsb, st);
  if (use_smem_ws(pr, kp, nevt, mode)) {
    const size_t smem = smem_ws_block_bytes(kp, mode);
    auto kern = mode == MGX_FLOAT ? me_kernel<float, true> : me_kernel<double, true>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return MGX_ERR_CUDA;
    const int64_t blocks = std::min<int64_t>((nevt + kSmemThreads - 1) / kSmemThreads, sm_count(pr->device));
    kern<<<(unsigned)blocks, kSmemThreads, smem, st>>>(kp, nevt, mom, as, rh, rc, me, sh, sc, mh, cw, nullptr,
                                                       blocks * kSmemThreads, mode);
    return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
  }
  const int64_t nt = grid_threads(pr, nevt, mode);
  const size_t need = (size_t)nt * thread_ws_bytes(kp, mode);
  if (wsb < need || ws == nullptr) return MGX_ERR_WORKSPACE_TOO_SMALL;
  const int blocks = (int)(nt / kThreads);
  const size_t shm = (size_t)kThreads * 4 * kp.npar * sizeof(double);
  if (mode == MGX_FLOAT)
    me_kernel<float, false><<<blocks, kThreads, shm, st>>>(kp, nevt, mom, as, rh, rc, me, sh, sc, mh, cw, (double*)ws, nt,
                                                    mode);
  else
    me_kernel<double, false><<<blocks, kThreads, shm, st>>>(kp, nevt, mom, as, rh, rc, me, sh, sc, mh, cw, (double*)ws, nt,
                                                     mode);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

}  // namespace

extern "C" {

void mgx_params_default(mgx_params* p) {
  if (!p) return;
  p->mt = 173.0; p->wt = 1.4915;
  p->mz = 91.1876; p->wz = 2.4414;
  p->mta = 1.777;
  p->alpha_em = 1.0 / 132.507;
  p->gf = 1.16639e-5;
  p->filter_sqrt_s = 1000.0;
}

int mgx_num_processes(void) { return mgx_num_programs; }

const char* mgx_process_name(int i) { return (i >= 0 && i < mgx_num_programs) ? mgx_programs[i].name : nullptr; }

int mgx_version(void) { return 100; }

const char* mgx_status_string(int s) {
  switch (s) {
    case MGX_OK: return "ok";
    case MGX_ERR_INVALID_ARGUMENT: return "invalid argument";
    case MGX_ERR_UNKNOWN_PROCESS: return "unknown process";
    case MGX_ERR_CUDA: return "CUDA error";
    case MGX_ERR_DEVICE_MISMATCH: return "device mismatch";
    case MGX_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case MGX_ERR_NO_GOOD_HELICITY: return "no helicity survives the filter";
    case MGX_ERR_UNSUPPORTED_MODE: return "unsupported mode";
    default: return "unknown status";
  }
}

void mgx_process_destroy(mgx_process* pr) {
  if (!pr) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(pr->device);
  cudaFree(pr->d_ops);
  cudaFree(pr->d_flows);
  cudaFree(pr->d_col);
  cudaFree(pr->d_colf);
  cudaFree(pr->d_terms);
  cudaFree(pr->d_tc_b32);
  cudaFree(pr->d_tc_b16);
  cudaFree(pr->d_status);
  for (int i = 0; i < 3; ++i) {
    cudaFree(pr->d_split_ops[i]);
    cudaFree(pr->d_split_start[i]);
  }
  cudaFree(pr->d_cta_ops);
  cudaFree(pr->d_cta_flows);
  cudaFree(pr->d_cta_terms);
  cudaFree(pr->d_cta_items);
  cudaFree(pr->d_cta_steps);
  cudaSetDevice(cur);
  delete pr;
}

int mgx_process_create(const char* process, const mgx_params* params, int device, uint64_t filter_seed,
                       mgx_process** out) {
  if (!process || !out) return MGX_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return MGX_ERR_INVALID_ARGUMENT;
  const std::string want = normalise(process);
  const mgx_program_desc* prog = nullptr;
  for (int i = 0; i < mgx_num_programs; ++i)
    if (normalise(mgx_programs[i].name) == want) prog = &mgx_programs[i];
  if (!prog) return MGX_ERR_UNKNOWN_PROCESS;
  mgx_params prm;
  mgx_params_default(&prm);
  if (params) prm = *params;

  int cur = 0;
  cudaGetDevice(&cur);
  if (cudaSetDevice(device) != cudaSuccess) return MGX_ERR_CUDA;
  mgx_process* pr = new mgx_process();
  pr->device = device;
  pr->prog = prog;
  pr->nhel = 1 << prog->npar;
  KParams& kp = pr->kp;
  kp.nops = prog->nops;
  kp.ncol = prog->ncol;
  kp.npar = prog->npar;
  kp.nin = prog->nin;
  kp.avg = 1.0 / prog->avg_den;
  kp.gs_power = prog->gs_power;
  kp.jamp_zero = prog->jamp_zero;
  // couplings
  const double e = std::sqrt(4.0 * M_PI * prm.alpha_em);
  const double mz2 = prm.mz * prm.mz;
  const double mw2 = 0.5 * mz2 + std::sqrt(0.25 * mz2 * mz2 - M_PI * prm.alpha_em * mz2 / (std::sqrt(2.0) * prm.gf));
  const double sw2 = 1.0 - mw2 / mz2, sw = std::sqrt(sw2), cw = std::sqrt(1.0 - sw2);
  for (int i = 0; i < prog->ncoupl && i < MAXCPL; ++i) {
    const int boson = (int)prog->coupl[3 * i];
    const double q = prog->coupl[3 * i + 1], t3 = prog->coupl[3 * i + 2];
    double* c = kp.cpl[i];
    if (boson == 0) {  // i g_s
      c[0] = 0; c[1] = 1; c[2] = 0; c[3] = 1;
      kp.cplflags[i] = CPL_GS;
    } else if (boson == 1) {  // -i e Q
      c[0] = 0; c[1] = -e * q; c[2] = 0; c[3] = -e * q;
      kp.cplflags[i] = 0;
    } else {  // -i gL, -i gR
      const double gl = e * (t3 - q * sw2) / (sw * cw), gr = -e * q * sw2 / (sw * cw);
      c[0] = 0; c[1] = -gl; c[2] = 0; c[3] = -gr;
      kp.cplflags[i] = CPL_CHIRAL;
    }
  }
  for (int i = 0; i < prog->nmass && i < MAXMASS; ++i) {
    kp.mass[i] = param_value(prm, prog->mass[2 * i]);
    kp.width[i] = param_value(prm, prog->mass[2 * i + 1]);
    kp.massive[i] = kp.mass[i] > 0.0 ? 1 : 0;
  }
  // device tables
  const int n = prog->ncol;
  std::vector<double> cs((size_t)n * n, 0.0);
  std::vector<float> csf((size_t)n * n, 0.0f);
  pr->colour.assign(prog->colour, prog->colour + (size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double v = j == i ? prog->colour[i * n + j] : (j > i ? 2.0 * prog->colour[i * n + j] : 0.0);
      cs[(size_t)i * n + j] = v;
      csf[(size_t)i * n + j] = (float)v;
    }
  bool ok = cudaMalloc(&pr->d_terms, sizeof(int4) * 2 * std::max(1, prog->nterms_tab)) == cudaSuccess &&
            cudaMemcpy(pr->d_terms, prog->terms, sizeof(int4) * 2 * prog->nterms_tab, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMalloc(&pr->d_ops, sizeof(int32_t) * 16 * prog->nops) == cudaSuccess &&
            cudaMalloc(&pr->d_flows, sizeof(int2) * std::max(1, prog->nflows)) == cudaSuccess &&
            cudaMalloc(&pr->d_col, sizeof(double) * n * n) == cudaSuccess &&
            cudaMalloc(&pr->d_colf, sizeof(float) * n * n) == cudaSuccess;
  ok = ok && cudaMemcpy(pr->d_ops, prog->ops, sizeof(int32_t) * 16 * prog->nops, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(pr->d_flows, prog->flows, sizeof(int32_t) * 2 * prog->nflows, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(pr->d_col, cs.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(pr->d_colf, csf.data(), sizeof(float) * n * n, cudaMemcpyHostToDevice) == cudaSuccess;
  const auto& ct = prog->cta;
  if (ok && ct.nops > 0) {
    ok = cudaMalloc(&pr->d_cta_ops, sizeof(int32_t) * 16 * ct.nops) == cudaSuccess &&
         cudaMalloc(&pr->d_cta_flows, sizeof(int2) * std::max(1, ct.nflows)) == cudaSuccess &&
         cudaMalloc(&pr->d_cta_terms, sizeof(int4) * 2 * std::max(1, ct.nterms)) == cudaSuccess &&
         cudaMalloc(&pr->d_cta_items, sizeof(int) * std::max(1, ct.nitems)) == cudaSuccess &&
         cudaMalloc(&pr->d_cta_steps, sizeof(int3) * std::max(1, ct.nsteps)) == cudaSuccess;
    ok = ok && cudaMemcpy(pr->d_cta_ops, ct.ops, sizeof(int32_t) * 16 * ct.nops, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(pr->d_cta_flows, ct.flows, sizeof(int32_t) * 2 * ct.nflows, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(pr->d_cta_terms, ct.terms, sizeof(int4) * 2 * ct.nterms, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(pr->d_cta_items, ct.items, sizeof(int) * ct.nitems, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(pr->d_cta_steps, ct.steps, sizeof(int3) * ct.nsteps, cudaMemcpyHostToDevice) == cudaSuccess;
  }
  if (!ok) {
    mgx_process_destroy(pr);
    cudaSetDevice(cur);
    return MGX_ERR_CUDA;
  }
  if (ok) {
    // integer-scaled colour matrix Cs = den C as canonical K-major tiles, one per 32-column K chunk
    // (and per bf16 part), in the order the fused colour sum stages them
    pr->tc_kpad = (n + 7) / 8 * 8;
    pr->tc_kpad16 = (n + 15) / 16 * 16;
    pr->tc_npad = (n + 15) / 16 * 16;
    pr->tc_cols = 32;   // one accumulator, or two (Re and Im) when the contraction is one stage
    const int tc_need = pr->tc_kpad16 <= kTcKc ? 2 * pr->tc_npad : pr->tc_npad;
    while (pr->tc_cols < tc_need) pr->tc_cols *= 2;
    const int np = pr->tc_npad;
    std::vector<float> b32;
    std::vector<uint16_t> b16;
    pr->bf16_exact = true;
    for (int k0 = 0; k0 < pr->tc_kpad; k0 += kTcKc) {
      const int kc = std::min(kTcKc, pr->tc_kpad - k0);
      const size_t o = b32.size();
      b32.resize(o + (size_t)np * kc, 0.0f);
      for (int r = 0; r < n; ++r)
        for (int k = k0; k < std::min(n, k0 + kc); ++k)
          b32[o + umma::kmajor_offset(r, k - k0, kc, 4) / 4] = (float)(prog->colour[r * n + k] * prog->col_den);
    }
    for (int k0 = 0; k0 < pr->tc_kpad16; k0 += kTcKc) {
      const int kc = std::min(kTcKc, pr->tc_kpad16 - k0);
      const size_t o = b16.size(), tile = (size_t)np * kc;
      b16.resize(o + 2 * tile, 0);
      for (int r = 0; r < n; ++r)
        for (int k = k0; k < std::min(n, k0 + kc); ++k) {
          const float c = (float)(prog->colour[r * n + k] * prog->col_den);
          const uint16_t h = bf16_bits(c), l = bf16_bits(c - bf16_value(h));
          pr->bf16_exact = pr->bf16_exact && bf16_value(h) + bf16_value(l) == c;
          const size_t off = umma::kmajor_offset(r, k - k0, kc, 2) / 2;
          b16[o + off] = h;
          b16[o + tile + off] = l;
        }
    }
    ok = cudaMalloc(&pr->d_tc_b32, sizeof(float) * b32.size()) == cudaSuccess &&
         cudaMemcpy(pr->d_tc_b32, b32.data(), sizeof(float) * b32.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMalloc(&pr->d_tc_b16, sizeof(uint16_t) * b16.size()) == cudaSuccess &&
         cudaMemcpy(pr->d_tc_b16, b16.data(), sizeof(uint16_t) * b16.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMalloc(&pr->d_status, 256) == cudaSuccess && cudaMemset(pr->d_status, 0, 256) == cudaSuccess;
    for (int i = 0; i < 3 && ok; ++i) {
      const auto& sp = prog->split[i];
      const int nops = sp.start[sp.nparts];
      ok = cudaMalloc(&pr->d_split_ops[i], sizeof(int) * std::max(1, nops)) == cudaSuccess &&
           cudaMemcpy(pr->d_split_ops[i], sp.ops, sizeof(int) * nops, cudaMemcpyHostToDevice) == cudaSuccess &&
           cudaMalloc(&pr->d_split_start[i], sizeof(int) * (sp.nparts + 1)) == cudaSuccess &&
           cudaMemcpy(pr->d_split_start[i], sp.start, sizeof(int) * (sp.nparts + 1), cudaMemcpyHostToDevice) ==
               cudaSuccess;
    }
  }
  if (!ok) {
    mgx_process_destroy(pr);
    cudaSetDevice(cur);
    return MGX_ERR_CUDA;
  }
  kp.ops = pr->d_ops;
  kp.flows = pr->d_flows;
  kp.terms = pr->d_terms;
  kp.colsym = pr->d_col;
  kp.colsym_f = pr->d_colf;

  // ---- helicity filter: every helicity on 16 seeded RAMBO events; keep those nonzero anywhere
  const int nf = 16;
  std::vector<double> masses;
  for (int p = 2; p < prog->npar; ++p) masses.push_back(kp.mass[prog->extmass[p]]);
  const double sqrts = prm.filter_sqrt_s > 0.0 ? prm.filter_sqrt_s : 1000.0;
  std::vector<double> hmom;
  filter_events(nf, prog->npar, sqrts, masses, filter_seed, hmom);
  KParams fk = kp;
  fk.ngood = pr->nhel;
  for (int h = 0; h < pr->nhel; ++h) {
    fk.good[h] = h;
    fk.hidx[h] = (signed char)h;
  }
  set_layout(fk, prog->ws_doubles, fk.ngood, n);
  const int64_t nt = grid_threads(pr, nf);
  const size_t wsb = (size_t)nt * fk.ws_doubles * sizeof(double);
  double *d_mom = nullptr, *d_as = nullptr, *d_me = nullptr, *d_mh = nullptr, *d_ws = nullptr;
  std::vector<double> as(nf, 0.118), mh((size_t)nf * pr->nhel);
  ok = cudaMalloc(&d_mom, sizeof(double) * hmom.size()) == cudaSuccess &&
       cudaMalloc(&d_as, sizeof(double) * nf) == cudaSuccess && cudaMalloc(&d_me, sizeof(double) * nf) == cudaSuccess &&
       cudaMalloc(&d_mh, sizeof(double) * mh.size()) == cudaSuccess && cudaMalloc(&d_ws, wsb) == cudaSuccess;
  ok = ok && cudaMemcpy(d_mom, hmom.data(), sizeof(double) * hmom.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(d_as, as.data(), sizeof(double) * nf, cudaMemcpyHostToDevice) == cudaSuccess;
  int rc = MGX_OK;
  // the filter evaluates every helicity with the whole-event thread kernel (the good-helicity list
  // that the other kernels' choices depend on does not exist yet)
  pr->kernel = MGX_KERNEL_THREAD;
  if (ok) rc = launch(pr, fk, nf, d_mom, d_as, nullptr, nullptr, d_me, nullptr, nullptr, d_mh, nullptr, MGX_FP64, d_ws, wsb, 0);
  pr->kernel = MGX_KERNEL_AUTO;
  ok = ok && rc == MGX_OK && cudaMemcpy(mh.data(), d_mh, sizeof(double) * mh.size(), cudaMemcpyDeviceToHost) == cudaSuccess;
  cudaFree(d_mom); cudaFree(d_as); cudaFree(d_me); cudaFree(d_mh); cudaFree(d_ws);
  if (!ok) {
    mgx_process_destroy(pr);
    cudaSetDevice(cur);
    return rc != MGX_OK ? rc : MGX_ERR_CUDA;
  }
  for (int h = 0; h < pr->nhel; ++h) {
    bool nz = false;
    for (int ev = 0; ev < nf; ++ev) nz |= mh[(size_t)ev * pr->nhel + h] != 0.0;
    if (nz) pr->good.push_back(h);
  }
  if (pr->good.empty()) {
    mgx_process_destroy(pr);
    cudaSetDevice(cur);
    return MGX_ERR_NO_GOOD_HELICITY;
  }
  kp.ngood = (int)pr->good.size();
  for (int h = 0; h < MAXHEL; ++h) kp.hidx[h] = -1;
  for (int i = 0; i < kp.ngood; ++i) {
    kp.good[i] = pr->good[i];
    kp.hidx[pr->good[i]] = (signed char)i;
  }
  set_layout(kp, prog->ws_doubles, kp.ngood, n);
  build_work_model(pr);
  cudaSetDevice(cur);
  *out = pr;
  return MGX_OK;
}

int mgx_process_info(const mgx_process* pr, int* npar, int* nhel, int* ngood, int* ndiagrams, int* nterms,
                     int* ncol) {
  if (!pr) return MGX_ERR_INVALID_ARGUMENT;
  if (npar) *npar = pr->prog->npar;
  if (nhel) *nhel = pr->nhel;
  if (ngood) *ngood = (int)pr->good.size();
  if (ndiagrams) *ndiagrams = pr->prog->ndiag;
  if (nterms) *nterms = pr->prog->nterm;
  if (ncol) *ncol = pr->prog->ncol;
  return MGX_OK;
}

int mgx_good_helicities(const mgx_process* pr, int32_t* out) {
  if (!pr || !out) return MGX_ERR_INVALID_ARGUMENT;
  for (size_t i = 0; i < pr->good.size(); ++i) out[i] = pr->good[i];
  return MGX_OK;
}

int mgx_colour_matrix(const mgx_process* pr, double* out) {
  if (!pr || !out) return MGX_ERR_INVALID_ARGUMENT;
  std::copy(pr->colour.begin(), pr->colour.end(), out);
  return MGX_OK;
}

int mgx_workspace_bytes(const mgx_process* pr, int64_t nevt, int mode, size_t* bytes) {
  if (!pr || !bytes || nevt < 0) return MGX_ERR_INVALID_ARGUMENT;
  if (!mode_ok(mode)) return MGX_ERR_UNSUPPORTED_MODE;
  if (mode_tc(mode)) {
    *bytes = nevt == 0 ? 0 : (size_t)grid_threads(pr, nevt) * thread_ws_bytes(pr->kp, MGX_FP64);
    return MGX_OK;
  }
  HelPlan hp;
  if (nevt > 0 && use_hel_kernel(pr, pr->kp, nevt, mode, &hp)) {
    *bytes = hel_layout(pr, pr->kp, hp, nevt, mode, grid_threads(pr, plan_items(hp, nevt), mode)).total;
    return MGX_OK;
  }
  *bytes = (nevt == 0 || use_cta_kernel(pr, pr->kp, nevt, mode) || use_smem_ws(pr, pr->kp, nevt, mode))
               ? 0
               : (size_t)grid_threads(pr, nevt, mode) * thread_ws_bytes(pr->kp, mode);
  return MGX_OK;
}

int mgx_compute_ex(mgx_process* pr, int64_t nevt, const double* momenta, const double* alpha_s,
                   const double* rnd_hel, const double* rnd_col, double* me, int32_t* selhel, int32_t* selcol,
                   double* mh, double* colw, int mode, void* workspace, size_t workspace_bytes, void* stream) {
  if (!pr || nevt < 0) return MGX_ERR_INVALID_ARGUMENT;
  if (!mode_ok(mode)) return MGX_ERR_UNSUPPORTED_MODE;
  if (nevt == 0) return MGX_OK;
  if (!momenta || !alpha_s || !me) return MGX_ERR_INVALID_ARGUMENT;
  if ((selhel && !rnd_hel) || (selcol && !rnd_col)) return MGX_ERR_INVALID_ARGUMENT;
  if (reinterpret_cast<uintptr_t>(momenta) % 16 != 0 || reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
    return MGX_ERR_INVALID_ARGUMENT;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return MGX_ERR_CUDA;
  if (cur != pr->device) return MGX_ERR_DEVICE_MISMATCH;
  return launch(pr, pr->kp, nevt, momenta, alpha_s, rnd_hel, rnd_col, me, selhel, selcol, mh, colw, mode, workspace,
                workspace_bytes, (cudaStream_t)stream);
}

int mgx_compute(mgx_process* pr, int64_t nevt, const double* momenta, const double* alpha_s, const double* rnd_hel,
                const double* rnd_col, double* me, int32_t* selhel, int32_t* selcol, int mode, void* workspace,
                size_t workspace_bytes, void* stream) {
  return mgx_compute_ex(pr, nevt, momenta, alpha_s, rnd_hel, rnd_col, me, selhel, selcol, nullptr, nullptr, mode,
                        workspace, workspace_bytes, stream);
}

int mgx_host_workspace_bytes(const mgx_process* pr, int64_t nevt, int mode, size_t* bytes) {
  size_t ws = 0;
  const int rc = mgx_workspace_bytes(pr, nevt, mode, &ws);
  if (rc != MGX_OK) return rc;
  const size_t n = (size_t)nevt;
  *bytes = align256(n * 4 * pr->prog->npar * 8) + 3 * align256(n * 8) + align256(n * 8) + 2 * align256(n * 4) +
           align256(ws);
  return MGX_OK;
}

int mgx_compute_host(mgx_process* pr, int64_t nevt, const double* momenta, const double* alpha_s,
                     const double* rnd_hel, const double* rnd_col, double* me, int32_t* selhel, int32_t* selcol,
                     int mode, void* workspace, size_t workspace_bytes, void* stream) {
  if (!pr || nevt < 0) return MGX_ERR_INVALID_ARGUMENT;
  size_t need = 0;
  int rc = mgx_host_workspace_bytes(pr, nevt, mode, &need);
  if (rc != MGX_OK) return rc;
  if (nevt == 0) return MGX_OK;
  if (!momenta || !alpha_s || !me || (selhel && !rnd_hel) || (selcol && !rnd_col)) return MGX_ERR_INVALID_ARGUMENT;
  if (workspace_bytes < need || !workspace || reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
    return MGX_ERR_WORKSPACE_TOO_SMALL;
  const size_t n = (size_t)nevt;
  char* p = (char*)workspace;
  double* d_mom = (double*)p; p += align256(n * 4 * pr->prog->npar * 8);
  double* d_as = (double*)p; p += align256(n * 8);
  double* d_rh = (double*)p; p += align256(n * 8);
  double* d_rc = (double*)p; p += align256(n * 8);
  double* d_me = (double*)p; p += align256(n * 8);
  int32_t* d_sh = (int32_t*)p; p += align256(n * 4);
  int32_t* d_sc = (int32_t*)p; p += align256(n * 4);
  void* d_ws = p;
  const size_t wsb = workspace_bytes - (size_t)(p - (char*)workspace);
  cudaStream_t st = (cudaStream_t)stream;
  bool ok = cudaMemcpyAsync(d_mom, momenta, n * 4 * pr->prog->npar * 8, cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(d_as, alpha_s, n * 8, cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (ok && selhel) ok = cudaMemcpyAsync(d_rh, rnd_hel, n * 8, cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (ok && selcol) ok = cudaMemcpyAsync(d_rc, rnd_col, n * 8, cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (!ok) return MGX_ERR_CUDA;
  rc = mgx_compute(pr, nevt, d_mom, d_as, d_rh, d_rc, d_me, selhel ? d_sh : nullptr, selcol ? d_sc : nullptr, mode,
                   d_ws, wsb, stream);
  if (rc != MGX_OK) return rc;
  ok = cudaMemcpyAsync(me, d_me, n * 8, cudaMemcpyDeviceToHost, st) == cudaSuccess;
  if (ok && selhel) ok = cudaMemcpyAsync(selhel, d_sh, n * 4, cudaMemcpyDeviceToHost, st) == cudaSuccess;
  if (ok && selcol) ok = cudaMemcpyAsync(selcol, d_sc, n * 4, cudaMemcpyDeviceToHost, st) == cudaSuccess;
  ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
  return ok ? MGX_OK : MGX_ERR_CUDA;
}

int mgx_process_set_kernel(mgx_process* pr, int kernel) {
  if (!pr || kernel < MGX_KERNEL_AUTO || kernel > MGX_KERNEL_SPLIT) return MGX_ERR_INVALID_ARGUMENT;
  if (kernel == MGX_KERNEL_CTA && !cta_usable(pr, pr->kp)) return MGX_ERR_INVALID_ARGUMENT;
  if (kernel == MGX_KERNEL_THREAD_SMEM && !smem_usable(pr->kp, MGX_FP64)) return MGX_ERR_INVALID_ARGUMENT;
  pr->kernel = kernel;
  return MGX_OK;
}

int mgx_process_get_kernel(const mgx_process* pr) {
  if (!pr) return MGX_ERR_INVALID_ARGUMENT;
  if (use_cta(pr, pr->kp)) return MGX_KERNEL_CTA;
  if (pr->kernel == MGX_KERNEL_HELICITY || pr->kernel == MGX_KERNEL_SPLIT) return pr->kernel;
  return pr->kernel == MGX_KERNEL_THREAD_SMEM ? MGX_KERNEL_THREAD_SMEM : MGX_KERNEL_THREAD;
}

int mgx_process_plan(const mgx_process* pr, int64_t nevt, int mode, int* kernel, int* groups, int* parts) {
  if (!pr || nevt < 0 || !mode_ok(mode)) return MGX_ERR_INVALID_ARGUMENT;
  int k = MGX_KERNEL_THREAD, g = 1, d = 1;
  HelPlan hp;
  if (nevt > 0 && !mode_tc(mode)) {
    if (use_cta_kernel(pr, pr->kp, nevt, mode)) k = MGX_KERNEL_CTA;
    else if (use_smem_ws(pr, pr->kp, nevt, mode)) k = MGX_KERNEL_THREAD_SMEM;
    else if (use_hel_kernel(pr, pr->kp, nevt, mode, &hp)) {
      k = hp.split ? MGX_KERNEL_SPLIT : MGX_KERNEL_HELICITY;
      g = 1 << hp.gshift;
      d = hp.nparts;
    }
  }
  if (kernel) *kernel = k;
  if (groups) *groups = g;
  if (parts) *parts = d;
  return MGX_OK;
}

int mgx_process_device_errors(mgx_process* pr, int* count, int reset) {
  if (!pr || !count) return MGX_ERR_INVALID_ARGUMENT;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return MGX_ERR_CUDA;
  if (cur != pr->device) return MGX_ERR_DEVICE_MISMATCH;
  if (cudaMemcpy(count, pr->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return MGX_ERR_CUDA;
  if (reset && cudaMemset(pr->d_status, 0, sizeof(int)) != cudaSuccess) return MGX_ERR_CUDA;
  return MGX_OK;
}

int mgx_process_set_tc_wait_test(mgx_process* pr, int skip_mma, double wait_ms) {
  if (!pr || wait_ms <= 0.0 || wait_ms > 10000.0) return MGX_ERR_INVALID_ARGUMENT;
  pr->tc_skip_mma = skip_mma ? 1 : 0;
  pr->tc_wait_ns = (unsigned long long)(wait_ms * 1e6);
  return MGX_OK;
}

int mgx_process_set_blocks_per_sm(mgx_process* pr, int blocks_per_sm) {
  if (!pr || blocks_per_sm < 1 || blocks_per_sm > 16) return MGX_ERR_INVALID_ARGUMENT;
  pr->blocks_per_sm = blocks_per_sm;
  return MGX_OK;
}

// Float64 work per event of the amplitude program, counted from the device code in
// mgx_ops.cuh: (fma, mul, add) instructions per variant / per good helicity of each op kind.
// Returns instructions (flops = false) or flops with an fma counted as 2 (flops = true).
static double fp64_work(const mgx_process* pr, int mode, bool flops) {
  const int* c = pr->prog->counts;
  const double ngood = (double)pr->good.size();
  const double n = pr->prog->ncol;
  struct K { double fma, mul, add; };
  const K ffv_f{48, 16, 0}, ffv_v{24, 24, 24}, bil{16, 16, 24}, rbil{24, 8, 0}, vvv{46, 10, 0},
      vvvv{24, 8, 0}, run{14, 2, 0}, term_add{0, 0, 8}, run_add{0, 0, 2}, flow{0, 0, 2},
      vvv_dot{6, 2, 0}, vvvv_dot{14, 4, 0}, slash{0, 0, 8}, slash_pref{8, 8, 0};
  auto w = [&](const K& k) { return flops ? 2 * k.fma + k.mul + k.add : k.fma + k.mul + k.add; };
  double t = w(ffv_f) * (c[0] + c[1]) + w(ffv_v) * c[2] + w(vvv) * c[3] + w(vvvv) * c[4] + w(bil) * c[5] +
             w(rbil) * c[6];
  // per good helicity: one product per run, a 4-vector add per further term of a run, an add per
  // further run of a group, and an add per (group, flow) except each flow's first (a write)
  const double flow_adds = c[9] - (pr->prog->jamp_zero ? 0.0 : n);
  t += ngood * (w(run) * c[11] + w(term_add) * (c[8] - c[11]) + w(run_add) * (c[11] - c[10]) + w(flow) * flow_adds);
  t += w(term_add) * c[12];                        // sum currents, per variant of their legs
  t += w(vvv_dot) * c[13] + w(vvvv_dot) * c[14];   // per-event child dot tables of VVV / VVVV
  t += w(slash) * c[15] + w(slash_pref) * c[16];  // per-event slash blocks of f f V vertices
  if (mode == MGX_FP64) t += ngood * (flops ? 2 * n * n + 4 * n : n * n + 3 * n);  // quadratic form
  else if (!flops) t += ngood * (mode_tc(mode) ? 4 * n : 2 * n);  // f64 -> f32 conversions (the tensor-core
                                                                   // colour sum converts for the stage and the dot)
  t += ngood * (flops ? 4 * n : 2 * n);                                             // colour weights
  return t;
}

int mgx_kernel_launches(const mgx_process* pr, int64_t nevt, int mode) {
  if (!pr || nevt < 0 || !mode_ok(mode)) return -1;
  if (nevt == 0) return 0;
  HelPlan hp;
  if (!use_hel_kernel(pr, pr->kp, nevt, mode, &hp)) return 1;
  return hp.split ? 3 : 2;   // split, combine and finish kernels; or the helicity-parallel kernel and its finish
}

double mgx_fp64_ops_per_event(const mgx_process* pr, int mode) { return pr ? fp64_work(pr, mode, false) : 0.0; }

double mgx_fp64_flops_per_event(const mgx_process* pr, int mode) { return pr ? fp64_work(pr, mode, true) : 0.0; }

}  // extern "C"

// ------------------------------------------------------------------ batched launch and autotuning
struct mgx_batch {
  int device = 0;
  std::vector<mgx_process*> procs;
  int blocks_per_sm = 4;
  std::vector<int> epi;       // events per work item, per process
  int max_ws = 0, max_npar4 = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

constexpr int kBatchMaxBlocksPerSm = 4;

int batch_launch(mgx_batch* b, const mgx_batch_io* io, int mode, void* ws, size_t wsb, cudaStream_t st,
                 int blocks_per_sm, const int* epi) {
  const int n = (int)b->procs.size();
  BatchDesc D{};
  D.nproc = n;
  D.max_npar4 = b->max_npar4;
  D.item_start[0] = 0;
  for (int p = 0; p < n; ++p) {
    if (epi[p] < 1) return MGX_ERR_INVALID_ARGUMENT;
    D.epi[p] = epi[p];
    D.item_start[p + 1] = D.item_start[p] + (io[p].nevt + epi[p] - 1) / epi[p];
  }
  BatchIO ios[kMaxBatch];
  for (int p = 0; p < n; ++p) {
    if (io[p].nevt < 0 || (io[p].nevt > 0 && (!io[p].momenta || !io[p].alpha_s || !io[p].me))) return MGX_ERR_INVALID_ARGUMENT;
    if ((io[p].selhel && !io[p].rnd_hel) || (io[p].selcol && !io[p].rnd_col)) return MGX_ERR_INVALID_ARGUMENT;
    if (reinterpret_cast<uintptr_t>(io[p].momenta) % 16 != 0) return MGX_ERR_INVALID_ARGUMENT;
    ios[p] = BatchIO{io[p].nevt, io[p].momenta, io[p].alpha_s, io[p].rnd_hel, io[p].rnd_col, io[p].me, io[p].selhel,
                     io[p].selcol};
  }
  if (D.item_start[n] == 0) return MGX_OK;
  const int64_t nt = (int64_t)sm_count(b->device) * blocks_per_sm * kThreads;
  const size_t need = 256 + (size_t)nt * b->max_ws * sizeof(double);
  if (!ws || wsb < need || reinterpret_cast<uintptr_t>(ws) % 256 != 0) return MGX_ERR_WORKSPACE_TOO_SMALL;
  unsigned long long* counter = (unsigned long long*)ws;
  double* w = (double*)((char*)ws + 256);
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st) != cudaSuccess) return MGX_ERR_CUDA;
  static_assert(sizeof(BatchParams) + sizeof(BatchDesc) + 64 < 32000, "batch kernel parameters too large");
  BatchParams bp;
  for (int p = 0; p < n; ++p) {
    bp.kp[p] = b->procs[p]->kp;
    bp.io[p] = ios[p];
  }
  const size_t shm = (size_t)kThreads * b->max_npar4 * sizeof(double);
  batch_kernel<<<(unsigned)(nt / kThreads), kThreads, shm, st>>>(bp, D, counter, w, nt, mode);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

}  // namespace

extern "C" int mgx_batch_create(mgx_process* const* procs, int nproc, mgx_batch** out) {
  if (!procs || !out || nproc < 1 || nproc > kMaxBatch) return MGX_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  for (int p = 0; p < nproc; ++p)
    if (!procs[p] || procs[p]->device != procs[0]->device) return MGX_ERR_DEVICE_MISMATCH;
  mgx_batch* b = new mgx_batch();
  b->device = procs[0]->device;
  b->epi.assign(nproc, 512);
  for (int p = 0; p < nproc; ++p) {
    b->procs.push_back(procs[p]);
    b->max_ws = std::max(b->max_ws, procs[p]->kp.ws_doubles);
    b->max_npar4 = std::max(b->max_npar4, 4 * procs[p]->kp.npar);
  }
  *out = b;
  return MGX_OK;
}

extern "C" void mgx_batch_destroy(mgx_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  delete b;
}

extern "C" int mgx_batch_workspace_bytes(const mgx_batch* b, size_t* bytes) {
  if (!b || !bytes) return MGX_ERR_INVALID_ARGUMENT;
  *bytes = 256 + (size_t)sm_count(b->device) * kBatchMaxBlocksPerSm * kThreads * b->max_ws * sizeof(double);
  return MGX_OK;
}

extern "C" int mgx_batch_compute(mgx_batch* b, const mgx_batch_io* io, int mode, void* ws, size_t wsb, void* stream) {
  if (!b || !io) return MGX_ERR_INVALID_ARGUMENT;
  if (mode != MGX_FP64 && mode != MGX_MIXED_FP32) return MGX_ERR_UNSUPPORTED_MODE;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return MGX_ERR_CUDA;
  if (cur != b->device) return MGX_ERR_DEVICE_MISMATCH;
  return batch_launch(b, io, mode, ws, wsb, (cudaStream_t)stream, b->blocks_per_sm, b->epi.data());
}

extern "C" int mgx_batch_capture(mgx_batch* b, const mgx_batch_io* io, int mode, void* ws, size_t wsb, void* stream) {
  if (!b || !io || !stream) return MGX_ERR_INVALID_ARGUMENT;
  if (mode != MGX_FP64 && mode != MGX_MIXED_FP32) return MGX_ERR_UNSUPPORTED_MODE;
  cudaStream_t st = (cudaStream_t)stream;
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MGX_ERR_CUDA;
  const int rc = batch_launch(b, io, mode, ws, wsb, st, b->blocks_per_sm, b->epi.data());
  cudaGraph_t g = nullptr;
  const bool ended = cudaStreamEndCapture(st, &g) == cudaSuccess;
  if (rc != MGX_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (!ended || !g) return MGX_ERR_CUDA;
  b->graph = g;
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) return MGX_ERR_CUDA;
  return MGX_OK;
}

extern "C" int mgx_batch_replay(mgx_batch* b, void* stream) {
  if (!b || !b->exec) return MGX_ERR_INVALID_ARGUMENT;
  return cudaGraphLaunch(b->exec, (cudaStream_t)stream) == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}

extern "C" int mgx_batch_autotune(mgx_batch* b, const mgx_batch_io* io, int mode, void* ws, size_t wsb, void* stream,
                                  int* blocks_per_sm, int* events_per_item) {
  if (!b || !io) return MGX_ERR_INVALID_ARGUMENT;
  if (mode != MGX_FP64 && mode != MGX_MIXED_FP32) return MGX_ERR_UNSUPPORTED_MODE;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int n = (int)b->procs.size();
  // time one schedule: a warm-up launch, then two timed launches
  auto timed = [&](int bps, const std::vector<int>& epi, float* ms) -> int {
    int rc = batch_launch(b, io, mode, ws, wsb, st, bps, epi.data());
    if (rc != MGX_OK) return rc;
    cudaEventRecord(e0, st);
    for (int r = 0; r < 2; ++r) batch_launch(b, io, mode, ws, wsb, st, bps, epi.data());
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) return MGX_ERR_CUDA;
    cudaEventElapsedTime(ms, e0, e1);
    return MGX_OK;
  };
  float best = 1e30f;
  int bb = b->blocks_per_sm;
  std::vector<int> be = b->epi;
  int rc = MGX_OK;
  // a candidate replaces the incumbent only when at least 2% faster, so that schedules within the
  // timing noise of each other do not make the choice vary from run to run
  const float kGain = 0.98f;
  // stage 1: blocks per SM x one common work-item size
  for (int bps : {4, 3, 2})
    for (int e : {512, 128, 2048}) {
      std::vector<int> cand(n, e);
      float ms = 0.0f;
      if ((rc = timed(bps, cand, &ms)) != MGX_OK) break;
      if (ms < kGain * best) { best = ms; bb = bps; be = cand; }
    }
  // stage 2: each process's work-item size in turn, the others fixed
  for (int p = 0; p < n && rc == MGX_OK; ++p)
    for (int e : {64, 128, 256, 512, 1024, 2048, 4096}) {
      if (e == be[p]) continue;
      std::vector<int> cand = be;
      cand[p] = e;
      float ms = 0.0f;
      if ((rc = timed(bb, cand, &ms)) != MGX_OK) break;
      if (ms < kGain * best) { best = ms; be = cand; }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != MGX_OK) return rc;
  b->blocks_per_sm = bb;
  b->epi = be;
  if (blocks_per_sm) *blocks_per_sm = bb;
  if (events_per_item)
    for (int p = 0; p < n; ++p) events_per_item[p] = be[p];
  return MGX_OK;
}

extern "C" int mgx_process_autotune(mgx_process* pr, int64_t nevt, const double* momenta, const double* alpha_s,
                                    int mode, void* workspace, size_t workspace_bytes, void* stream, int* kernel,
                                    int* blocks_per_sm, double* me_scratch) {
  if (!pr || nevt <= 0 || !momenta || !alpha_s || !me_scratch) return MGX_ERR_INVALID_ARGUMENT;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  struct Cand { int kernel, bps; };
  std::vector<Cand> cands = {{MGX_KERNEL_THREAD, 2}, {MGX_KERNEL_THREAD, 4}};
  if (cta_usable(pr, pr->kp) && mode_f64(mode)) cands.push_back({MGX_KERNEL_CTA, 4});
  if (smem_usable(pr->kp, mode)) cands.push_back({MGX_KERNEL_THREAD_SMEM, 4});
  if (mode_f64(mode) || mode == MGX_FLOAT) {
    cands.push_back({MGX_KERNEL_HELICITY, 4});
    cands.push_back({MGX_KERNEL_SPLIT, 4});
  }
  const int save_k = pr->kernel, save_b = pr->blocks_per_sm;
  float best = 1e30f;
  Cand pick{save_k, save_b};
  for (const Cand& c : cands) {
    pr->kernel = c.kernel;
    pr->blocks_per_sm = c.bps;
    size_t need = 0;
    mgx_workspace_bytes(pr, nevt, mode, &need);
    if (need > workspace_bytes) continue;
    int rc = mgx_compute(pr, nevt, momenta, alpha_s, nullptr, nullptr, me_scratch, nullptr, nullptr, mode, workspace,
                         workspace_bytes, stream);
    if (rc != MGX_OK) continue;
    cudaEventRecord(e0, st);
    for (int r = 0; r < 2; ++r)
      mgx_compute(pr, nevt, momenta, alpha_s, nullptr, nullptr, me_scratch, nullptr, nullptr, mode, workspace,
                  workspace_bytes, stream);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; pick = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  pr->kernel = pick.kernel;
  pr->blocks_per_sm = pick.bps;
  if (kernel) *kernel = pick.kernel;
  if (blocks_per_sm) *blocks_per_sm = pick.bps;
  return best < 1e30f ? MGX_OK : MGX_ERR_CUDA;
}

// ------------------------------------------------------------------ allocation-free entry point
// Some callers cannot allocate device memory at the point where they evaluate matrix elements:
// a Fortran event-generation loop that links this library but has no CUDA allocator of its
// own, or a plugin running inside a host framework that owns the device memory pool and does
// not let third-party code call cudaMalloc.  For them mgx_compute_noalloc runs the
// thread-per-event kernel with its workspace in this fixed array instead of a caller buffer.
// The array is module-scope device memory: every GPU that loads the library holds it until the
// process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)128 << 20;   // 128 MiB
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchBytes / sizeof(double)];

static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[256] = {};   // device address of g_noalloc_scratch, per device ordinal

// Host code must not hand the array's name to a kernel (in host code it is a host-side
// stand-in, not a device address): look the device address up once per device, with that
// device current.
static int noalloc_scratch(int device, double** out) {
  if (device < 0 || device >= 256) return MGX_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) return MGX_ERR_CUDA;
    g_noalloc_ptr[device] = ptr;
  }
  *out = (double*)g_noalloc_ptr[device];
  return MGX_OK;
}

extern "C" size_t mgx_noalloc_scratch_bytes(void) { return kNoAllocScratchBytes; }

extern "C" int mgx_compute_noalloc(mgx_process* pr, int64_t nevt, const double* momenta, const double* alpha_s,
                                   const double* rnd_hel, const double* rnd_col, double* me, int32_t* selhel,
                                   int32_t* selcol, int mode, void* stream) {
  if (!pr || nevt < 0) return MGX_ERR_INVALID_ARGUMENT;
  if (mode != MGX_FP64 && mode != MGX_MIXED_FP32) return MGX_ERR_UNSUPPORTED_MODE;
  if (nevt == 0) return MGX_OK;
  if (!momenta || !alpha_s || !me) return MGX_ERR_INVALID_ARGUMENT;
  if ((selhel && !rnd_hel) || (selcol && !rnd_col)) return MGX_ERR_INVALID_ARGUMENT;
  if (reinterpret_cast<uintptr_t>(momenta) % 16 != 0) return MGX_ERR_INVALID_ARGUMENT;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return MGX_ERR_CUDA;
  if (cur != pr->device) return MGX_ERR_DEVICE_MISMATCH;
  // one 128-thread block needs 128 per-event workspaces; the grid is sized to fit the array
  const size_t per_block = (size_t)kThreads * pr->kp.ws_doubles * sizeof(double);
  if (per_block > kNoAllocScratchBytes) return MGX_ERR_WORKSPACE_TOO_SMALL;
  double* scratch = nullptr;
  const int rc = noalloc_scratch(cur, &scratch);
  if (rc != MGX_OK) return rc;
  const int64_t fit = (int64_t)(kNoAllocScratchBytes / per_block);
  const int64_t want = (nevt + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)sm_count(pr->device) * pr->blocks_per_sm;
  const int64_t blocks = std::max<int64_t>(1, std::min({fit, want, cap}));
  const int64_t nt = blocks * kThreads;
  const size_t shm = (size_t)kThreads * 4 * pr->kp.npar * sizeof(double);
  me_kernel<double, false><<<(unsigned)blocks, kThreads, shm, (cudaStream_t)stream>>>(
      pr->kp, nevt, momenta, alpha_s, rnd_hel, rnd_col, me, selhel, selcol, nullptr, nullptr, scratch, nt, mode);
  return cudaGetLastError() == cudaSuccess ? MGX_OK : MGX_ERR_CUDA;
}


