// mgx: C-ABI library for batched tree-level |M|^2 on one GB300 (sm_103a).
// Host API, helicity filter and the launch of the event-parallel kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cctype>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mgx.h"
#include "mgx_ops.cuh"

namespace {

struct mgx_program_desc {
  const char* name;
  int npar, nin, root, nops;
  const int32_t* ops;
  int nflows;
  const int32_t* flows;
  int ncol;
  const double* colour;
  int ncoupl;
  const double* coupl;   // (boson id, Q, T3) per entry
  int nmass;
  const int32_t* mass;   // (mass param, width param) per entry
  const int32_t* extmass;
  int ws_doubles, ndiag, nterm, avg_den;
  int counts[8];         // variants: ffv_f, ffv_fb, ffv_v, vvv, vvvv; current ops; amp ops; amp flows
};

#include "generated/programs.inc"

}  // namespace

using namespace mgx;

// ------------------------------------------------------------------ kernel
namespace {

constexpr int kThreads = 128;

__device__ inline void colour_stage(const KParams& P, const WS& W, int mode) {
  const int n = P.ncol;
  for (int ih = 0; ih < P.ngood; ++ih) {
    const int jb = P.jamp_off + 2 * n * ih;
    double mh;
    if (mode == MGX_MIXED_FP32) {
      float acc = 0.0f;
      for (int i = 0; i < n; ++i) {
        const float ri = (float)W[jb + 2 * i], ii = (float)W[jb + 2 * i + 1];
        const float* crow = P.colsym_f + i * n;
        float zr = __ldg(crow + i) * ri, zi = __ldg(crow + i) * ii;
        for (int j = i + 1; j < n; ++j) {
          const float c = __ldg(crow + j);
          zr = fmaf(c, (float)W[jb + 2 * j], zr);
          zi = fmaf(c, (float)W[jb + 2 * j + 1], zi);
        }
        acc = fmaf(ri, zr, fmaf(ii, zi, acc));
      }
      mh = (double)acc;
    } else {
      double acc = 0.0;
      for (int i = 0; i < n; ++i) {
        const double ri = W[jb + 2 * i], ii = W[jb + 2 * i + 1];
        const double* crow = P.colsym + i * n;
        double zr = __ldg(crow + i) * ri, zi = __ldg(crow + i) * ii;
        for (int j = i + 1; j < n; ++j) {
          const double c = __ldg(crow + j);
          zr = fma(c, W[jb + 2 * j], zr);
          zi = fma(c, W[jb + 2 * j + 1], zi);
        }
        acc = fma(ri, zr, fma(ii, zi, acc));
      }
      mh = acc;
    }
    W[P.mh_off + ih] = mh;
  }
}

__global__ void __launch_bounds__(kThreads)
    me_kernel(const KParams P, int64_t nevt, const double* __restrict__ mom, const double* __restrict__ alphas,
              const double* __restrict__ rhel, const double* __restrict__ rcol, double* __restrict__ me,
              int32_t* __restrict__ selhel, int32_t* __restrict__ selcol, double* __restrict__ mh_out,
              double* __restrict__ colw_out, double* __restrict__ ws, int64_t nthreads, int mode) {
  extern __shared__ double smem[];
  const int npar4 = 4 * P.npar;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const WS W{ws + tid, nthreads};
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nevt; base += nthreads) {
    // stage this block's momenta (contiguous [events][npar][4]) through shared memory
    const int64_t nb = min((int64_t)blockDim.x, nevt - base);
    const double2* src = reinterpret_cast<const double2*>(mom + base * npar4);
    double2* dst = reinterpret_cast<double2*>(smem);
    __syncthreads();
    for (int i = threadIdx.x; i < (int)(nb * npar4 / 2); i += blockDim.x) dst[i] = __ldg(src + i);
    __syncthreads();
    const int64_t e = base + threadIdx.x;
    if (e >= nevt) continue;
    const double* pe = smem + threadIdx.x * npar4;
    const double gs = sqrt(4.0 * M_PI * alphas[e]);
    for (int i = 0; i < 2 * P.ncol * P.ngood; ++i) W[P.jamp_off + i] = 0.0;
    for (int iop = 0; iop < P.nops; ++iop) {
      const Op o = load_op(P.ops, iop);
      switch (o.code) {
        case OP_EXT: op_ext(P, o, pe, W); break;
        case OP_FFV_F: op_ffv_f(P, o, gs, W); break;
        case OP_FFV_FB: op_ffv_fb(P, o, gs, W); break;
        case OP_FFV_V: op_ffv_v(P, o, gs, W); break;
        case OP_VVV: op_vvv(P, o, gs, W); break;
        case OP_VVVV: op_vvvv(P, o, gs, W); break;
        default: op_amp(P, o, gs, W); break;
      }
    }
    colour_stage(P, W, mode);
    // helicity sum (float64, canonical order) and selections
    double tot = 0.0;
    for (int ih = 0; ih < P.ngood; ++ih) tot += W[P.mh_off + ih];
    me[e] = tot * P.avg;
    if (mh_out)
      for (int ih = 0; ih < P.ngood; ++ih) mh_out[e * P.ngood + ih] = W[P.mh_off + ih];
    const bool want_col = (selcol != nullptr) || (colw_out != nullptr);
    if (want_col) {
      for (int i = 0; i < P.ncol; ++i) {
        double w = 0.0;
        for (int ih = 0; ih < P.ngood; ++ih) {
          const int jb = P.jamp_off + 2 * P.ncol * ih + 2 * i;
          w = fma(W[jb], W[jb], fma(W[jb + 1], W[jb + 1], w));
        }
        W[P.colw_off + i] = w;
        if (colw_out) colw_out[e * P.ncol + i] = w;
      }
    }
    if (selhel) {
      const double target = rhel[e] * tot;
      double acc = 0.0;
      int sel = P.good[P.ngood - 1];
      for (int ih = 0; ih < P.ngood; ++ih) {
        acc += W[P.mh_off + ih];
        if (acc > target) { sel = P.good[ih]; break; }
      }
      selhel[e] = sel;
    }
    if (selcol) {
      double wt = 0.0;
      for (int i = 0; i < P.ncol; ++i) wt += W[P.colw_off + i];
      const double target = rcol[e] * wt;
      double acc = 0.0;
      int sel = P.ncol - 1;
      for (int i = 0; i < P.ncol; ++i) {
        acc += W[P.colw_off + i];
        if (acc > target) { sel = i; break; }
      }
      selcol[e] = sel;
    }
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
  int blocks_per_sm = 1;
};

namespace {

int64_t grid_threads(const mgx_process* pr, int64_t nevt) {
  const int64_t cap = (int64_t)sm_count(pr->device) * pr->blocks_per_sm * kThreads;
  const int64_t need = ((nevt + kThreads - 1) / kThreads) * kThreads;
  return std::max<int64_t>(kThreads, std::min(cap, need));
}

int64_t ws_doubles_per_thread(const KParams& kp) { return kp.ws_doubles; }

void set_layout(KParams& kp, int cur_doubles, int ngood, int ncol) {
  kp.cur_doubles = cur_doubles;
  kp.jamp_off = cur_doubles;
  kp.mh_off = kp.jamp_off + 2 * ncol * ngood;
  kp.colw_off = kp.mh_off + ngood;
  kp.ws_doubles = kp.colw_off + ncol;
}

int launch(mgx_process* pr, const KParams& kp, int64_t nevt, const double* mom, const double* as,
           const double* rh, const double* rc, double* me, int32_t* sh, int32_t* sc, double* mh, double* cw,
           int mode, void* ws, size_t wsb, cudaStream_t st) {
  if (nevt == 0) return MGX_OK;
  const int64_t nt = grid_threads(pr, nevt);
  const size_t need = (size_t)nt * ws_doubles_per_thread(kp) * sizeof(double);
  if (wsb < need || ws == nullptr) return MGX_ERR_WORKSPACE_TOO_SMALL;
  const int blocks = (int)(nt / kThreads);
  const size_t shm = (size_t)kThreads * 4 * kp.npar * sizeof(double);
  me_kernel<<<blocks, kThreads, shm, st>>>(kp, nevt, mom, as, rh, rc, me, sh, sc, mh, cw, (double*)ws, nt, mode);
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
  bool ok = cudaMalloc(&pr->d_ops, sizeof(int32_t) * 16 * prog->nops) == cudaSuccess &&
            cudaMalloc(&pr->d_flows, sizeof(int2) * std::max(1, prog->nflows)) == cudaSuccess &&
            cudaMalloc(&pr->d_col, sizeof(double) * n * n) == cudaSuccess &&
            cudaMalloc(&pr->d_colf, sizeof(float) * n * n) == cudaSuccess;
  ok = ok && cudaMemcpy(pr->d_ops, prog->ops, sizeof(int32_t) * 16 * prog->nops, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(pr->d_flows, prog->flows, sizeof(int32_t) * 2 * prog->nflows, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(pr->d_col, cs.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(pr->d_colf, csf.data(), sizeof(float) * n * n, cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    mgx_process_destroy(pr);
    cudaSetDevice(cur);
    return MGX_ERR_CUDA;
  }
  kp.ops = pr->d_ops;
  kp.flows = pr->d_flows;
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
  for (int h = 0; h < pr->nhel; ++h) fk.good[h] = h;
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
  if (ok) rc = launch(pr, fk, nf, d_mom, d_as, nullptr, nullptr, d_me, nullptr, nullptr, d_mh, nullptr, MGX_FP64, d_ws, wsb, 0);
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
  for (int i = 0; i < kp.ngood; ++i) kp.good[i] = pr->good[i];
  set_layout(kp, prog->ws_doubles, kp.ngood, n);
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
  if (mode != MGX_FP64 && mode != MGX_MIXED_FP32) return MGX_ERR_UNSUPPORTED_MODE;
  *bytes = nevt == 0 ? 0 : (size_t)grid_threads(pr, nevt) * pr->kp.ws_doubles * sizeof(double);
  return MGX_OK;
}

int mgx_compute_ex(mgx_process* pr, int64_t nevt, const double* momenta, const double* alpha_s,
                   const double* rnd_hel, const double* rnd_col, double* me, int32_t* selhel, int32_t* selcol,
                   double* mh, double* colw, int mode, void* workspace, size_t workspace_bytes, void* stream) {
  if (!pr || nevt < 0) return MGX_ERR_INVALID_ARGUMENT;
  if (mode != MGX_FP64 && mode != MGX_MIXED_FP32) return MGX_ERR_UNSUPPORTED_MODE;
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

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

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

double mgx_fp64_ops_per_event(const mgx_process* pr, int mode) {
  if (!pr) return 0.0;
  // float64 instruction counts per variant / per good helicity of each op kind, read off the
  // device code in mgx_ops.cuh (fma, mul and add each count as one operation)
  const int* c = pr->prog->counts;
  const double ngood = (double)pr->good.size();
  const int n = pr->prog->ncol;
  double ops = 96.0 * c[0] + 96.0 * c[1] + 80.0 * c[2] + 70.0 * c[3] + 60.0 * c[4];
  ops += ngood * (60.0 * c[6] + 2.0 * c[7]);
  if (mode == MGX_FP64) ops += ngood * (2.0 * n * (n + 1) + 2.0);
  return ops;
}

}  // extern "C"
