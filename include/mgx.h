/*
 * mgx — batched tree-level squared matrix elements on one GB300 (sm_103a).
 *
 * C ABI of the event-parallel matrix-element library.  The operation is the
 * third step of the matrix-element generator chain of arXiv:2503.21935, Sec. 2
 * (random numbers -> phase-space momenta -> matrix element), exposed through
 * the multi-event interface the paper describes in Sec. 2: reentrant, stateless
 * compute calls with well-defined input and output buffers for a whole batch
 * of events.  For each event the library returns the spin- and colour-averaged
 * |M|^2 summed over the non-vanishing helicities (Feynman diagrams in double
 * precision, followed by the colour-matrix quadratic form J^dagger C J, Sec. 3),
 * plus one helicity and one colour flow selected from per-event random numbers.
 *
 * Conventions
 *   - Momenta: float64, layout [nevt][npar][4] = (E, px, py, pz) in GeV, the
 *     particles in process-string order (two incoming partons first).
 *   - Helicity index h in [0, 2^npar): bit (npar-1-p) of h is 1 when particle p
 *     has helicity +1 and 0 for -1 (particle 0 varies slowest).
 *   - Colour flows: the strings (T^{a_s1} ... T^{a_sn})_{ij} over the permutations
 *     s of the gluon legs in lexicographic order, i the colour of the fermion line's
 *     barred end (an outgoing quark or incoming antiquark), j of its other end.
 *   - me = 1/(4 * Ncol_in * S) * sum_h sum_colours |M|^2, with S the product of
 *     n! over identical final-state particles.
 *   - selected helicity: smallest canonical h whose cumulative |M_h|^2 (canonical
 *     order) exceeds rnd_hel * total; selected colour: smallest flow s whose
 *     cumulative w_s exceeds rnd_col * sum(w), w_s = sum_h |J_s(h)|^2.
 *
 * Ownership: the caller owns every buffer passed to mgx_compute (device
 * pointers) and the workspace; the library owns only the process handle.
 * Errors: every call returns MGX_OK (0) or a negative mgx_status; nothing
 * throws across the ABI.  mgx_compute is asynchronous on the given stream and
 * performs no allocation and no host synchronisation.
 */
#ifndef MGX_H
#define MGX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mgx_process mgx_process; /* opaque, library-owned */

enum mgx_status {
  MGX_OK = 0,
  MGX_ERR_INVALID_ARGUMENT = -1,
  MGX_ERR_UNKNOWN_PROCESS = -2,
  MGX_ERR_CUDA = -3,
  MGX_ERR_DEVICE_MISMATCH = -4,
  MGX_ERR_WORKSPACE_TOO_SMALL = -5,
  MGX_ERR_NO_GOOD_HELICITY = -6,
  MGX_ERR_UNSUPPORTED_MODE = -7
};

/* Arithmetic precision (Sec. 3: the double, float and "mixed" builds; mixed computes the
 * diagrams in double precision and the colour-matrix quadratic form in single precision).
 * The helicity sum and the selections are float64 in every mode. */
enum mgx_mode {
  MGX_FP64 = 0,       /* float64 amplitudes and colour sum */
  MGX_MIXED_FP32 = 1, /* float64 amplitudes; jamps rounded to float32, float32 quadratic form */
  MGX_MIXED_TF32 = 2, /* float64 amplitudes; tensor-core colour sum (tcgen05, fused into the
                         thread-per-event kernel): jamps rounded to float32 and split into two tf32
                         terms times the integer-scaled colour matrix (exact in tf32), float32
                         accumulation */
  MGX_MIXED_BF16X3 = 3, /* float64 amplitudes; tensor-core colour sum in bf16: jamps split into three
                         bf16 terms, the integer-scaled colour matrix into two (exact below 2^16;
                         otherwise MGX_ERR_UNSUPPORTED_MODE), float32 accumulation */
  MGX_FLOAT = 4       /* float32 amplitudes and colour sum (the paper's float build); thread-per-
                         event kernel only */
};

/* Standard-Model inputs.  Electroweak scheme {alpha_em(mZ), G_F, mZ}. */
typedef struct mgx_params {
  double mt, wt;       /* top mass and width [GeV] */
  double mz, wz;       /* Z mass and width [GeV] */
  double mta;          /* tau mass [GeV] */
  double alpha_em;     /* 1/132.507 */
  double gf;           /* Fermi constant [GeV^-2] */
  double filter_sqrt_s;/* partonic energy of the helicity-filter events [GeV]; <= 0: 1000 */
} mgx_params;

/* Fill *p with the default parameters (mt 173, wt 1.4915, mz 91.1876,
 * wz 2.4414, mta 1.777, alpha 1/132.507, G_F 1.16639e-5). */
void mgx_params_default(mgx_params* p);

/* Number of built-in processes and the process string of entry i (NULL if out
 * of range).  Strings use the names e+ e- mu+ mu- ta+ ta- u u~ t t~ g. */
int mgx_num_processes(void);
const char* mgx_process_name(int i);

/* Create a process on CUDA device `device`: the set-up half of the multi-event ME interface of
 * Sec. 2 (a process with its couplings and masses is prepared once, then evaluated for many event
 * batches; the paper does not describe the helicity filter, which drops the helicities whose
 * |M_h|^2 vanishes identically so that no batch evaluates them).  Resolves the couplings and masses,
 * uploads the process's op table and colour matrix, and runs the helicity
 * filter: all 2^npar helicities are evaluated on 16 flat phase-space events
 * (Philox-4x32-10 keyed by filter_seed, RAMBO at params->filter_sqrt_s) and
 * those with |M_h|^2 == 0 on every event are dropped.  Synchronous.
 * process: e.g. "g g > t t~ g g" (whitespace-insensitive).  params may be NULL
 * for the defaults.  On success *out receives a handle to free with
 * mgx_process_destroy.  Errors: INVALID_ARGUMENT (NULL out, bad device),
 * UNKNOWN_PROCESS, CUDA, NO_GOOD_HELICITY. */
int mgx_process_create(const char* process, const mgx_params* params, int device,
                       uint64_t filter_seed, mgx_process** out);

/* Sizes of a process: particles, helicities before/after the filter, Feynman
 * diagrams, diagram terms (one per colour structure of each four-gluon vertex)
 * and colour flows.  Any pointer may be NULL. */
int mgx_process_info(const mgx_process* proc, int* npar, int* nhel, int* ngood,
                     int* ndiagrams, int* nterms, int* ncol);

/* Copy the canonical indices of the good helicities (ascending) to host array
 * out[ngood]. */
int mgx_good_helicities(const mgx_process* proc, int32_t* out);

/* Copy the float64 colour matrix to host array out[ncol*ncol] (row-major). */
int mgx_colour_matrix(const mgx_process* proc, double* out);

/* Device workspace (bytes) that mgx_compute needs for nevt events in `mode`. */
int mgx_workspace_bytes(const mgx_process* proc, int64_t nevt, int mode, size_t* bytes);

/* Compute a batch: the reentrant, stateless multi-event ME call of Sec. 2 (well-defined input and
 * output buffers for a whole batch of events), evaluating per event the Feynman diagrams, the
 * colour-matrix quadratic form J^dagger C J and the helicity sum of Sec. 3, plus the helicity and
 * colour selection that the event record needs.  All arrays are DEVICE pointers on the process's device:
 *   momenta [nevt][npar][4] f64, alpha_s [nevt] f64, rnd_hel/rnd_col [nevt] f64 in [0,1)
 *   outputs me [nevt] f64, selhel [nevt] i32 (canonical helicity index),
 *           selcol [nevt] i32 (colour-flow index).
 * rnd_hel/rnd_col/selhel/selcol may all be NULL to skip selection.
 * workspace: device buffer of at least mgx_workspace_bytes(nevt, mode) bytes
 * (256-byte aligned; may be NULL when that is 0, as for the small batches that AUTO runs
 * one block per event or with the workspace in shared memory); stream: a cudaStream_t
 * (NULL = legacy default stream).
 * Asynchronous; errors: INVALID_ARGUMENT, DEVICE_MISMATCH, WORKSPACE_TOO_SMALL,
 * UNSUPPORTED_MODE, CUDA (launch failure). */
int mgx_compute(mgx_process* proc, int64_t nevt, const double* momenta, const double* alpha_s,
                const double* rnd_hel, const double* rnd_col, double* me, int32_t* selhel,
                int32_t* selcol, int mode, void* workspace, size_t workspace_bytes, void* stream);

/* As mgx_compute, with optional extra DEVICE outputs (each may be NULL):
 *   mh   [nevt][ngood] f64: colour-summed |M_h|^2 per good helicity (not averaged)
 *   colw [nevt][ncol]  f64: colour-selection weights w_s = sum_h |J_s(h)|^2. */
int mgx_compute_ex(mgx_process* proc, int64_t nevt, const double* momenta, const double* alpha_s,
                   const double* rnd_hel, const double* rnd_col, double* me, int32_t* selhel,
                   int32_t* selcol, double* mh, double* colw, int mode, void* workspace,
                   size_t workspace_bytes, void* stream);

/* End-to-end variant with HOST buffers (pinned memory recommended): copies the
 * inputs to the device, computes, copies me/selhel/selcol back and
 * synchronises the stream.  The device workspace must hold
 * mgx_host_workspace_bytes(nevt, mode) bytes (staging + compute workspace). */
int mgx_host_workspace_bytes(const mgx_process* proc, int64_t nevt, int mode, size_t* bytes);
int mgx_compute_host(mgx_process* proc, int64_t nevt, const double* momenta, const double* alpha_s,
                     const double* rnd_hel, const double* rnd_col, double* me, int32_t* selhel,
                     int32_t* selcol, int mode, void* workspace, size_t workspace_bytes,
                     void* stream);

/* Kernel variant (for tuning and testing).  THREAD: one thread per event, current variants
 * and jamps in the global workspace (what AUTO resolves to for throughput batches).  CTA: one
 * thread block per event with the event's currents in shared memory; available when the
 * process's current store fits in shared memory and ncol <= 32 (MGX_FP64, MGX_MIXED_FP32), and
 * what AUTO picks in those modes for a batch too small to fill the thread kernel's grid: at most
 * 32 events per SM, or 8 per SM for a process that has THREAD_SMEM (no caller workspace needed).
 * THREAD_SMEM: the thread-per-event kernel with each thread's workspace in shared memory
 * (64 threads per block, no caller workspace needed); available for small processes (e+ e- >
 * mu+ mu-, g g > t t~), and what AUTO picks otherwise when the whole batch fits one block per SM
 * (a latency-bound batch).  HELICITY: the helicity-parallel mapping (Sec. 2: different helicity
 * combinations of one event processed in parallel, so that far fewer events fill the GPU): the
 * helicities are split into 2^k groups by their values on k fixed particles, one thread per
 * (event, group) computes the current variants and amplitudes its group uses, and a second kernel
 * sums each event's helicities in canonical order and selects; the fixed particles and k come
 * from a work model of the op table (MGX_FP64, MGX_MIXED_FP32, MGX_FLOAT).  SPLIT: the diagram
 * split: the process compiler cuts the amplitude groups into 2, 4 or 8 contiguous parts, each with
 * the current ops its terms need; one thread per (event, helicity group, part) writes partial
 * jamps, a combine kernel sums them per (event, helicity) and forms the colour sum, and the finish
 * kernel selects (same modes; the split and the fixed particles from the same work model).  AUTO
 * takes HELICITY or SPLIT for a batch that leaves the thread kernel's grid underfilled when that
 * model predicts at least a 1.1x gain and the batch is too large for CTA / THREAD_SMEM.  All give
 * identical results up to float64 rounding. */
enum mgx_kernel { MGX_KERNEL_AUTO = 0, MGX_KERNEL_THREAD = 1, MGX_KERNEL_CTA = 2, MGX_KERNEL_THREAD_SMEM = 3,
                  MGX_KERNEL_HELICITY = 4, MGX_KERNEL_SPLIT = 5 };
int mgx_process_set_kernel(mgx_process* proc, int kernel);  /* INVALID_ARGUMENT if unusable */
/* The kernel a compute of nevt events in `mode` runs with the current settings (AUTO resolved), and
 * for HELICITY / SPLIT the number of helicity groups and diagram parts per event (else 1, 1). */
int mgx_process_plan(const mgx_process* proc, int64_t nevt, int mode, int* kernel, int* groups, int* parts);
/* the kernel set; for AUTO, THREAD (the choice for throughput batches; AUTO picks CTA or
 * THREAD_SMEM per call for small batches, as above) */
int mgx_process_get_kernel(const mgx_process* proc);
/* Thread blocks of 128 threads per SM for the thread-per-event kernel (1..16, default 4; the
 * float mode launches twice as many, its kernel having half the registers); the workspace
 * size grows with it.  The CTA-per-event kernel serves MGX_FP64 and MGX_MIXED_FP32 only. */
int mgx_process_set_blocks_per_sm(mgx_process* proc, int blocks_per_sm);

/* ---- batched multi-process launch (one persistent kernel over several processes) ----
 * Work items of events_per_item events of one process are numbered process after process and
 * taken from a device counter by the CTAs of one persistent grid (no waits), so processes with
 * very different event counts and costs share the GPU in one launch.  Results are identical to
 * per-process mgx_compute (each event is evaluated by the same code). */
typedef struct mgx_batch mgx_batch;
typedef struct mgx_batch_io {
  int64_t nevt;
  const double* momenta;  /* DEVICE [nevt][npar][4] */
  const double* alpha_s;  /* DEVICE [nevt] */
  const double* rnd_hel;  /* DEVICE [nevt] or NULL */
  const double* rnd_col;  /* DEVICE [nevt] or NULL */
  double* me;             /* DEVICE [nevt] */
  int32_t* selhel;        /* DEVICE [nevt] or NULL */
  int32_t* selcol;        /* DEVICE [nevt] or NULL */
} mgx_batch_io;
/* procs[nproc] (1..16) on one device; the handles must outlive the batch. */
int mgx_batch_create(mgx_process* const* procs, int nproc, mgx_batch** out);
void mgx_batch_destroy(mgx_batch* batch);
/* DEVICE workspace bytes (independent of the event counts). */
int mgx_batch_workspace_bytes(const mgx_batch* batch, size_t* bytes);
/* io[nproc], one entry per process in creation order; modes MGX_FP64 / MGX_MIXED_FP32. Async. */
int mgx_batch_compute(mgx_batch* batch, const mgx_batch_io* io, int mode, void* workspace, size_t workspace_bytes,
                      void* stream);
/* Capture the batched launch (counter reset + kernel) for these buffers into a CUDA graph owned
 * by the batch (stream must not be the legacy default stream); mgx_batch_replay launches it. */
int mgx_batch_capture(mgx_batch* batch, const mgx_batch_io* io, int mode, void* workspace, size_t workspace_bytes,
                      void* stream);
int mgx_batch_replay(mgx_batch* batch, void* stream);
/* Autotuner: times the batched launch on these buffers, first for blocks per SM in {2, 3, 4} x
 * one common work-item size in {128, 512, 2048}, then each process's own work-item size in
 * {64, ..., 4096} in turn with the others fixed; keeps the fastest schedule for later launches
 * and captures.  events_per_item: NULL or [nproc] (the chosen size per process).  Synchronous. */
int mgx_batch_autotune(mgx_batch* batch, const mgx_batch_io* io, int mode, void* workspace,
                       size_t workspace_bytes, void* stream, int* blocks_per_sm, int* events_per_item);
/* Autotuner of a single process: times mgx_compute on these inputs for the thread-per-event
 * kernel at 2 and 4 blocks per SM, the CTA-per-event kernel and the shared-memory thread kernel
 * (each when usable), keeps the fastest (me_scratch: DEVICE [nevt] output buffer).  Query
 * mgx_workspace_bytes again afterwards.  Synchronous. */
int mgx_process_autotune(mgx_process* proc, int64_t nevt, const double* momenta, const double* alpha_s, int mode,
                         void* workspace, size_t workspace_bytes, void* stream, int* kernel, int* blocks_per_sm,
                         double* me_scratch);

/* Failure detection of the tensor-core colour sum (modes MGX_MIXED_TF32, MGX_MIXED_BF16X3).  Every
 * wait of a block for its own tensor-core work has a time limit; when one runs out, the block adds 1
 * to the process's device error counter, writes NaN to me (and -1 to the selections) of its events
 * from then on, and stops using the tensor cores, so a stuck colour sum shows as NaN, never as a
 * hang or a wrong number.  mgx_process_device_errors copies the counter to *count (synchronous:
 * call it after the computes it should cover have completed) and zeroes it when reset != 0. */
int mgx_process_device_errors(mgx_process* proc, int* count, int reset);
/* Test hook for that path: with skip_mma != 0 the tensor-core colour sum issues no MMA, so each of
 * its waits runs out after wait_ms (0 < wait_ms <= 10000; the default limit is 1000 ms); nothing is
 * in flight when the block frees its tensor memory.  skip_mma = 0 restores normal operation. */
int mgx_process_set_tc_wait_test(mgx_process* proc, int skip_mma, double wait_ms);

/* Float64 work per event of this process in `mode`, from the op table and per-op
 * instruction counts of the device code: instructions (add, multiply and fused
 * multiply-add each one) and flops (a fused multiply-add counted as two).  Used for
 * roofline reporting. */
double mgx_fp64_ops_per_event(const mgx_process* proc, int mode);
double mgx_fp64_flops_per_event(const mgx_process* proc, int mode);

/* Number of this library's kernels one mgx_compute of nevt events in `mode` launches with the
 * process's current settings (1: every mode, the tensor-core colour sums included, is one fused
 * kernel); -1 on invalid arguments. */
int mgx_kernel_launches(const mgx_process* proc, int64_t nevt, int mode);

/* Allocation-free variant of mgx_compute.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory where they evaluate matrix elements,
 * e.g. a Fortran event-generation loop with no CUDA allocator of its own, or a plugin inside a
 * host framework that owns the device memory pool and forbids cudaMalloc from third-party code.
 * Arguments are those of mgx_compute without the workspace (DEVICE pointers; the caller still
 * passes every input and output).  The thread-per-event kernel's workspace lives in one fixed
 * module-scope device array of mgx_noalloc_scratch_bytes() = 128 MiB, which every GPU that
 * loads the library holds until the process exits; the grid is sized so the workspace fits, i.e.
 * floor(128 MiB / (128 x per-event workspace)) blocks of 128 threads, at most the usual persistent
 * grid: g g > t t~ g g gets 12 blocks (1536 events in flight instead of 77824), g g > t t~ g g g
 * a single block (128 events in flight), so their throughput through this entry point is
 * about 1/50 and 1/600 of mgx_compute's on a full batch; the small processes get the full grid.
 * The call itself allocates nothing (no cudaMalloc/cudaFree, no allocating library call); the
 * process handle must have been created beforehand.  Set-up: the first call on a device looks
 * up the array's device address with that device current, so make that first call before any
 * stream capture.  The kernel initialises everything it reads (including the jamp
 * accumulators) for every event, so no clearing is needed between calls; but every call shares
 * the one array, so calls whose kernels overlap on the GPU (different streams, or several
 * threads) race and must be serialised by the caller.  Errors: as mgx_compute, plus
 * WORKSPACE_TOO_SMALL when one 128-thread block's workspace (128 x the process's per-event
 * workspace) exceeds the array. */
size_t mgx_noalloc_scratch_bytes(void);
int mgx_compute_noalloc(mgx_process* proc, int64_t nevt, const double* momenta, const double* alpha_s,
                        const double* rnd_hel, const double* rnd_col, double* me, int32_t* selhel,
                        int32_t* selcol, int mode, void* stream);

/* ---- device-side event generation (random numbers -> momenta, Sec. 2) ----
 * Philox-4x32-10 words for event e come from counter (e mod 2^32, block, stream, e >> 32)
 * and key = seed, so results depend only on (seed, stream, event index) and equal the host
 * generator bit for bit (the Python package `phasespace`). */

/* out[i] = uniform in [0,1) with 53 bits from block 0 of event first+i (DEVICE array). */
int mgx_uniforms(int64_t n, int64_t first, uint64_t seed, uint32_t stream_id, double* out, void* stream);

/* Flat phase space by RAMBO for events first .. first+n-1: momenta [n][nfinal+2][4] (DEVICE):
 * two beams along +-z with E = sqrts/2, then nfinal particles of masses masses_dev[nfinal]
 * (DEVICE array); weight [n] (DEVICE, may be NULL) = phase-space weight.  nfinal <= 8. */
int mgx_rambo(int64_t n, int64_t first, double sqrts, int nfinal, const double* masses_dev, uint64_t seed,
              double* momenta, double* weight, void* stream);

/* The same events first + index[r], r < m (index: DEVICE int32 [m]): momenta [m][nfinal+2][4], weight [m],
 * bit-identical to the corresponding rows of mgx_rambo (regenerating selected events in float64). */
int mgx_rambo_indexed(int64_t m, const int32_t* index, int64_t first, double sqrts, int nfinal,
                      const double* masses_dev, uint64_t seed, double* momenta, double* weight, void* stream);
/* RAMBO in float32 (the same random numbers; momenta and weight to float32 accuracy): cheap proposals
 * for the first stage of the two-stage unweighting, whose survivors are regenerated in float64. */
int mgx_rambo_f32(int64_t n, int64_t first, double sqrts, int nfinal, const double* masses_dev, uint64_t seed,
                  float* momenta, float* weight, void* stream);

/* Generator-level cuts: pass[i] = 1 when every particle listed in list_dev[nlist] (indices into
 * npar) has pT > ptmin and |eta| < etamax and every listed pair has dR > drmin, else 0. */
int mgx_cuts(int64_t n, int npar, const double* momenta, int nlist, const int* list_dev, double ptmin,
             double etamax, double drmin, uint8_t* pass, void* stream);
/* The cuts on float32 momenta with thresholds widened by a relative margin (0 <= margin < 0.5):
 * pT > ptmin (1 - margin), |eta| < etamax (1 + margin), dR > drmin (1 - margin), so that the region
 * they accept contains the one the float64 cuts accept (for margins well above float32 rounding). */
int mgx_cuts_f32(int64_t n, int npar, const float* momenta, int nlist, const int* list_dev, double ptmin,
                 double etamax, double drmin, double margin, uint8_t* pass, void* stream);

/* ---- learned surrogate of log|M|^2 (two-stage unweighting) ----
 * MLP x[24] -> 4 x 256 SiLU -> scalar; float32 master weights, bfloat16 tensor-core products
 * with float32 accumulation.  Parameters are one flat float32 vector of mgx_mlp_num_params()
 * entries: per hidden layer l, W_l [256][kin_l] row-major (kin_0 = 32: the 24 inputs zero-padded,
 * padded columns zero) then b_l [256]; then w_out [256] and b_out.  Inputs are float32 [n][24]. */
typedef struct mgx_mlp mgx_mlp;
int mgx_mlp_num_params(void);
/* Create a network on `device` with He-uniform weights from a seeded generator.  Synchronous. */
int mgx_mlp_create(int device, uint64_t seed, mgx_mlp** out);
void mgx_mlp_destroy(mgx_mlp* net);
/* DEVICE workspace bytes for a training batch of n rows (training != 0, n <= 2^24) or for
 * inference over any n (processed in passes of at most 2^22 rows, about 1.1 KB per row). */
int mgx_mlp_workspace_bytes(int64_t n, int training, size_t* bytes);
/* Host copies of the flat float32 parameter vector (set also refreshes the bfloat16 copies). */
int mgx_mlp_get_params(const mgx_mlp* net, float* host);
int mgx_mlp_set_params(mgx_mlp* net, const float* host);
/* y[n] = network(x[n][24]); DEVICE arrays; asynchronous on stream.  Inference runs one persistent
 * tcgen05 kernel per layer: the layer's bf16 weights stay in shared memory, 128-row activation
 * tiles stream through it by bulk copies, accumulate in tensor memory, and bias + SiLU (and, in the
 * last layer, the 256 -> 1 output) are applied in the epilogue. */
int mgx_mlp_forward(mgx_mlp* net, int64_t n, const float* x, float* y, void* ws, size_t wsb, void* stream);
/* The same from float64 momenta [n][24] (an event's four-momenta in order), the network's inputs
 * being float32(momenta / scale) (scale: sqrt(s)/2 for the surrogate), without a separate
 * feature array. */
int mgx_mlp_forward_momenta(mgx_mlp* net, int64_t n, const double* momenta, double scale, float* y, void* ws,
                            size_t wsb, void* stream);
/* The same from float32 momenta (inputs float32(momenta x (1/scale))). */
int mgx_mlp_forward_momenta_f32(mgx_mlp* net, int64_t n, const float* momenta, double scale, float* y, void* ws,
                                size_t wsb, void* stream);
/* Gradient of the mean squared error over one batch of n rows (targets t[n]) into grad
 * (DEVICE, num_params floats, may be NULL) and the loss into loss (DEVICE float, may be NULL). */
int mgx_mlp_gradients(mgx_mlp* net, int n, const float* x, const float* t, float* grad, float* loss, void* ws,
                      size_t wsb, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at learning rate lr on one batch. */
int mgx_mlp_train_step(mgx_mlp* net, int n, const float* x, const float* t, float lr, float* loss, void* ws,
                       size_t wsb, void* stream);
/* The same two calls on a batch the library draws from a training set of ntotal examples (x
 * [ntotal][24], t [ntotal], DEVICE): batch row r (0 <= r < batch) takes example
 * j = floor(u ntotal), where u is the first 32-bit word of the Philox-4x32-10 block with counter
 * (r, step mod 2^32, 0x4D4C5053, 0) under the 64-bit key seed, divided by 2^32 (sampling with
 * replacement; a replica uses its own seed).  The batch rows are gathered into the workspace
 * (workspace bytes as for a training batch of `batch` rows). */
int mgx_mlp_gradients_sampled(mgx_mlp* net, int ntotal, const float* x, const float* t, int batch, uint64_t seed,
                              uint64_t step, float* grad, float* loss, void* ws, size_t wsb, void* stream);
int mgx_mlp_train_step_sampled(mgx_mlp* net, int ntotal, const float* x, const float* t, int batch, uint64_t seed,
                               uint64_t step, float lr, float* loss, void* ws, size_t wsb, void* stream);
/* One Adam step on a gradient the caller supplies (DEVICE, num_params floats): the update half of a
 * data-parallel training step, after the per-replica gradients of mgx_mlp_gradients have been
 * averaged across replicas (weighted by their batch sizes).  Replicas that start from the same
 * parameters and apply the same averaged gradient stay identical.  Asynchronous on stream. */
int mgx_mlp_adam_step(mgx_mlp* net, const float* grad, float lr, void* stream);
/* Failure detection of the network's tensor-core GEMMs: every wait for the tile's MMAs has a time
 * limit; a tile whose wait runs out writes NaN to its outputs and adds 1 to the network's device
 * error counter.  mgx_mlp_device_errors copies the counter to *count (synchronous; call it after
 * the work it covers has completed) and zeroes it when reset != 0.  mgx_mlp_set_wait_test is the
 * test hook: with skip_mma != 0 no MMA is issued and each wait runs out after wait_ms
 * (0 < wait_ms <= 10000, default limit 1000 ms). */
int mgx_mlp_device_errors(mgx_mlp* net, int* count, int reset);
int mgx_mlp_set_wait_test(mgx_mlp* net, int skip_mma, double wait_ms);

/* ---- unweighting (plain hit-or-miss and two-stage with the surrogate) ----
 * Plain: keep with probability min(1, w/w_max), weight max(1, w/w_max).  Two-stage
 * (Danziger, Janssen, Schumann, Siegert, arXiv:2109.11964): stage 1 keeps with probability
 * min(1, s/s_max) on the surrogate weight s, stage 2 evaluates the exact weight w of the
 * survivors and keeps them with probability min(1, (w/s)/r_max); the kept event carries
 * max(1, s/s_max) max(1, (w/s)/r_max), so the unweighted sample is unbiased.  All arrays DEVICE. */
/* x[i][j] = float(momenta[i][j] / scale), j < ncomp (the flattened momenta of one event). */
int mgx_features(int64_t n, int ncomp, const double* momenta, double scale, float* x, void* stream);
/* s = exp(mean + sd y) * wps * pass (wps, pass may be NULL). */
int mgx_surrogate_weight(int64_t n, const float* y, double mean, double sd, const double* wps,
                         const uint8_t* pass, double* s, void* stream);
/* The same with a float32 phase-space weight wps (from mgx_rambo_f32), computed in float32
 * (fast-math exponential, a few ulp; s = float(exp(float(mean) + float(sd) y) wps)) when the
 * exponent's magnitude is below 80 and in float64 otherwise: a proposal weight only has to be
 * positive wherever the exact weight is. */
int mgx_surrogate_weight_f32(int64_t n, const float* y, double mean, double sd, const float* wps,
                             const uint8_t* pass, double* s, void* stream);
/* w = me * wps * pass (wps, pass may be NULL). */
int mgx_exact_weight(int64_t n, const double* me, const double* wps, const uint8_t* pass, double* w,
                     void* stream);
/* ratio = w/wref (wref NULL: w); keep = r * wmax < ratio; overweight = max(1, ratio/wmax) (may be NULL). */
int mgx_accept(int64_t n, const double* w, const double* wref, double wmax, const double* r, uint8_t* keep,
               double* overweight, void* stream);
/* Deterministic stream compaction: index[0..count) = ascending i with keep[i] != 0; count to count_dev. */
int mgx_compact_workspace_bytes(int64_t n, size_t* bytes);
int mgx_compact(int64_t n, const uint8_t* keep, int32_t* index, int32_t* count_dev, void* ws, size_t wsb,
                void* stream);
/* dst[r][0..row) = src[index[r]][0..row) for r < m (float64 rows). */
int mgx_gather(int64_t m, const int32_t* index, int row, const double* src, double* dst, void* stream);
/* Training targets of the surrogate from exact matrix elements me[n] and the cut flags pass[n]
 * (may be NULL: all pass): keep[i] = pass[i] && 0 < me[i] < inf, logme[i] = log(me[i]) where kept,
 * 0 elsewhere.  DEVICE arrays; asynchronous. */
int mgx_log_targets(int64_t n, const double* me, const uint8_t* pass, double* logme, uint8_t* keep, void* stream);
/* sums[0] = sum y[i], sums[1] = sum y[i]^2, sums[2] = max y[i] (-inf when n = 0) over n float64
 * values (DEVICE), in a fixed order (the same bits on every call): MGX_MOMENTS_BLOCKS blocks reduce
 * contiguous ranges, then one block combines their partials.  sums is a DEVICE array of
 * MGX_MOMENTS_LEN doubles; entries 3 .. MGX_MOMENTS_LEN - 1 are the partials (scratch).
 * Asynchronous. */
#define MGX_MOMENTS_BLOCKS 256
#define MGX_MOMENTS_LEN (3 * (1 + MGX_MOMENTS_BLOCKS))
int mgx_moments(int64_t n, const double* y, double* sums, void* stream);
/* t[i] = float32((y[i] - mean) / sd), sd > 0 (the network's standardised targets).  DEVICE. */
int mgx_standardize_f32(int64_t n, const double* y, double mean, double sd, float* t, void* stream);
/* The unweighted events of one batch from the compacted survivors: event j of the output is
 * idx2[j] of the last stage, or idx1[idx2[j]] with a first stage (idx1 may be NULL); weight[j] =
 * over1[event] x over2[idx2[j]] (over2 may be NULL: a single stage), index[j] = first + event.
 * DEVICE arrays (index int64); asynchronous. */
int mgx_unweighted_out(int64_t m, const int32_t* idx2, const int32_t* idx1, const double* over1, const double* over2,
                       int64_t first, double* weight, int64_t* index, void* stream);
/* Reference maxima of the unweighting from n calibration events (exact weights w, surrogate weights
 * s; DEVICE): maxima[0..2] (HOST) = the q-quantiles (0 < q <= 1; linear interpolation between
 * order statistics at position q (m - 1); q = 1: the maxima) of w, s and w/s over the m events with
 * w > 0 and s > 0, computed on the host after copying w and s back (synchronous on stream). */
int mgx_unweighting_maxima(int64_t n, const double* w, const double* s, double q, double* maxima, void* stream);

/* Measured fused-multiply-add throughput (TFLOP/s, fma = 2 flops) of the float64
 * (precision 64) or float32 (precision 32) pipe of `device`: independent FMA chains, no memory
 * traffic.  Source of the float64 roofline peak (2 DFMA/clk/SM on GB300).  Synchronous;
 * allocates a small buffer. */
int mgx_measure_fma_tflops(int device, int precision, double* tflops);

void mgx_process_destroy(mgx_process* proc);
const char* mgx_status_string(int status);
int mgx_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MGX_H */
