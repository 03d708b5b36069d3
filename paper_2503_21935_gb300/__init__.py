"""mgx: GB300-native batched tree-level |M|^2 (arXiv:2503.21935 hot path).

Thin Python binding over the C ABI in include/mgx.h (libmgx.so, built in-tree by
paper_2503_21935_gb300.build).  Only argument marshalling happens here; every
step of the matrix-element computation runs in the library's CUDA kernels.
PyTorch provides device memory and streams.  There is no CPU fallback: importing
the package without a built library, or calling it without a GPU, raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmgx.so")

MGX_OK = 0
MGX_FP64 = 0
MGX_MIXED_FP32 = 1
MGX_MIXED_TF32 = 2
MGX_MIXED_BF16X3 = 3
MGX_FLOAT = 4
MODES = {"fp64": MGX_FP64, "mixed_fp32": MGX_MIXED_FP32, "mixed_tf32": MGX_MIXED_TF32,
         "mixed_bf16x3": MGX_MIXED_BF16X3, "float": MGX_FLOAT}
MGX_KERNEL_AUTO, MGX_KERNEL_THREAD, MGX_KERNEL_CTA, MGX_KERNEL_THREAD_SMEM = 0, 1, 2, 3
MGX_MOMENTS_BLOCKS = 256
MGX_MOMENTS_LEN = 3 * (1 + MGX_MOMENTS_BLOCKS)   # doubles of mgx_moments' output (3 results + partials)


class MgxError(RuntimeError):
    pass


class mgx_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("mt", "wt", "mz", "wz", "mta", "alpha_em", "gf", "filter_sqrt_s")]


_lib = None


def lib():
    """The loaded libmgx.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise MgxError(f"libmgx.so is not built ({LIB_PATH}); run paper_2503_21935_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I64, SZ, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t, ctypes.c_double
        I, U64 = ctypes.c_int, ctypes.c_uint64
        sig = {
            "mgx_params_default": (None, [ctypes.POINTER(mgx_params)]),
            "mgx_num_processes": (I, []),
            "mgx_process_name": (ctypes.c_char_p, [I]),
            "mgx_process_create": (I, [ctypes.c_char_p, ctypes.POINTER(mgx_params), I, U64, ctypes.POINTER(P)]),
            "mgx_process_info": (I, [P] + [ctypes.POINTER(I)] * 6),
            "mgx_good_helicities": (I, [P, P]),
            "mgx_colour_matrix": (I, [P, P]),
            "mgx_workspace_bytes": (I, [P, I64, I, ctypes.POINTER(SZ)]),
            "mgx_compute": (I, [P, I64, P, P, P, P, P, P, P, I, P, SZ, P]),
            "mgx_compute_ex": (I, [P, I64, P, P, P, P, P, P, P, P, P, I, P, SZ, P]),
            "mgx_host_workspace_bytes": (I, [P, I64, I, ctypes.POINTER(SZ)]),
            "mgx_compute_host": (I, [P, I64, P, P, P, P, P, P, P, I, P, SZ, P]),
            "mgx_fp64_ops_per_event": (D, [P, I]),
            "mgx_fp64_flops_per_event": (D, [P, I]),
            "mgx_kernel_launches": (I, [P, I64, I]),
            "mgx_process_set_kernel": (I, [P, I]),
            "mgx_process_get_kernel": (I, [P]),
            "mgx_process_plan": (I, [P, I64, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
            "mgx_process_set_blocks_per_sm": (I, [P, I]),
            "mgx_process_device_errors": (I, [P, ctypes.POINTER(I), I]),
            "mgx_process_set_tc_wait_test": (I, [P, I, D]),
            "mgx_process_destroy": (None, [P]),
            "mgx_measure_fma_tflops": (I, [I, I, ctypes.POINTER(D)]),
            "mgx_uniforms": (I, [I64, I64, U64, ctypes.c_uint32, P, P]),
            "mgx_rambo": (I, [I64, I64, D, I, P, U64, P, P, P]),
            "mgx_cuts": (I, [I64, I, P, I, P, D, D, D, P, P]),
            "mgx_cuts_f32": (I, [I64, I, P, I, P, D, D, D, D, P, P]),
            "mgx_rambo_indexed": (I, [I64, P, I64, D, I, P, U64, P, P, P]),
            "mgx_rambo_f32": (I, [I64, I64, D, I, P, U64, P, P, P]),
            "mgx_surrogate_weight_f32": (I, [I64, P, D, D, P, P, P, P]),
            "mgx_mlp_forward_momenta_f32": (I, [P, I64, P, D, P, P, SZ, P]),
            "mgx_features": (I, [I64, I, P, D, P, P]),
            "mgx_surrogate_weight": (I, [I64, P, D, D, P, P, P, P]),
            "mgx_exact_weight": (I, [I64, P, P, P, P, P]),
            "mgx_accept": (I, [I64, P, P, D, P, P, P, P]),
            "mgx_compact_workspace_bytes": (I, [I64, ctypes.POINTER(SZ)]),
            "mgx_compact": (I, [I64, P, P, P, P, SZ, P]),
            "mgx_gather": (I, [I64, P, I, P, P, P]),
            "mgx_log_targets": (I, [I64, P, P, P, P, P]),
            "mgx_moments": (I, [I64, P, P, P]),
            "mgx_standardize_f32": (I, [I64, P, D, D, P, P]),
            "mgx_unweighted_out": (I, [I64, P, P, P, P, I64, P, P, P]),
            "mgx_unweighting_maxima": (I, [I64, P, P, D, P, P]),
            "mgx_batch_create": (I, [P, I, ctypes.POINTER(P)]),
            "mgx_batch_destroy": (None, [P]),
            "mgx_batch_workspace_bytes": (I, [P, ctypes.POINTER(SZ)]),
            "mgx_batch_compute": (I, [P, P, I, P, SZ, P]),
            "mgx_batch_capture": (I, [P, P, I, P, SZ, P]),
            "mgx_batch_replay": (I, [P, P]),
            "mgx_batch_autotune": (I, [P, P, I, P, SZ, P, ctypes.POINTER(I), ctypes.POINTER(I)]),
            "mgx_process_autotune": (I, [P, I64, P, P, I, P, SZ, P, ctypes.POINTER(I), ctypes.POINTER(I), P]),
            "mgx_mlp_num_params": (I, []),
            "mgx_mlp_create": (I, [I, U64, ctypes.POINTER(P)]),
            "mgx_mlp_destroy": (None, [P]),
            "mgx_mlp_workspace_bytes": (I, [I64, I, ctypes.POINTER(SZ)]),
            "mgx_mlp_get_params": (I, [P, P]),
            "mgx_mlp_set_params": (I, [P, P]),
            "mgx_mlp_forward": (I, [P, I64, P, P, P, SZ, P]),
            "mgx_mlp_forward_momenta": (I, [P, I64, P, D, P, P, SZ, P]),
            "mgx_mlp_gradients": (I, [P, I, P, P, P, P, P, SZ, P]),
            "mgx_mlp_train_step": (I, [P, I, P, P, ctypes.c_float, P, P, SZ, P]),
            "mgx_mlp_adam_step": (I, [P, P, ctypes.c_float, P]),
            "mgx_mlp_gradients_sampled": (I, [P, I, P, P, I, U64, U64, P, P, P, SZ, P]),
            "mgx_mlp_train_step_sampled": (I, [P, I, P, P, I, U64, U64, ctypes.c_float, P, P, SZ, P]),
            "mgx_mlp_device_errors": (I, [P, ctypes.POINTER(I), I]),
            "mgx_mlp_set_wait_test": (I, [P, I, D]),
            "mgx_noalloc_scratch_bytes": (SZ, []),
            "mgx_compute_noalloc": (I, [P, I64, P, P, P, P, P, P, P, I, P]),
            "mgx_status_string": (ctypes.c_char_p, [I]),
            "mgx_version": (I, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_string(rc):
    """The library's message for a status code."""
    return lib().mgx_status_string(rc).decode()


def _check(rc, what):
    if rc != MGX_OK:
        raise MgxError(f"{what}: {status_string(rc)} ({rc})")


def default_params():
    p = mgx_params()
    lib().mgx_params_default(ctypes.byref(p))
    return p


def measure_fma_tflops(device=0, precision=64):
    """Measured FMA throughput of the float64 (64) or float32 (32) pipe in TFLOP/s."""
    v = ctypes.c_double()
    _check(lib().mgx_measure_fma_tflops(device, precision, ctypes.byref(v)), "mgx_measure_fma_tflops")
    return v.value


def _stream(device=None):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def uniforms(n, seed, stream_id, first=0, device=0):
    """Device tensor of n uniforms in [0,1) (Philox, identical to phasespace.uniform01)."""
    import torch
    out = torch.empty(n, dtype=torch.float64, device=f"cuda:{device}")
    _check(lib().mgx_uniforms(n, first, seed, stream_id, _ptr(out), _stream(out.device)), "mgx_uniforms")
    return out


def rambo(n, sqrts, masses, seed, first=0, device=0):
    """Device RAMBO: (momenta [n, len(masses)+2, 4], weight [n]), identical events to phasespace.rambo."""
    import torch
    dev = torch.device(f"cuda:{device}")
    m = torch.tensor(list(masses), dtype=torch.float64, device=dev)
    mom = torch.empty((n, len(masses) + 2, 4), dtype=torch.float64, device=dev)
    wt = torch.empty(n, dtype=torch.float64, device=dev)
    _check(lib().mgx_rambo(n, first, float(sqrts), len(masses), _ptr(m), seed, _ptr(mom), _ptr(wt), _stream(dev)),
           "mgx_rambo")
    return mom, wt


def rambo_indexed(index, first, sqrts, masses, seed, device=0):
    """Device float64 RAMBO for events first + index[r] (int32 device tensor): (momenta, weight)."""
    import torch
    dev = torch.device(f"cuda:{device}")
    m = torch.tensor(list(masses), dtype=torch.float64, device=dev)
    n = index.shape[0]
    mom = torch.empty((n, len(masses) + 2, 4), dtype=torch.float64, device=dev)
    wt = torch.empty(n, dtype=torch.float64, device=dev)
    _check(lib().mgx_rambo_indexed(n, _ptr(index), first, float(sqrts), len(masses), _ptr(m), seed, _ptr(mom),
                                   _ptr(wt), _stream(dev)), "mgx_rambo_indexed")
    return mom, wt


def rambo_f32(n, sqrts, masses, seed, first=0, device=0):
    """Device float32 RAMBO (the same events as rambo, to float32 accuracy): (momenta, weight)."""
    import torch
    dev = torch.device(f"cuda:{device}")
    m = torch.tensor(list(masses), dtype=torch.float64, device=dev)
    mom = torch.empty((n, len(masses) + 2, 4), dtype=torch.float32, device=dev)
    wt = torch.empty(n, dtype=torch.float32, device=dev)
    _check(lib().mgx_rambo_f32(n, first, float(sqrts), len(masses), _ptr(m), seed, _ptr(mom), _ptr(wt), _stream(dev)),
           "mgx_rambo_f32")
    return mom, wt


def cuts_f32(momenta, particles, ptmin, etamax, drmin, margin):
    """Device uint8 mask of the cuts on float32 momenta with thresholds widened by `margin`."""
    import torch
    dev = momenta.device
    lst = torch.tensor(list(particles), dtype=torch.int32, device=dev)
    out = torch.empty(momenta.shape[0], dtype=torch.uint8, device=dev)
    _check(lib().mgx_cuts_f32(momenta.shape[0], momenta.shape[1], _ptr(momenta), len(particles), _ptr(lst),
                              float(ptmin), float(etamax), float(drmin), float(margin), _ptr(out), _stream(dev)),
           "mgx_cuts_f32")
    return out


def cuts(momenta, particles, ptmin, etamax, drmin):
    """Device uint8 mask of events passing pT / |eta| / pairwise dR cuts on the listed particles."""
    import torch
    dev = momenta.device
    lst = torch.tensor(list(particles), dtype=torch.int32, device=dev)
    out = torch.empty(momenta.shape[0], dtype=torch.uint8, device=dev)
    _check(lib().mgx_cuts(momenta.shape[0], momenta.shape[1], _ptr(momenta), len(particles), _ptr(lst),
                          float(ptmin), float(etamax), float(drmin), _ptr(out), _stream(dev)), "mgx_cuts")
    return out


class mgx_batch_io(ctypes.Structure):
    _fields_ = [("nevt", ctypes.c_int64)] + [(n, ctypes.c_void_p) for n in
                                             ("momenta", "alpha_s", "rnd_hel", "rnd_col", "me", "selhel", "selcol")]


class Batch:
    """Several processes in one persistent launch (mgx_batch_*), optionally captured in a CUDA graph."""

    def __init__(self, processes):
        import torch
        self.procs = list(processes)
        arr = (ctypes.c_void_p * len(self.procs))(*[p._h.value for p in self.procs])
        h = ctypes.c_void_p()
        _check(lib().mgx_batch_create(arr, len(self.procs), ctypes.byref(h)), "mgx_batch_create")
        self._h = h
        b = ctypes.c_size_t()
        _check(lib().mgx_batch_workspace_bytes(h, ctypes.byref(b)), "mgx_batch_workspace_bytes")
        self.ws = torch.empty(b.value, dtype=torch.uint8, device=f"cuda:{self.procs[0].device}")
        self._io = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.mgx_batch_destroy(h)
            self._h = None

    def _make_io(self, inputs, outputs):
        io = (mgx_batch_io * len(self.procs))()
        for k, (inp, out) in enumerate(zip(inputs, outputs)):
            mom, a = inp[0], inp[1]
            rh = inp[2] if len(inp) > 2 else None
            rc = inp[3] if len(inp) > 3 else None
            io[k].nevt = mom.shape[0]
            io[k].momenta, io[k].alpha_s = mom.data_ptr(), a.data_ptr()
            io[k].rnd_hel = rh.data_ptr() if rh is not None else None
            io[k].rnd_col = rc.data_ptr() if rc is not None else None
            io[k].me = out["me"].data_ptr()
            io[k].selhel = out["selhel"].data_ptr() if out.get("selhel") is not None else None
            io[k].selcol = out["selcol"].data_ptr() if out.get("selcol") is not None else None
        self._io = io
        return io

    def compute(self, inputs, outputs, mode=MGX_FP64, stream=None):
        """inputs: per process (momenta, alpha_s[, rnd_hel, rnd_col]); outputs: per process dict(me, selhel, selcol)."""
        io = self._make_io(inputs, outputs)
        st = stream or _stream(self.ws.device)
        _check(lib().mgx_batch_compute(self._h, io, mode, _ptr(self.ws), self.ws.numel(),
                                       ctypes.c_void_p(st.cuda_stream) if hasattr(st, "cuda_stream") else st),
               "mgx_batch_compute")

    def capture(self, inputs, outputs, stream, mode=MGX_FP64):
        io = self._make_io(inputs, outputs)
        _check(lib().mgx_batch_capture(self._h, io, mode, _ptr(self.ws), self.ws.numel(),
                                       ctypes.c_void_p(stream.cuda_stream)), "mgx_batch_capture")

    def replay(self, stream):
        _check(lib().mgx_batch_replay(self._h, ctypes.c_void_p(stream.cuda_stream)), "mgx_batch_replay")

    def autotune(self, inputs, outputs, mode=MGX_FP64):
        """Returns (blocks per SM, [events per work item of each process])."""
        io = self._make_io(inputs, outputs)
        b = ctypes.c_int()
        e = (ctypes.c_int * len(self.procs))()
        _check(lib().mgx_batch_autotune(self._h, io, mode, _ptr(self.ws), self.ws.numel(), _stream(self.ws.device),
                                        ctypes.byref(b), e), "mgx_batch_autotune")
        return b.value, list(e)


class Mlp:
    """The MLP surrogate (mgx_mlp_*): forward, gradients and Adam steps in the library's kernels."""

    def __init__(self, seed=0, device=0):
        import torch
        if not torch.cuda.is_available():
            raise MgxError("no CUDA device: the mgx library has no CPU path")
        self.device = device
        h = ctypes.c_void_p()
        _check(lib().mgx_mlp_create(device, seed, ctypes.byref(h)), "mgx_mlp_create")
        self._h = h
        self.nparams = lib().mgx_mlp_num_params()
        self._ws = {}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.mgx_mlp_destroy(h)
            self._h = None

    def _dev(self, x, dtype=None):
        import torch
        if isinstance(x, np.ndarray):
            x = torch.from_numpy(np.ascontiguousarray(x))
        return x.to(device=f"cuda:{self.device}", dtype=dtype or x.dtype).contiguous()

    def _workspace(self, n, training):
        import torch
        b = ctypes.c_size_t()
        _check(lib().mgx_mlp_workspace_bytes(n, int(training), ctypes.byref(b)), "mgx_mlp_workspace_bytes")
        key = bool(training)
        ws = self._ws.get(key)
        if ws is None or ws.numel() < b.value:
            ws = torch.empty(b.value, dtype=torch.uint8, device=f"cuda:{self.device}")
            self._ws[key] = ws
        return ws

    def get_params(self):
        p = np.zeros(self.nparams, dtype=np.float32)
        _check(lib().mgx_mlp_get_params(self._h, p.ctypes.data_as(ctypes.c_void_p)), "mgx_mlp_get_params")
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().mgx_mlp_set_params(self._h, p.ctypes.data_as(ctypes.c_void_p)), "mgx_mlp_set_params")

    def forward(self, x, out=None):
        """x [n, 24] float32 (host or device) -> y [n] (numpy if x was numpy)."""
        import torch
        host = isinstance(x, np.ndarray)
        xd = self._dev(x, torch.float32)
        n = xd.shape[0]
        y = out if out is not None else torch.empty(n, dtype=torch.float32, device=xd.device)
        ws = self._workspace(n, False)
        _check(lib().mgx_mlp_forward(self._h, n, _ptr(xd), _ptr(y), _ptr(ws), ws.numel(), _stream(xd.device)),
               "mgx_mlp_forward")
        return y.cpu().numpy() if host else y

    def forward_momenta(self, momenta, scale, out=None):
        """y[n] = network(float32(momenta / scale)) for device momenta [n, 6, 4] (float64 or float32)."""
        import torch
        n = momenta.shape[0]
        y = out if out is not None else torch.empty(n, dtype=torch.float32, device=momenta.device)
        ws = self._workspace(n, False)
        f = lib().mgx_mlp_forward_momenta_f32 if momenta.dtype == torch.float32 else lib().mgx_mlp_forward_momenta
        _check(f(self._h, n, _ptr(momenta), float(scale), _ptr(y), _ptr(ws), ws.numel(), _stream(momenta.device)),
               "mgx_mlp_forward_momenta")
        return y

    def gradients(self, x, t):
        import torch
        xd, td = self._dev(x, torch.float32), self._dev(t, torch.float32)
        n = xd.shape[0]
        g = torch.empty(self.nparams, dtype=torch.float32, device=xd.device)
        loss = torch.empty(1, dtype=torch.float32, device=xd.device)
        ws = self._workspace(n, True)
        _check(lib().mgx_mlp_gradients(self._h, n, _ptr(xd), _ptr(td), _ptr(g), _ptr(loss), _ptr(ws), ws.numel(),
                                       _stream(xd.device)), "mgx_mlp_gradients")
        return float(loss.item()), g.cpu().numpy()

    def device_gradients(self, x, t, loss_out=None):
        """Gradient of the mean squared error on one batch as a device float32 tensor (no host copy)."""
        import torch
        xd, td = self._dev(x, torch.float32), self._dev(t, torch.float32)
        n = xd.shape[0]
        g = torch.empty(self.nparams, dtype=torch.float32, device=xd.device)
        ws = self._workspace(n, True)
        _check(lib().mgx_mlp_gradients(self._h, n, _ptr(xd), _ptr(td), _ptr(g), _ptr(loss_out), _ptr(ws), ws.numel(),
                                       _stream(xd.device)), "mgx_mlp_gradients")
        return g

    def device_errors(self, reset=True):
        """Tensor-core waits of the GEMMs that ran out since the last reset (synchronise first)."""
        c = ctypes.c_int()
        _check(lib().mgx_mlp_device_errors(self._h, ctypes.byref(c), int(reset)), "mgx_mlp_device_errors")
        return c.value

    def set_wait_test(self, skip_mma, wait_ms=1000.0):
        """Test hook: with skip_mma the GEMMs issue no MMA and their waits run out."""
        _check(lib().mgx_mlp_set_wait_test(self._h, int(skip_mma), float(wait_ms)), "mgx_mlp_set_wait_test")

    def adam_step(self, grad, lr=1e-3):
        """One Adam step on a device gradient (e.g. the replicas' average in data-parallel training)."""
        _check(lib().mgx_mlp_adam_step(self._h, _ptr(grad), ctypes.c_float(lr), _stream(grad.device)),
               "mgx_mlp_adam_step")

    def train_step(self, x, t, lr=1e-3, loss_out=None):
        import torch
        xd, td = self._dev(x, torch.float32), self._dev(t, torch.float32)
        n = xd.shape[0]
        ws = self._workspace(n, True)
        _check(lib().mgx_mlp_train_step(self._h, n, _ptr(xd), _ptr(td), ctypes.c_float(lr), _ptr(loss_out),
                                        _ptr(ws), ws.numel(), _stream(xd.device)), "mgx_mlp_train_step")

    def train_step_sampled(self, x, t, batch, seed, step, lr=1e-3, loss_out=None):
        """One Adam step on a batch the library draws (Philox, with replacement) from the device
        training set x [ntotal][24], t [ntotal] (float32): mgx_mlp_train_step_sampled."""
        import torch
        x, t = self._dev(x, torch.float32), self._dev(t, torch.float32)
        ws = self._workspace(batch, True)
        _check(lib().mgx_mlp_train_step_sampled(self._h, x.shape[0], _ptr(x), _ptr(t), int(batch), int(seed), int(step),
                                                ctypes.c_float(lr), _ptr(loss_out), _ptr(ws), ws.numel(),
                                                _stream(x.device)), "mgx_mlp_train_step_sampled")

    def device_gradients_sampled(self, x, t, batch, seed, step, loss_out=None):
        """Gradient (device float32) on a batch drawn as by train_step_sampled."""
        import torch
        x, t = self._dev(x, torch.float32), self._dev(t, torch.float32)
        g = torch.empty(self.nparams, dtype=torch.float32, device=x.device)
        ws = self._workspace(batch, True)
        _check(lib().mgx_mlp_gradients_sampled(self._h, x.shape[0], _ptr(x), _ptr(t), int(batch), int(seed), int(step),
                                               _ptr(g), _ptr(loss_out), _ptr(ws), ws.numel(), _stream(x.device)),
               "mgx_mlp_gradients_sampled")
        return g


def builtin_processes():
    return [lib().mgx_process_name(i).decode() for i in range(lib().mgx_num_processes())]


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Process:
    """A process on one CUDA device: mgx_process_create / mgx_compute / mgx_process_destroy."""

    def __init__(self, process, params=None, device=0, filter_seed=0):
        import torch
        if not torch.cuda.is_available():
            raise MgxError("no CUDA device: the mgx library has no CPU path")
        torch.cuda.init()
        self.device = device
        prm = default_params()
        for k, v in (params or {}).items():
            setattr(prm, k, float(v))
        h = ctypes.c_void_p()
        with torch.cuda.device(device):
            _check(lib().mgx_process_create(process.encode(), ctypes.byref(prm), device, filter_seed,
                                            ctypes.byref(h)), "mgx_process_create")
        self._h = h
        vals = [ctypes.c_int() for _ in range(6)]
        _check(lib().mgx_process_info(h, *[ctypes.byref(v) for v in vals]), "mgx_process_info")
        self.npar, self.nhel, self.ngood, self.ndiagrams, self.nterms, self.ncol = (v.value for v in vals)
        g = np.zeros(self.ngood, dtype=np.int32)
        _check(lib().mgx_good_helicities(h, g.ctypes.data_as(ctypes.c_void_p)), "mgx_good_helicities")
        self.good_helicities = g.tolist()
        self.process = process
        self._ws = {}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.mgx_process_destroy(h)
            self._h = None

    def colour_matrix(self):
        C = np.zeros((self.ncol, self.ncol))
        _check(lib().mgx_colour_matrix(self._h, C.ctypes.data_as(ctypes.c_void_p)), "mgx_colour_matrix")
        return C

    def workspace_bytes(self, nevt, mode=MGX_FP64, host=False):
        b = ctypes.c_size_t()
        f = lib().mgx_host_workspace_bytes if host else lib().mgx_workspace_bytes
        _check(f(self._h, nevt, mode, ctypes.byref(b)), "workspace_bytes")
        return b.value

    def workspace(self, nevt, mode=MGX_FP64, host=False):
        import torch
        need = self.workspace_bytes(nevt, mode, host)
        key = (host, mode in (MGX_MIXED_TF32, MGX_MIXED_BF16X3))
        ws = self._ws.get(key)
        if ws is None or ws.numel() < need:
            ws = torch.empty(max(need, 256), dtype=torch.uint8, device=f"cuda:{self.device}")
            self._ws[key] = ws
        return ws

    def set_kernel(self, kernel):
        """MGX_KERNEL_AUTO / MGX_KERNEL_THREAD / MGX_KERNEL_CTA / MGX_KERNEL_THREAD_SMEM.  AUTO picks per
        call by batch size: one block per event (CTA) or the shared-memory thread kernel for small
        batches, the thread kernel otherwise."""
        _check(lib().mgx_process_set_kernel(self._h, kernel), "mgx_process_set_kernel")

    @property
    def kernel(self):
        return lib().mgx_process_get_kernel(self._h)

    def plan(self, nevt, mode=MGX_FP64):
        """(kernel, helicity groups, diagram parts) a compute of nevt events would run."""
        k, g, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().mgx_process_plan(self._h, nevt, mode, ctypes.byref(k), ctypes.byref(g), ctypes.byref(d)),
               "mgx_process_plan")
        return k.value, g.value, d.value

    def set_blocks_per_sm(self, n):
        _check(lib().mgx_process_set_blocks_per_sm(self._h, n), "mgx_process_set_blocks_per_sm")
        self._ws = {}

    def autotune(self, momenta, alpha_s, mode=MGX_FP64):
        """Pick the fastest kernel / blocks-per-SM for these inputs (mgx_process_autotune)."""
        import torch
        n = momenta.shape[0]
        self.set_kernel(MGX_KERNEL_THREAD)
        self.set_blocks_per_sm(4)
        ws = self.workspace(n, mode)
        me = torch.empty(n, dtype=torch.float64, device=momenta.device)
        k, b = ctypes.c_int(), ctypes.c_int()
        _check(lib().mgx_process_autotune(self._h, n, _ptr(momenta), _ptr(alpha_s), mode, _ptr(ws), ws.numel(),
                                          _stream(momenta.device), ctypes.byref(k), ctypes.byref(b), _ptr(me)),
               "mgx_process_autotune")
        self._ws = {}
        return k.value, b.value

    def device_errors(self, reset=True):
        """Tensor-core waits that ran out since the last reset (synchronise the stream first)."""
        c = ctypes.c_int()
        _check(lib().mgx_process_device_errors(self._h, ctypes.byref(c), int(reset)), "mgx_process_device_errors")
        return c.value

    def set_tc_wait_test(self, skip_mma, wait_ms=1000.0):
        """Test hook: with skip_mma the tensor-core colour sum issues no MMA and its waits run out."""
        _check(lib().mgx_process_set_tc_wait_test(self._h, int(skip_mma), float(wait_ms)),
               "mgx_process_set_tc_wait_test")

    def fp64_ops_per_event(self, mode=MGX_FP64):
        """Float64 instructions per event (fma, mul, add one each)."""
        return lib().mgx_fp64_ops_per_event(self._h, mode)

    def fp64_flops_per_event(self, mode=MGX_FP64):
        """Float64 flops per event (fma counted as two)."""
        return lib().mgx_fp64_flops_per_event(self._h, mode)

    def kernel_launches(self, nevt, mode=MGX_FP64):
        """Kernels one compute() of nevt events launches."""
        n = lib().mgx_kernel_launches(self._h, nevt, mode)
        if n < 0:
            raise MgxError("mgx_kernel_launches: invalid argument")
        return n

    def compute(self, momenta, alpha_s, rnd_hel=None, rnd_col=None, mode=MGX_FP64, mh=False, colw=False,
                stream=None, out=None):
        """Device tensors in, device tensors out (asynchronous on `stream`)."""
        import torch
        nevt = momenta.shape[0]
        dev = momenta.device
        for t in (momenta, alpha_s, rnd_hel, rnd_col):
            if t is not None and (not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous()):
                raise MgxError("inputs must be contiguous float64 CUDA tensors")
        if momenta.shape[1:] != (self.npar, 4):
            raise MgxError(f"momenta must be [nevt, {self.npar}, 4]")
        o = out or {}
        me = o.get("me") if o.get("me") is not None else torch.empty(nevt, dtype=torch.float64, device=dev)
        sel = rnd_hel is not None and rnd_col is not None
        sh = (o.get("selhel") if o.get("selhel") is not None else torch.empty(nevt, dtype=torch.int32, device=dev)) if sel else None
        sc = (o.get("selcol") if o.get("selcol") is not None else torch.empty(nevt, dtype=torch.int32, device=dev)) if sel else None
        mh_t = torch.empty((nevt, self.ngood), dtype=torch.float64, device=dev) if mh else None
        cw_t = torch.empty((nevt, self.ncol), dtype=torch.float64, device=dev) if colw else None
        ws = self.workspace(nevt, mode)
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        _check(lib().mgx_compute_ex(self._h, nevt, _ptr(momenta), _ptr(alpha_s), _ptr(rnd_hel), _ptr(rnd_col),
                                    _ptr(me), _ptr(sh), _ptr(sc), _ptr(mh_t), _ptr(cw_t), mode, _ptr(ws),
                                    ws.numel(), ctypes.c_void_p(st.cuda_stream)), "mgx_compute")
        res = {"me": me}
        if sel:
            res["selhel"], res["selcol"] = sh, sc
        if mh:
            res["mh"] = mh_t
        if colw:
            res["colw"] = cw_t
        return res

    def compute_host(self, momenta, alpha_s, rnd_hel, rnd_col, me, selhel, selcol, mode=MGX_FP64, stream=None):
        """Host (ideally pinned) tensors in and out; copies happen inside the call."""
        import torch
        nevt = momenta.shape[0]
        ws = self.workspace(nevt, mode, host=True)
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        _check(lib().mgx_compute_host(self._h, nevt, _ptr(momenta), _ptr(alpha_s), _ptr(rnd_hel), _ptr(rnd_col),
                                      _ptr(me), _ptr(selhel), _ptr(selcol), mode, _ptr(ws), ws.numel(),
                                      ctypes.c_void_p(st.cuda_stream)), "mgx_compute_host")
