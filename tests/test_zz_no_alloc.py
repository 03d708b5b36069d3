"""The allocation-free entry point (mgx_compute_noalloc) against mgx_compute, through the C ABI.

Callers that cannot allocate device memory (a Fortran event loop without a CUDA allocator, a
plugin in a framework that owns the device memory pool) use mgx_compute_noalloc, whose workspace
is a fixed module-scope device array.  Its results must equal those of the ordinary entry point
(which uses a caller-provided workspace) within the float64 parity tolerance, on two calls in a
row (the array keeps the previous call's contents).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from phasespace import WORKLOADS, make_inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _noalloc(lib):
    f = lib.mgx_compute_noalloc
    P = ctypes.c_void_p
    f.restype = ctypes.c_int
    f.argtypes = [P, ctypes.c_int64, P, P, P, P, P, P, P, ctypes.c_int, P]
    lib.mgx_noalloc_scratch_bytes.restype = ctypes.c_size_t
    return f


@pytest.mark.parametrize("name,nevt", [("ggttgg", 3000), ("ggttggg", 40)])
def test_noalloc_matches_compute(name, nevt):
    import torch
    import paper_2503_21935_gb300 as pkg
    lib = pkg.lib()
    noalloc = _noalloc(lib)
    assert lib.mgx_noalloc_scratch_bytes() == 128 << 20
    wl = WORKLOADS[name]
    mom, a, rh, rc = make_inputs(wl, nevt)
    dev = torch.device("cuda:0")
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    M, A, RH, RC = t(mom), t(a), t(rh), t(rc)
    proc = pkg.Process(wl.process, device=0)
    proc.set_kernel(pkg.MGX_KERNEL_THREAD)     # the kernel the fixed-scratch entry point runs
    ref = proc.compute(M, A, RH, RC, mode=pkg.MGX_FP64)
    torch.cuda.synchronize()
    ptr = lambda x: ctypes.c_void_p(x.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    for call in range(2):
        me = torch.full((nevt,), float("nan"), dtype=torch.float64, device=dev)
        sh = torch.full((nevt,), -1, dtype=torch.int32, device=dev)
        sc = torch.full((nevt,), -1, dtype=torch.int32, device=dev)
        rc_ = noalloc(proc._h, nevt, ptr(M), ptr(A), ptr(RH), ptr(RC), ptr(me), ptr(sh), ptr(sc),
                      pkg.MGX_FP64, stream)
        assert rc_ == 0, lib.mgx_status_string(rc_)
        torch.cuda.synchronize()
        rel = (me / ref["me"] - 1.0).abs().max().item()
        assert rel <= TOL, f"call {call}: max rel {rel:.3e}"
        assert torch.equal(sh, ref["selhel"]) and torch.equal(sc, ref["selcol"])
