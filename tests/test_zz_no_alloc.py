"""The allocation-free entry point (mgx_compute_noalloc) against mgx_compute, through the C ABI.

Some callers cannot allocate device memory where they evaluate matrix elements: a Fortran event
loop that links the library but has no CUDA allocator of its own, or a plugin inside a framework
that owns the device memory pool and forbids cudaMalloc from third-party code.  They call
mgx_compute_noalloc, whose workspace is a fixed module-scope device array.  Its results must equal
those of the ordinary entry point (caller-provided workspace, same thread-per-event kernel) within
the float64 parity tolerance, on two calls in a row (the array keeps the previous call's contents),
in both modes it accepts.  The file name sorts last so that pytest collects it after every other
test file: a run that stops at the first failure has then already run all the other tests.
"""
import ctypes

import numpy as np
import pytest

from phasespace import WORKLOADS, make_inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "mixed_fp32"])
@pytest.mark.parametrize("name,nevt", [("ggttgg", 3000), ("ggttggg", 40)])
def test_noalloc_matches_compute(name, nevt, mode):
    import torch
    import paper_2503_21935_gb300 as pkg
    lib = pkg.lib()
    assert lib.mgx_noalloc_scratch_bytes() == 128 << 20
    wl = WORKLOADS[name]
    mom, a, rh, rc = make_inputs(wl, nevt)
    dev = torch.device("cuda:0")
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    M, A, RH, RC = t(mom), t(a), t(rh), t(rc)
    proc = pkg.Process(wl.process, device=0)
    proc.set_kernel(pkg.MGX_KERNEL_THREAD)     # the kernel the fixed-scratch entry point runs
    ref = proc.compute(M, A, RH, RC, mode=mode)
    torch.cuda.synchronize()
    ptr = lambda x: ctypes.c_void_p(x.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    for call in range(2):
        me = torch.full((nevt,), float("nan"), dtype=torch.float64, device=dev)
        sh = torch.full((nevt,), -1, dtype=torch.int32, device=dev)
        sc = torch.full((nevt,), -1, dtype=torch.int32, device=dev)
        rc_ = lib.mgx_compute_noalloc(proc._h, nevt, ptr(M), ptr(A), ptr(RH), ptr(RC), ptr(me), ptr(sh), ptr(sc),
                                      mode, stream)
        assert rc_ == 0, f"call {call}: {pkg.status_string(rc_)} ({rc_})"
        torch.cuda.synchronize()
        rel = (me / ref["me"] - 1.0).abs().max().item()
        assert rel <= TOL, f"call {call}: max rel {rel:.3e}"
        assert torch.equal(sh, ref["selhel"]) and torch.equal(sc, ref["selcol"])
