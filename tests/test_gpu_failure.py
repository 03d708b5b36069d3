"""Failure detection on the GPU without a fault: the tensor-core colour sum's bounded waits.

Every wait of the fused tcgen05 colour sum for its own MMAs has a time limit.  The test hook
mgx_process_set_tc_wait_test makes the kernel issue no MMA, so each block's first wait runs out
after 1 ms (nothing is in flight, nothing hangs).  The launch must return, the block must count
the error in the process's device counter and mark its events NaN (selections -1), and the context
must stay usable: the next normal call gives the oracle's results and no new error."""
import numpy as np
import pytest

from phasespace import WORKLOADS, make_inputs
from oracle.matrix_element import get as oracle_get

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [2, 3], ids=["tf32", "bf16x3"])
def test_tensor_core_wait_runs_out_and_recovers(mode):
    import torch
    import paper_2503_21935_gb300 as pkg
    wl = WORKLOADS["ggttg"]
    n = 3 * 128 + 5                       # four blocks, the last one ragged
    mom, a, rh, rc = make_inputs(wl, n)
    dev = torch.device("cuda:0")
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    M, A, RH, RC = t(mom), t(a), t(rh), t(rc)
    proc = pkg.Process(wl.process, device=0)
    assert proc.device_errors(reset=True) == 0
    proc.set_tc_wait_test(True, wait_ms=1.0)
    try:
        r = proc.compute(M, A, RH, RC, mode=mode)
        torch.cuda.synchronize()
    finally:
        proc.set_tc_wait_test(False)
    me = r["me"].cpu().numpy()
    assert np.isnan(me).all()
    assert (r["selhel"].cpu().numpy() == -1).all() and (r["selcol"].cpu().numpy() == -1).all()
    blocks = (n + 127) // 128
    assert proc.device_errors(reset=True) == blocks           # one count per block, each gave up once
    assert proc.device_errors(reset=False) == 0
    # the context and the process are usable: a normal call matches the oracle
    r = proc.compute(M, A, RH, RC, mode=mode)
    torch.cuda.synchronize()
    ref = oracle_get(wl.process).evaluate(mom, a)
    assert np.abs(r["me"].cpu().numpy() / ref["me"] - 1.0).max() <= 1e-5
    assert proc.device_errors(reset=False) == 0
    with pytest.raises(pkg.MgxError):
        proc.set_tc_wait_test(True, wait_ms=0.0)


def test_mlp_gemm_wait_runs_out_and_recovers():
    """The network's tcgen05 GEMMs under the same hook: every tile's wait runs out after 1 ms, the
    outputs are NaN, the errors are counted, and a normal forward pass afterwards is finite."""
    import torch
    import paper_2503_21935_gb300 as pkg
    net = pkg.Mlp(seed=3)
    x = np.random.default_rng(0).normal(size=(300, 24)).astype(np.float32)
    assert net.device_errors() == 0
    net.set_wait_test(True, wait_ms=1.0)
    try:
        y = net.forward(x)
    finally:
        net.set_wait_test(False)
    assert np.isnan(y).all()
    # inference: 4 layer launches of 3 persistent blocks (one 128-row tile each), each block gives up once
    assert net.device_errors(reset=True) == 12
    t = np.zeros(300, dtype=np.float32)
    net.set_wait_test(True, wait_ms=1.0)
    try:
        loss, g = net.gradients(x, t)                 # the training GEMMs under the same hook
    finally:
        net.set_wait_test(False)
    assert np.isnan(g).any() and net.device_errors(reset=True) > 0
    y = net.forward(x)
    loss, g = net.gradients(x, t)
    assert np.isfinite(y).all() and np.isfinite(g).all() and net.device_errors(reset=False) == 0
