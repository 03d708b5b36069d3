"""Parity at the benchmark workloads' full sizes, in the launch configuration bench.py times (FP64,
default kernel, one launch over the whole batch): sampled events against the oracle one by one
(with the first and last event of the batch among them), and properties that hold for every event."""
import numpy as np
import pytest

from phasespace import WORKLOADS, make_inputs
from oracle.matrix_element import get as oracle_get
from _parity import TOL, bounds, check_selection

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,nsample", [("eemumu", 256), ("ggttgg", 48), ("ggttggg", 10)])
def test_full_size_sampled(name, nsample):
    import torch
    import paper_2503_21935_gb300 as pkg
    wl = WORKLOADS[name]
    nevt = wl.nevt
    mom, a, rh, rc = make_inputs(wl, nevt)
    dev = torch.device("cuda:0")
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    proc = pkg.Process(wl.process, device=0)
    res = proc.compute(t(mom), t(a), t(rh), t(rc), mode=pkg.MGX_FP64)
    torch.cuda.synchronize()
    me = res["me"].cpu().numpy()
    sh = res["selhel"].cpu().numpy()
    sc = res["selcol"].cpu().numpy()
    # every event: finite, positive, selections in range
    assert np.all(np.isfinite(me)) and np.all(me > 0.0)
    assert np.all(np.isin(sh, proc.good_helicities))
    assert sc.min() >= 0 and sc.max() < proc.ncol
    # sampled events against the oracle
    rng = np.random.default_rng(2024)
    idx = np.unique(np.concatenate([[0, nevt - 1], rng.choice(nevt, nsample - 2, replace=False)]))
    ref = oracle_get(wl.process).evaluate(mom[idx], a[idx], rh[idx], rc[idx])
    rel = np.abs(me[idx] / ref["me"] - 1.0)
    assert np.all(rel <= bounds(wl.process, mom[idx], a[idx], rel)), f"max rel {rel.max():.3e}"
    check_selection(sh[idx], ref["selhel"], ref["mh"], rh[idx], TOL, f"{name} selhel")
    check_selection(sc[idx], ref["selcol"], ref["colw"], rc[idx], TOL, f"{name} selcol")
