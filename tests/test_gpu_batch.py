"""Batched multi-process launch, CUDA-graph replay and autotuning: results against the float64
oracle (float64 and mixed float32 colour sum, per-event alpha_s), and identical to the
per-process entry point."""
import numpy as np
import pytest

from phasespace import WORKLOADS, make_inputs
from oracle.matrix_element import get as oracle_get
from _parity import TOL, bounds, check_selection

pytestmark = pytest.mark.gpu

SET = [("ggtt", 3000), ("ggttg", 700), ("ggttgg", 300), ("gu_tataggu", 129)]


def _setup():
    import torch
    import paper_2503_21935_gb300 as pkg
    dev = torch.device("cuda:0")
    procs, inputs, outs, refs = [], [], [], []
    for name, n in SET:
        wl = WORKLOADS[name]
        mom, a, rh, rc = make_inputs(wl, n)
        t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
        inp = (t(mom), t(a), t(rh), t(rc))
        p = pkg.Process(wl.process)
        p.set_kernel(pkg.MGX_KERNEL_THREAD)   # the batch kernel runs the same per-thread code
        ref = p.compute(*inp)
        p.set_kernel(pkg.MGX_KERNEL_AUTO)
        procs.append(p)
        inputs.append(inp)
        outs.append({"me": torch.zeros(n, dtype=torch.float64, device=dev),
                     "selhel": torch.zeros(n, dtype=torch.int32, device=dev),
                     "selcol": torch.zeros(n, dtype=torch.int32, device=dev)})
        refs.append(ref)
    return pkg, procs, inputs, outs, refs


def _same(outs, refs):
    import torch
    for o, r in zip(outs, refs):
        assert torch.equal(o["me"], r["me"])
        assert torch.equal(o["selhel"], r["selhel"]) and torch.equal(o["selcol"], r["selcol"])


def test_batch_equals_per_process():
    import torch
    pkg, procs, inputs, outs, refs = _setup()
    b = pkg.Batch(procs)
    b.compute(inputs, outs)
    torch.cuda.synchronize()
    _same(outs, refs)


def test_batch_graph_replay_and_autotune():
    import torch
    pkg, procs, inputs, outs, refs = _setup()
    b = pkg.Batch(procs)
    bps, epi = b.autotune(inputs, outs)
    assert bps in (2, 3, 4) and len(epi) == len(procs)
    assert all(e in (64, 128, 256, 512, 1024, 2048, 4096) for e in epi)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        b.capture(inputs, outs, st)
        for _ in range(2):
            for o in outs:
                o["me"].zero_()
            b.replay(st)
    st.synchronize()
    _same(outs, refs)


def test_process_autotune_keeps_results():
    import torch
    import paper_2503_21935_gb300 as pkg
    wl = WORKLOADS["ggttg"]
    mom, a, _, _ = make_inputs(wl, 20000)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    p = pkg.Process(wl.process)
    ref = p.compute(t(mom), t(a))["me"].clone()
    k, bps = p.autotune(t(mom), t(a))
    assert k in (1, 2)
    got = p.compute(t(mom), t(a))["me"]
    assert torch.equal(got, ref) or (got / ref - 1).abs().max().item() < 1e-14


@pytest.mark.parametrize("mode,bound", [(0, TOL), (1, 1e-5)], ids=["fp64", "mixed_fp32"])
def test_batch_matches_oracle(mode, bound):
    """Each process of one batched launch against the oracle on a sample of its events (the first,
    the last and a seeded random choice), with alpha_s drawn per event."""
    import torch
    import paper_2503_21935_gb300 as pkg
    dev = torch.device("cuda:0")
    sets = [("ggtt", 3000, 64), ("ggttg", 700, 48), ("ggttgg", 300, 32), ("gu_tataggu", 129, 32)]
    procs, inputs, outs, host = [], [], [], []
    for name, n, _ in sets:
        wl = WORKLOADS[name]
        mom, a, rh, rc = make_inputs(wl, n, alpha_s_range=(0.08, 0.2))
        t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
        procs.append(pkg.Process(wl.process))
        inputs.append((t(mom), t(a), t(rh), t(rc)))
        outs.append({"me": torch.full((n,), float("nan"), dtype=torch.float64, device=dev),
                     "selhel": torch.full((n,), -1, dtype=torch.int32, device=dev),
                     "selcol": torch.full((n,), -1, dtype=torch.int32, device=dev)})
        host.append((mom, a, rh, rc))
    b = pkg.Batch(procs)
    b.compute(inputs, outs, mode=mode)
    torch.cuda.synchronize()
    rng = np.random.default_rng(77)
    for (name, n, k), (mom, a, rh, rc), o in zip(sets, host, outs):
        wl = WORKLOADS[name]
        idx = np.unique(np.concatenate([[0, n - 1], rng.choice(n, k - 2, replace=False)]))
        ref = oracle_get(wl.process).evaluate(mom[idx], a[idx], rh[idx], rc[idx])
        me = o["me"].cpu().numpy()[idx]
        rel = np.abs(me / ref["me"] - 1.0)
        if mode == 0:
            assert np.all(rel <= bounds(wl.process, mom[idx], a[idx], rel)), f"{name}: max rel {rel.max():.3e}"
        else:
            assert rel.max() <= bound, f"{name}: max rel {rel.max():.3e}"
        check_selection(o["selhel"].cpu().numpy()[idx], ref["selhel"], ref["mh"], rh[idx], bound,
                        f"batch {name} mode {mode} selhel")
        check_selection(o["selcol"].cpu().numpy()[idx], ref["selcol"], ref["colw"], rc[idx], TOL,
                        f"batch {name} mode {mode} selcol")
