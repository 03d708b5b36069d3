"""The process compiler's op tables run on the CPU by a float64 numpy interpreter of the kernels'
op semantics (`op_emulator.py`), against the oracle: me, every helicity's |M_h|^2 and the colour
weights to the float64 parity bar, selections equal away from near-ties.  This checks what the
compiler emits (block offsets, helicity masks, headers, sum currents, runs, phases, colour flows
and their first writes) without a GPU; the GPU tests check the kernels on the same tables."""
import numpy as np
import pytest

from phasespace import WORKLOADS, make_inputs
from oracle.matrix_element import get as oracle_get
from _parity import TOL, bounds, check_selection
from op_emulator import Emulator

CASES = [("eemumu", 64), ("ggtt", 64), ("ggttg", 48), ("ggttgg", 32), ("gu_tataggu", 32), ("ggttggg", 2)]


def _check(wl, mom, a, rh, rc, got):
    ref = oracle_get(wl.process).evaluate(mom, a, rh, rc)
    rel = np.abs(got["me"] / ref["me"] - 1.0)
    assert np.all(rel <= bounds(wl.process, mom, a, rel)), f"me: max rel {rel.max():.3e}"
    dmh = np.abs(got["mh"] - ref["mh"]) / ref["mh"].sum(axis=1, keepdims=True)
    assert np.all(dmh <= bounds(wl.process, mom, a, dmh))
    dcw = np.abs(got["colw"] - ref["colw"]) / ref["colw"].sum(axis=1, keepdims=True)
    assert np.all(dcw <= bounds(wl.process, mom, a, dcw))
    check_selection(got["selhel"], ref["selhel"], ref["mh"], rh, TOL, f"{wl.name} selhel")
    check_selection(got["selcol"], ref["selcol"], ref["colw"], rc, TOL, f"{wl.name} selcol")


@pytest.mark.parametrize("name,nevt", CASES)
def test_op_tables_match_oracle(name, nevt):
    """The thread-per-event program: ops in order, each current's variants together."""
    wl = WORKLOADS[name]
    mom, a, rh, rc = make_inputs(wl, nevt)
    _check(wl, mom, a, rh, rc, Emulator(wl.process).evaluate(mom, a, rh, rc))


@pytest.mark.parametrize("name,nevt", [c for c in CASES if c[0] != "ggttggg"])
def test_block_schedule_matches_oracle_without_races(name, nevt):
    """The block-per-event schedule (waves of header and variant items, then amplitude steps into
    zeroed jamps): the same results, and no item of a wave touches a slot that another item of
    that wave writes, so the block's threads may run a wave's items in any order."""
    wl = WORKLOADS[name]
    mom, a, rh, rc = make_inputs(wl, nevt)
    _check(wl, mom, a, rh, rc, Emulator(wl.process).evaluate_cta(mom, a, rh, rc))


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_work_counts_match_execution(name):
    """The compiler's work counts per event (variants per vertex kind, sum-current additions,
    header tables, amplitude groups, terms, runs and flow updates), which the library's float64
    work model multiplies by per-op instruction counts for the roofline, equal what one run of
    the tables executes."""
    wl = WORKLOADS[name]
    mom, a, _, _ = make_inputs(wl, 1)
    E = Emulator(wl.process)
    E.evaluate(mom, a)
    c = E.P.flop_counts
    for k in ("var_ffv_f", "var_ffv_fb", "var_ffv_v", "var_vvv", "var_vvvv", "var_bil", "var_rbil", "sum_adds",
              "vvv_hdr", "vvvv_hdr", "slash_hdr", "slash_pref_hdr", "amp", "amp_terms", "amp_runs", "amp_flows"):
        assert E.count[k] == c[k], (k, E.count[k], c[k])


@pytest.mark.parametrize("name,nevt", [c for c in CASES if c[0] != "ggttggg"])
def test_helicity_groups_match_oracle(name, nevt):
    """The helicity-parallel program: per group of helicities (their bits on a set of fixed legs),
    a fresh NaN workspace in which only that group's current variants, header tables and
    amplitudes are computed.  Every single fixed leg and a seeded choice of larger leg sets must
    reproduce the oracle, so no group reads a variant or table that only another group computes."""
    wl = WORKLOADS[name]
    mom, a, rh, rc = make_inputs(wl, nevt)
    em = Emulator(wl.process)
    npar = em.P.npar
    rng = np.random.default_rng(len(name))
    fixes = [1 << b for b in range(npar)]
    fixes += sorted({int(x) for x in rng.integers(1, 1 << npar, size=4)})
    for fix in fixes:
        _check(wl, mom, a, rh, rc, em.evaluate_groups(mom, a, fix, rh, rc))


@pytest.mark.parametrize("name,nevt", [c for c in CASES if c[0] != "ggttggg"])
def test_diagram_split_parts_match_oracle(name, nevt):
    """The diagram-split program: every part of the compiler's 2-, 4- and 8-part splits runs only
    its ops (in program order, with the thread program's block offsets) on a fresh NaN workspace
    into zeroed partial jamps, alone and within helicity groups; the summed partial jamps must give
    the oracle's results.  A part missing an op it reads, or reading a block after another of its
    ops reused it, fails.  The parts cover every amplitude group exactly once."""
    from op_emulator import OP_AMP
    wl = WORKLOADS[name]
    mom, a, rh, rc = make_inputs(wl, nevt)
    em = Emulator(wl.process)
    amps = [i for i, op in enumerate(em.P.ops) if op[0] == OP_AMP]
    for nparts, parts in em.P.splits.items():
        assert 1 <= len(parts) <= nparts
        assert sorted(i for p in parts for i in p if em.P.ops[i][0] == OP_AMP) == amps
        for fix in (0, 1 << (em.P.npar - 1)):
            _check(wl, mom, a, rh, rc, em.evaluate_parts(mom, a, parts, fix, rh, rc))
