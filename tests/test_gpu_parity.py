"""GPU parity: the CUDA path through the C ABI against the float64 oracle, element by element.

Bar (float64 path): per-event relative deviation of me, and of every per-helicity
|M_h|^2 and colour weight relative to the event total, at most 1e-12, except for events
the oracle's condition estimate marks cancellation-limited (reported, held to 1e-14 x kappa);
helicity and colour selection bit-exact except where a cumulative weight lies within 1e-12 of
the random threshold.
"""
import numpy as np
import pytest

from phasespace import WORKLOADS, make_inputs, rambo, incoming_beams
from oracle.matrix_element import get as oracle_get
from _parity import TOL, bounds as _bounds, check_selection, check_mode

pytestmark = pytest.mark.gpu

_procs = {}


def _proc(name):
    import paper_2503_21935_gb300 as pkg
    if name not in _procs:
        _procs[name] = pkg.Process(name, device=0)
    return _procs[name]


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _run(proc, mom, a, rh, rc, mode=0):
    import torch
    r = proc.compute(_dev(mom), _dev(a), _dev(rh), _dev(rc), mode=mode, mh=True, colw=True)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in r.items()}


CASES = [("eemumu", 300), ("ggtt", 300), ("ggttg", 260), ("ggttgg", 160), ("ggttggg", 20), ("gu_tataggu", 140)]
KERNELS = {"auto": 0, "thread": 1, "cta": 2, "smem": 3, "helicity": 4, "split": 5}
SMEM_PROCESSES = ("eemumu", "ggtt")        # per-thread workspace small enough for shared memory


_refs = {}


def _oracle(process, mom, a, rh, rc):
    """The oracle's outputs for one seeded sample, computed once per (process, sample size)."""
    key = (process, mom.shape[0], hash(mom.tobytes()), hash(a.tobytes()), hash(rh.tobytes()), hash(rc.tobytes()))
    if key not in _refs:
        _refs[key] = oracle_get(process).evaluate(mom, a, rh, rc)
    return _refs[key]


@pytest.mark.parametrize("kernel", ["auto", "thread", "cta", "smem", "helicity", "split"])
@pytest.mark.parametrize("name,nevt", CASES)
def test_parity_fp64(name, nevt, kernel):
    wl = WORKLOADS[name]
    mom, a, rh, rc = make_inputs(wl, nevt)
    proc = _proc(wl.process)
    if kernel == "cta" and name == "ggttggg":
        pytest.skip("g g > t t~ g g g: current store does not fit in shared memory (thread kernel only)")
    if kernel == "smem" and name not in SMEM_PROCESSES:
        pytest.skip("per-thread workspace too large for the shared-memory kernel")
    proc.set_kernel(KERNELS[kernel])
    try:
        got = _run(proc, mom, a, rh, rc)
    finally:
        proc.set_kernel(0)
    ref = _oracle(wl.process, mom, a, rh, rc)
    rel = np.abs(got["me"] / ref["me"] - 1.0)
    assert np.all(rel <= _bounds(wl.process, mom, a, rel)), f"me: max rel {rel.max():.3e}"
    tot = ref["mh"].sum(axis=1, keepdims=True)
    good = proc.good_helicities
    assert np.abs(ref["mh"][:, [h for h in range(proc.nhel) if h not in good]]).max(initial=0.0) == 0.0
    dmh = np.abs(got["mh"] - ref["mh"][:, good]) / tot
    assert np.all(dmh <= _bounds(wl.process, mom, a, dmh))
    ctot = ref["colw"].sum(axis=1, keepdims=True)
    dcw = np.abs(got["colw"] - ref["colw"]) / ctot
    assert np.all(dcw <= _bounds(wl.process, mom, a, dcw))
    check_selection(got["selhel"], ref["selhel"], ref["mh"], rh, TOL, f"{name} {kernel} selhel")
    check_selection(got["selcol"], ref["selcol"], ref["colw"], rc, TOL, f"{name} {kernel} selcol")


def _check_fp64(proc, wl, mom, a, rh, rc, got, what):
    """Every output of a float64 run against the oracle at the float64 bar."""
    ref = oracle_get(wl.process).evaluate(mom, a, rh, rc)
    rel = np.abs(got["me"] / ref["me"] - 1.0)
    assert np.all(rel <= _bounds(wl.process, mom, a, rel)), f"{what}: me max rel {rel.max():.3e}"
    tot = ref["mh"].sum(axis=1, keepdims=True)
    dmh = np.abs(got["mh"] - ref["mh"][:, proc.good_helicities]) / tot
    assert np.all(dmh <= _bounds(wl.process, mom, a, dmh))
    dcw = np.abs(got["colw"] - ref["colw"]) / ref["colw"].sum(axis=1, keepdims=True)
    assert np.all(dcw <= _bounds(wl.process, mom, a, dcw))
    check_selection(got["selhel"], ref["selhel"], ref["mh"], rh, TOL, f"{what} selhel")
    check_selection(got["selcol"], ref["selcol"], ref["colw"], rc, TOL, f"{what} selcol")
    return ref


@pytest.mark.parametrize("kernel", ["auto", "thread", "cta", "helicity", "split"])
@pytest.mark.parametrize("name,nevt", [("ggttg", 200), ("ggttgg", 120), ("gu_tataggu", 100)])
def test_parity_per_event_alpha_s(name, nevt, kernel):
    """alpha_s drawn per event in [0.08, 0.2): the per-event coupling (4 pi alpha_s)^p of each event
    must be its own (a kernel reading another event's alpha_s, or the first one, fails), and me
    must differ from the constant-alpha_s run by exactly the events' coupling ratio."""
    wl = WORKLOADS[name]
    mom, a, rh, rc = make_inputs(wl, nevt, alpha_s_range=(0.08, 0.2))
    assert a.std() > 0.02
    proc = _proc(wl.process)
    proc.set_kernel(KERNELS[kernel])
    try:
        got = _run(proc, mom, a, rh, rc)
    finally:
        proc.set_kernel(0)
    _check_fp64(proc, wl, mom, a, rh, rc, got, f"{name} {kernel} per-event alpha_s")


@pytest.mark.parametrize("mode,bound", [(1, 1e-5), (2, 1e-5), (3, 1e-5)], ids=["mixed_fp32", "tf32", "bf16x3"])
def test_parity_per_event_alpha_s_reduced_precision(mode, bound):
    """The per-event coupling in the reduced-precision colour sums (applied after the colour sum)."""
    wl = WORKLOADS["ggttgg"]
    mom, a, rh, rc = make_inputs(wl, 130, alpha_s_range=(0.08, 0.2))
    proc = _proc(wl.process)
    got = _run(proc, mom, a, rh, rc, mode=mode)
    ref = _oracle(wl.process, mom, a, rh, rc)
    check_mode(proc, got, ref, rh, rc, bound, f"ggttgg mode {mode} per-event alpha_s")


@pytest.mark.parametrize("name", ["eemumu", "ggtt", "ggttg", "ggttgg", "ggttggg", "gu_tataggu"])
def test_helicity_filter_matches_oracle(name):
    wl = WORKLOADS[name]
    proc = _proc(wl.process)
    # the library's filter events: 16 RAMBO events at 1000 GeV, Philox key = filter seed 0, stream 0
    po, _ = rambo(16, 1000.0, wl.final_masses(), seed=0)
    p = np.concatenate([incoming_beams(16, 1000.0), po], axis=1)
    assert proc.good_helicities == oracle_get(wl.process).helicity_filter(p, np.full(16, 0.118))


MODE_CASES = [("eemumu", 64, 1e-5), ("ggtt", 300, 1e-5), ("ggttg", 200, 1e-5), ("ggttgg", 130, 1e-5),
              ("ggttggg", 12, 1e-5), ("gu_tataggu", 140, 1e-5)]


@pytest.mark.parametrize("kernel", ["thread", "cta", "helicity", "split"])
@pytest.mark.parametrize("name,nevt,bound", MODE_CASES)
def test_parity_mixed_fp32_colour_sum(name, nevt, bound, kernel):
    """Float64 amplitudes, float32 colour sum: me, every |M_h|^2 and the helicity selection at the
    mode's bound; colour weights (float64 jamps) and the colour selection at the float64 bar."""
    if kernel == "cta" and name == "ggttggg":
        pytest.skip("g g > t t~ g g g: current store does not fit in shared memory (thread kernel only)")
    wl = WORKLOADS[name]
    mom, a, rh, rc = make_inputs(wl, nevt)
    proc = _proc(wl.process)
    proc.set_kernel(KERNELS[kernel])
    try:
        got = _run(proc, mom, a, rh, rc, mode=1)
    finally:
        proc.set_kernel(0)
    ref = _oracle(wl.process, mom, a, rh, rc)
    check_mode(proc, got, ref, rh, rc, bound, f"{name} {kernel} mixed_fp32")
    dcw = np.abs(got["colw"] - ref["colw"]) / ref["colw"].sum(axis=1, keepdims=True)
    assert np.all(dcw <= _bounds(wl.process, mom, a, dcw))
    check_selection(got["selcol"], ref["selcol"], ref["colw"], rc, TOL, f"{name} {kernel} mixed_fp32 selcol")


def test_auto_kernel_by_batch_size():
    """AUTO runs a float64 batch of at most 32 events per SM one block per event (no caller
    workspace) when the process has a block-per-event schedule; larger batches, the float mode
    and processes without that schedule take a kernel with a workspace."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    proc = _proc(WORKLOADS["ggttgg"].process)
    assert proc.workspace_bytes(32 * sms) == 0 and proc.workspace_bytes(32 * sms, mode=1) == 0
    assert proc.plan(32 * sms)[0] == 2
    assert proc.workspace_bytes(32 * sms + 1) > 0
    assert proc.workspace_bytes(1000, mode=4) > 0
    assert _proc(WORKLOADS["ggttggg"].process).workspace_bytes(100) > 0


@pytest.mark.parametrize("mode", [2, 3], ids=["tf32", "bf16x3"])
@pytest.mark.parametrize("name,nevt,bound", MODE_CASES)
def test_parity_tensor_core_colour_sum(name, nevt, bound, mode):
    """tcgen05 colour sums: jamps as two tf32 terms x the integer-scaled colour matrix (kind::tf32), or
    three bf16 terms x its two bf16 parts (kind::f16); f32 accumulation in tensor memory.  me, every
    |M_h|^2 and the helicity selection at the mode's bound; colour weights (float64 jamps) and the
    colour selection at the float64 bar."""
    wl = WORKLOADS[name]
    mom, a, rh, rc = make_inputs(wl, nevt)
    proc = _proc(wl.process)
    got = _run(proc, mom, a, rh, rc, mode=mode)
    ref = _oracle(wl.process, mom, a, rh, rc)
    check_mode(proc, got, ref, rh, rc, bound, f"{name} mode {mode}")
    dcw = np.abs(got["colw"] - ref["colw"]) / ref["colw"].sum(axis=1, keepdims=True)
    assert np.all(dcw <= _bounds(wl.process, mom, a, dcw))
    check_selection(got["selcol"], ref["selcol"], ref["colw"], rc, TOL, f"{name} mode {mode} selcol")


# float32 amplitudes and colour sum (the paper's float build); bounds are the measured
# per-event maxima on these seeded samples with a margin of about 3x, not a prediction.  The
# electroweak process (Z propagator, photon-Z interference) loses more digits to cancellation.
FLOAT_CASES = [("eemumu", 300, 1e-4), ("ggtt", 300, 1e-4), ("ggttg", 260, 1e-4), ("ggttgg", 160, 1e-4),
               ("ggttggg", 20, 1e-4), ("gu_tataggu", 140, 1e-2)]


@pytest.mark.parametrize("kernel", ["thread", "cta", "smem", "helicity", "split"])
@pytest.mark.parametrize("name,nevt,bound", FLOAT_CASES)
def test_parity_float_mode(name, nevt, bound, kernel):
    """Float32 path: me within the stated bound; |M_h|^2 and colour weights relative to the event total too."""
    wl = WORKLOADS[name]
    mom, a, rh, rc = make_inputs(wl, nevt)
    proc = _proc(wl.process)
    if kernel == "cta" and name == "ggttggg":
        pytest.skip("g g > t t~ g g g: no CTA kernel to select")
    if kernel == "smem" and name not in SMEM_PROCESSES:
        pytest.skip("per-thread workspace too large for the shared-memory kernel")
    proc.set_kernel(KERNELS[kernel])   # the float path runs the thread-per-event or helicity-parallel kernel
    try:
        got = _run(proc, mom, a, rh, rc, mode=4)
    finally:
        proc.set_kernel(0)
    ref = _oracle(wl.process, mom, a, rh, rc)
    assert np.all(np.isfinite(got["me"]))
    assert np.abs(got["me"] / ref["me"] - 1.0).max() <= bound
    tot = ref["mh"].sum(axis=1, keepdims=True)
    assert (np.abs(got["mh"] - ref["mh"][:, proc.good_helicities]) / tot).max() <= bound
    assert (np.abs(got["colw"] - ref["colw"]) / ref["colw"].sum(axis=1, keepdims=True)).max() <= bound


@pytest.mark.parametrize("mode", [2, 3], ids=["tf32", "bf16x3"])
def test_tensor_core_colour_sum_chunks_and_tail(mode):
    """Several chunks and a ragged last tile give the same me as the float32 SIMT colour sum."""
    wl = WORKLOADS["ggttg"]
    n = 100003
    mom, a, rh, rc = make_inputs(wl, n)
    proc = _proc(wl.process)
    tc = _run(proc, mom, a, rh, rc, mode=mode)
    f32 = _run(proc, mom, a, rh, rc, mode=1)
    assert np.all(np.isfinite(tc["me"]))
    assert np.abs(tc["me"] / f32["me"] - 1.0).max() <= 2e-5


@pytest.mark.parametrize("nevt", [1, 127, 128, 129])
def test_ragged_sizes(nevt):
    wl = WORKLOADS["ggttg"]
    mom, a, rh, rc = make_inputs(wl, nevt)
    got = _run(_proc(wl.process), mom, a, rh, rc)
    ref = oracle_get(wl.process).evaluate(mom, a)
    rel = np.abs(got["me"] / ref["me"] - 1.0)
    assert np.all(rel <= _bounds(wl.process, mom, a, rel))


def test_shared_memory_workspace_kernel_multi_pass_and_auto():
    """The shared-memory-workspace kernel over several passes of its grid equals the global-workspace
    kernel; AUTO takes it for a latency-bound batch and needs no caller workspace then."""
    import paper_2503_21935_gb300 as pkg
    wl = WORKLOADS["ggtt"]
    n = 64 * 152 * 3 + 17
    mom, a, rh, rc = make_inputs(wl, n)
    proc = _proc(wl.process)
    proc.set_kernel(3)
    try:
        assert proc.kernel == 3
        sm = _run(proc, mom, a, rh, rc)
        assert proc.workspace_bytes(n) == 0
    finally:
        proc.set_kernel(1)
    try:
        gl = _run(proc, mom, a, rh, rc)
    finally:
        proc.set_kernel(0)
    assert np.abs(sm["me"] / gl["me"] - 1.0).max() <= TOL
    assert np.array_equal(sm["selhel"], gl["selhel"]) and np.array_equal(sm["selcol"], gl["selcol"])
    assert proc.workspace_bytes(1000) == 0 and proc.workspace_bytes(1 << 20) > 0
    with pytest.raises(pkg.MgxError):
        _proc(WORKLOADS["ggttgg"].process).set_kernel(3)


def _degenerate_events():
    """Hand-built events on the special branches of the spinor and polarisation code: particles
    exactly along +z and -z (massless and massive), massive particles at rest."""
    out = {}
    e = 250.0
    beams = [[e, 0, 0, e], [e, 0, 0, -e]]
    out["e+ e- > mu+ mu-"] = np.array([beams + [[e, 0, 0, e], [e, 0, 0, -e]],
                                       beams + [[e, 0, 0, -e], [e, 0, 0, e]],
                                       beams + [[e, e, 0, 0], [e, -e, 0, 0]]], dtype=float)
    mt = 173.0
    out["g g > t t~"] = np.array([[[mt, 0, 0, mt], [mt, 0, 0, -mt], [mt, 0, 0, 0], [mt, 0, 0, 0]],
                                  [[750, 0, 0, 750], [750, 0, 0, -750], [750, 0, 0, np.sqrt(750 ** 2 - mt ** 2)],
                                   [750, 0, 0, -np.sqrt(750 ** 2 - mt ** 2)]]], dtype=float)
    # a final gluon along the beam axis would make a t-channel propagator vanish (collinear
    # singularity), so the 2 -> 3 event puts the gluon along +x and the tops back to back in z
    pz = np.sqrt(600.0 ** 2 - mt ** 2 - 150.0 ** 2)
    out["g g > t t~ g"] = np.array([[[750, 0, 0, 750], [750, 0, 0, -750], [600, -150, 0, pz], [600, -150, 0, -pz],
                                     [300, 300, 0, 0]]], dtype=float)
    return out


def test_degenerate_kinematics():
    for proc_name, mom in _degenerate_events().items():
        n = mom.shape[0]
        a = np.full(n, 0.118)
        rh = np.linspace(0.1, 0.9, n)
        rc = np.linspace(0.2, 0.8, n)
        proc = _proc(proc_name)
        got = _run(proc, mom, a, rh, rc)
        ref = oracle_get(proc_name).evaluate(mom, a, rh, rc)
        assert np.all(np.isfinite(got["me"]))
        rel = np.abs(got["me"] / ref["me"] - 1.0)
        assert np.all(rel <= _bounds(proc_name, mom, a, rel)), f"{proc_name}: max rel {rel.max():.3e}"
        tot = ref["mh"].sum(axis=1, keepdims=True)
        assert (np.abs(got["mh"] - ref["mh"][:, proc.good_helicities]) / tot).max() <= TOL


def test_empty_batch_and_errors():
    import torch
    import paper_2503_21935_gb300 as pkg
    proc = _proc(WORKLOADS["ggtt"].process)
    z = torch.empty((0, 4, 4), dtype=torch.float64, device="cuda:0")
    r = proc.compute(z, torch.empty(0, dtype=torch.float64, device="cuda:0"))
    assert r["me"].numel() == 0
    with pytest.raises(pkg.MgxError):
        pkg.Process("g g > nothing", device=0)
    with pytest.raises(pkg.MgxError):
        proc.compute(torch.zeros((4, 5, 4), dtype=torch.float64, device="cuda:0"),
                     torch.zeros(4, dtype=torch.float64, device="cuda:0"))
    # too-small workspace is rejected before launch (the thread-per-event kernel needs one)
    import ctypes
    proc.set_kernel(1)
    m = torch.zeros((8, 4, 4), dtype=torch.float64, device="cuda:0")
    o = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    ws = torch.empty(256, dtype=torch.uint8, device="cuda:0")
    rc = pkg.lib().mgx_compute(proc._h, 8, ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(o.data_ptr()), None, None,
                               ctypes.c_void_p(o.data_ptr()), None, None, 0, ctypes.c_void_p(ws.data_ptr()), 256, None)
    proc.set_kernel(0)
    assert rc == -5
    for bad_mode in (5, 9, -1):   # unassigned mode numbers
        rc = pkg.lib().mgx_compute(proc._h, 8, ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(o.data_ptr()), None,
                                   None, ctypes.c_void_p(o.data_ptr()), None, None, bad_mode,
                                   ctypes.c_void_p(ws.data_ptr()), 256, None)
        assert rc == -7


def test_host_buffer_entry_point():
    import torch
    wl = WORKLOADS["ggttg"]
    mom, a, rh, rc = make_inputs(wl, 200)
    proc = _proc(wl.process)
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    me = torch.empty(200, dtype=torch.float64).pin_memory()
    sh = torch.empty(200, dtype=torch.int32).pin_memory()
    sc = torch.empty(200, dtype=torch.int32).pin_memory()
    proc.compute_host(pin(mom), pin(a), pin(rh), pin(rc), me, sh, sc)
    dev = _run(proc, mom, a, rh, rc)
    assert np.array_equal(me.numpy(), dev["me"])
    assert np.array_equal(sh.numpy(), dev["selhel"]) and np.array_equal(sc.numpy(), dev["selcol"])


def test_helicity_kernel_many_passes_and_auto():
    """The helicity-parallel kernel over several passes of its grid (a batch larger than the grid
    holds items) equals the thread kernel; AUTO picks it for a mid-size batch of g g > t t~ g g g
    (which has no block-per-event schedule), and the thread kernel for a full batch."""
    import torch
    import paper_2503_21935_gb300 as pkg
    wl = WORKLOADS["ggttg"]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = 2 * sms * 4 * 128 + 77
    mom, a, rh, rc = make_inputs(wl, n)
    proc = _proc(wl.process)
    proc.set_kernel(4)
    try:
        assert proc.kernel == 4 and proc.kernel_launches(n) == 2
        hp = _run(proc, mom, a, rh, rc)
    finally:
        proc.set_kernel(1)
    try:
        th = _run(proc, mom, a, rh, rc)
    finally:
        proc.set_kernel(0)
    assert np.abs(hp["me"] / th["me"] - 1.0).max() <= TOL
    assert np.array_equal(hp["selhel"], th["selhel"]) and np.array_equal(hp["selcol"], th["selcol"])
    big = _proc(WORKLOADS["ggttggg"].process)
    assert big.kernel_launches(2000) in (2, 3) and big.kernel_launches(1 << 20) == 1


@pytest.mark.parametrize("name", ["ggttgg", "ggttggg"])
def test_split_kernel_many_passes(name):
    """The diagram-split kernel with items over several passes of its grid (and, for g g > t t~ g g g,
    parts larger than a block) equals the whole-event thread kernel on the same events."""
    import torch
    wl = WORKLOADS[name]
    n = 3000 if name == "ggttgg" else 700
    mom, a, rh, rc = make_inputs(wl, n)
    proc = _proc(wl.process)
    proc.set_kernel(5)
    try:
        assert proc.kernel == 5 and proc.kernel_launches(n) == 3
        sp = _run(proc, mom, a, rh, rc)
    finally:
        proc.set_kernel(1)
    try:
        th = _run(proc, mom, a, rh, rc)
    finally:
        proc.set_kernel(0)
    rel = np.abs(sp["me"] / th["me"] - 1.0)
    assert np.all(rel <= _bounds(wl.process, mom, a, rel))
    check_selection(sp["selhel"], th["selhel"], th["mh"], rh, TOL, f"{name} split vs thread selhel")
