"""Throughput of the batched tree-level |M|^2 hot path on GB300.

Workload: g g > t t~ g g (123 diagrams, 24 colour flows, 64 helicities), 2^20 flat
RAMBO events per GPU at partonic sqrt(s) = 1500 GeV, m_t = 173 GeV, fixed
alpha_s = 0.118; one step = one mgx_compute over the whole batch (momenta,
alpha_s and random numbers already resident in HBM): external wavefunctions,
every diagram amplitude, jamps, colour sum, helicity sum, helicity and colour
selection.  Metric: |M|^2 evaluations per second (whole job).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--mode fp64|mixed_fp32|mixed_tf32|mixed_bf16x3|float] [--impl reference]
                  [--workload ggttgg|ggttggg] [--kernel auto|thread|cta|smem|helicity|split]

--workload ggttggg (g g > t t~ g g g) and --kernel (a fixed schedule instead of AUTO's choice) serve
profiling captures of the other kernels; the default line is the one above.

Under torchrun each rank processes its own 2^20 events (weak scaling, no data
collective); rank 0 prints one JSON line.  --impl reference times the float64
CPU oracle on the host cores instead (bounded sample of the same workload).
"""
import argparse
import gc
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "ggttgg"
NEVT = 1 << 20
METRIC = "gg->ttgg |M|^2 evals/s (FP64)"
METRICS = {"ggttgg": METRIC, "ggttggg": "gg->ttggg |M|^2 evals/s (FP64)"}
KERNELS = {"auto": 0, "thread": 1, "cta": 2, "smem": 3, "helicity": 4, "split": 5}
# FP64 pipe: 152 SMs x 2 DFMA/clk/SM (measured: 1.20 TFLOP/s at 1995 MHz) x 2 flop x 2070 MHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FP64_PEAK_GINST = 152 * 2 * 2.070e9 / 1e9       # float64 instructions per second, any of fma/mul/add
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP32_PEAK_GINST = 152 * 128 * 2.070e9 / 1e9


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--mode", default="fp64", choices=["fp64", "mixed_fp32", "mixed_tf32", "mixed_bf16x3", "float"])
    ap.add_argument("--impl", default="mgx", choices=["mgx", "reference"])
    ap.add_argument("--nevt", type=int, default=NEVT)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(METRICS))
    ap.add_argument("--kernel", default="auto", choices=list(KERNELS))
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ CPU oracle timing
ORACLE_CHUNK = 768      # events per oracle call (bounds its [terms, events, helicities] arrays)


def _oracle_worker(args):
    wl_name, first, n = args
    sys.path.insert(0, ROOT)
    from phasespace import WORKLOADS, make_inputs
    from oracle.matrix_element import get
    wl = WORKLOADS[wl_name]
    mom, a, rh, rc = make_inputs(wl, n, first=first)
    me = get(wl.process)
    me.evaluate(mom[:1], a[:1])          # warm caches / einsum paths outside the timing
    t0 = time.perf_counter()
    for c in range(0, n, ORACLE_CHUNK):
        s = slice(c, c + ORACLE_CHUNK)
        me.evaluate(mom[s], a[s], rh[s], rc[s])
    return time.perf_counter() - t0, n


_ONE_THREAD = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def cpu_oracle_rate(wl_name, per_core, cores):
    """Events/s of the float64 oracle on `cores` single-threaded host processes, per_core events each."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    jobs = [(wl_name, 1000 + i * per_core, per_core) for i in range(cores)]
    saved = {k: os.environ.get(k) for k in _ONE_THREAD}
    os.environ.update({k: "1" for k in _ONE_THREAD})     # spawned workers inherit it before numpy loads
    try:
        t0 = time.perf_counter()
        with ctx.Pool(cores) as pool:
            res = pool.map(_oracle_worker, jobs)
        wall = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    busy = max(t for t, _ in res)
    n = sum(k for _, k in res)
    return n / busy, n, busy, wall


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# the translation unit of the amplitude kernels: mgx.cu, the headers it includes, the generated tables
_KERNEL_SOURCES = ("mgx.cu", "mgx_ops.cuh", "mgx_kernel.cuh", "real.cuh", "colour_tc.cuh", "umma.cuh",
                   os.path.join("generated", "programs.inc"))


def _source_sha():
    """Hash of the sources the amplitude kernels are compiled from (a traffic figure taken on other
    sources no longer describes the kernel)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2503_21935_gb300", "csrc")
    for f in _KERNEL_SOURCES:
        path = os.path.join(csrc, f)
        if os.path.exists(path):
            h.update(open(path, "rb").read())
    return h.hexdigest()[:16]


def _traffic_per_event(kernel, workload):
    """DRAM bytes per event of `kernel` from the committed ncu summary, if taken on this source."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        d = json.load(open(path))
        e = d[f"{kernel}:{workload}"]
        if e.get("source_sha") == _source_sha():
            return e["dram_bytes_per_event"]
    except (OSError, KeyError, ValueError):
        pass
    return None


def _workload_config(nevt, mode, workload=WORKLOAD, ws_bytes=None):
    from phasespace import WORKLOADS
    wl = WORKLOADS[workload]
    cfg = {"workload": f"{wl.process}, {nevt} flat RAMBO events/GPU, sqrt(s)=1500 GeV, mt=173, alpha_s=0.118",
           "process": wl.process, "nevt_per_gpu": nevt, "mode": mode}
    if ws_bytes is None:
        cfg["l2"] = "inputs larger than L2 (192 MiB momenta, 6.3 GB workspace)"
    else:
        cfg["l2"] = (f"workspace {ws_bytes / 2**30:.1f} GiB, "
                     + ("larger than L2" if ws_bytes > (129 << 20) else "smaller than L2 (a profiling case)"))
    return cfg


# ------------------------------------------------------------------ reference arm (oracle)
def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    cores = _host_cores()
    per_core = 384
    rates = []
    for i in range(args.warmup + args.steps):
        r, n, busy, wall = cpu_oracle_rate(args.workload, per_core, cores)
        if i >= args.warmup:
            rates.append((r, n, busy))
    value = statistics.median(r for r, _, _ in rates)
    n = rates[0][1]
    line = {"impl": "reference", "metric": METRICS[args.workload], "value": value, "unit": "events/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(b for _, _, b in rates),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _workload_config(args.nevt, args.mode, args.workload),
            "cpu_baseline": {"value": value, "unit": "events/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step evaluates {n} events of this workload on the host cores "
                                       f"({per_core} events per core x {cores} spawn processes)"},
            "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ secondary workloads
def _timed(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def extra_modes(pkg, proc, M, A, RH, RC, nevt, stream):
    """ggttgg at 2^20 events with the float32 SIMT and tensor-core (tcgen05 tf32, bf16x3) colour sums,
    and the float32 path (amplitudes and colour sum)."""
    out = {}
    for name in ("mixed_fp32", "mixed_tf32", "mixed_bf16x3", "float"):
        mode = pkg.MODES[name]
        ms = _timed(lambda: proc.compute(M, A, RH, RC, mode=mode, stream=stream), 3, 1, stream)
        out[name] = {"value": nevt / (ms * 1e-3), "unit": "events/s", "ms_per_step": ms}
    return out


def extra_ggttggg(pkg, dev, stream):
    """g g > t t~ g g g, 2^18 events: float64, mixed float32 colour sum, the two tensor-core colour
    sums (tcgen05 tf32 and bf16x3, fused into the amplitude kernel) and the float32 path, 3 timed
    steps after 1 warm-up each."""
    import numpy as np
    import torch
    from phasespace import WORKLOADS, make_inputs
    wl = WORKLOADS["ggttggg"]
    mom, a, rh, rc = make_inputs(wl, wl.nevt)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    M, A, RH, RC = t(mom), t(a), t(rh), t(rc)
    proc = pkg.Process(wl.process, device=dev.index)
    out = {"nevt": wl.nevt, "ndiagrams": proc.ndiagrams, "ncol": proc.ncol, "ngood": proc.ngood}
    for name in ("fp64", "mixed_fp32", "mixed_tf32", "mixed_bf16x3", "float"):
        mode = pkg.MODES[name]
        ms = _timed(lambda: proc.compute(M, A, RH, RC, mode=mode, stream=stream), 3, 1, stream)
        out[name] = {"value": wl.nevt / (ms * 1e-3), "unit": "events/s", "ms_per_step": ms,
                     "fp64_flops_per_event": proc.fp64_flops_per_event(mode)}
        if name == "fp64":
            # FP64 roofline of the thread kernel, and its DRAM traffic where a capture on these sources exists
            out[name]["frac_fp64_peak"] = out[name]["value"] * proc.fp64_flops_per_event(mode) / 1e12 / FP64_PEAK_TFLOPS
            per_evt = _traffic_per_event("me_kernel", "ggttggg")
            out[name]["traffic_per_launch"] = None if per_evt is None else per_evt * wl.nevt
    return out


def extra_small_batches(pkg, dev, stream):
    """Batches too small to fill the thread-per-event grid (the paper's O(1000)-event madevent
    jobs): ms per launch of the whole-event thread kernel, the block-per-event kernel (where the
    process has one), the helicity-parallel and diagram-split kernels and AUTO's choice, FP64."""
    import numpy as np
    import torch
    from phasespace import WORKLOADS, make_inputs
    kernels = (("thread", 1), ("cta", 2), ("helicity", 4), ("split", 5), ("auto", 0))
    out = []
    for name, sizes in (("ggttgg", (2048, 16384)), ("ggttggg", (512, 4096))):
        wl = WORKLOADS[name]
        mom, a, rh, rc = make_inputs(wl, max(sizes))
        t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
        M, A, RH, RC = t(mom), t(a), t(rh), t(rc)
        proc = pkg.Process(wl.process, device=dev.index)
        for n in sizes:
            row = {"process": name, "nevt": n, "ms": {}}
            for kname, k in kernels:
                try:
                    proc.set_kernel(k)
                except pkg.MgxError:
                    continue
                row["ms"][kname] = _timed(lambda: proc.compute(M[:n], A[:n], RH[:n], RC[:n], stream=stream),
                                          2 if name == "ggttgg" else 1, 1, stream)
            proc.set_kernel(0)
            row["auto_launches"] = proc.kernel_launches(n)
            out.append(row)
    return {"rows": out}


def extra_eemumu(pkg, dev, stream):
    """e+ e- > mu+ mu-, 8192 events: a small batch.  Microseconds per launch, launched directly and
    replayed from a CUDA graph of 20 launches; the HBM bandwidth that the algorithmic bytes
    (momenta, alpha_s, two random numbers in; me and two selections out) imply, and the FP64 pipe
    fraction that the batch's float64 instructions imply."""
    import numpy as np
    import torch
    from phasespace import WORKLOADS, make_inputs
    wl = WORKLOADS["eemumu"]
    mom, a, rh, rc = make_inputs(wl, wl.nevt)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    M, A, RH, RC = t(mom), t(a), t(rh), t(rc)
    proc = pkg.Process(wl.process, device=dev.index)
    n = wl.nevt
    out = {"me": torch.empty(n, dtype=torch.float64, device=dev),
           "selhel": torch.empty(n, dtype=torch.int32, device=dev),
           "selcol": torch.empty(n, dtype=torch.int32, device=dev)}
    side = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        step = lambda: proc.compute(M, A, RH, RC, stream=side, out=out)
        direct_ms = _timed(step, 200, 10, side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            for _ in range(20):
                step()
        graph_ms = _timed(g.replay, 20, 2, side) / 20
    algo = n * (4 * 4 * 8 + 3 * 8 + 8 + 4 + 4)
    inst = proc.fp64_ops_per_event(0) * n
    return {"nevt": n, "ngood": proc.ngood, "workspace_in_shared_memory": proc.workspace_bytes(n) == 0,
            "fp64_inst_per_event": inst / n, "fp64_pipe_frac_graph": inst / (graph_ms * 1e-3) / (FP64_PEAK_GINST * 1e9),
            "direct_us_per_launch": direct_ms * 1e3, "graph_us_per_launch": graph_ms * 1e3,
            "events_per_s_direct": n / (direct_ms * 1e-3), "events_per_s_graph": n / (graph_ms * 1e-3),
            "algorithmic_bytes_per_launch": algo, "hbm_gbs_graph": algo / (graph_ms * 1e-3) / 1e9}


def extra_phase_space(pkg, dev):
    """Device random numbers and flat phase space for the g g > t t~ g g final state at
    sqrt(s) = 1500 GeV: 2^26 Philox-4x32-10 uniforms (512 MiB, more than L2) and 2^22 RAMBO events
    (massive Newton rescaling), in units/s and the HBM bandwidth their algorithmic bytes imply
    (8 B per uniform out; 192 B of momenta and an 8 B weight per event out), beside the host
    generator (numpy, one process) that makes the bench's inputs."""
    import torch
    from phasespace import WORKLOADS
    from phasespace.rambo import rambo as host_rambo
    wl = WORKLOADS["ggttgg"]
    n = 1 << 22
    masses = wl.final_masses()
    L = pkg.lib()
    m = torch.tensor(masses, dtype=torch.float64, device=dev)
    mom = torch.empty((n, len(masses) + 2, 4), dtype=torch.float64, device=dev)
    wt = torch.empty(n, dtype=torch.float64, device=dev)
    nu = 1 << 26
    u = torch.empty(nu, dtype=torch.float64, device=dev)
    side = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        st = pkg._stream(dev)

        def uni():
            pkg._check(L.mgx_uniforms(nu, 0, 7, 1, pkg._ptr(u), st), "mgx_uniforms")

        def ram():
            pkg._check(L.mgx_rambo(n, 0, wl.sqrts, len(masses), pkg._ptr(m), 7, pkg._ptr(mom), pkg._ptr(wt), st),
                       "mgx_rambo")
        uni_ms = _timed(uni, 20, 3, side)
        ram_ms = _timed(ram, 10, 3, side)
    nh = 1 << 16
    t0 = time.perf_counter()
    host_rambo(nh, wl.sqrts, masses, 7)
    host_s = time.perf_counter() - t0
    rbytes = n * ((len(masses) + 2) * 32 + 8)
    return {"nevt": n, "final_masses": masses,
            "uniforms_per_s": nu / (uni_ms * 1e-3), "uniforms_hbm_gbs": 8 * nu / (uni_ms * 1e-3) / 1e9,
            "rambo_events_per_s": n / (ram_ms * 1e-3), "rambo_hbm_gbs": rbytes / (ram_ms * 1e-3) / 1e9,
            "rambo_ms": ram_ms, "host_rambo_events_per_s": nh / host_s, "host_sample": f"{nh} events, one process"}


def extra_batched(pkg, dev, stream):
    """g g > t t~ (2^22), t t~ g (2^20), t t~ g g (2^18), g u~ > ta+ ta- g g u~ (2^16): one
    autotuned persistent launch captured in a CUDA graph vs one launch per process."""
    import numpy as np
    import torch
    from phasespace import WORKLOADS, make_inputs
    sets = [("ggtt", 1 << 22), ("ggttg", 1 << 20), ("ggttgg", 1 << 18), ("gu_tataggu", 1 << 16)]
    procs, inputs, outs = [], [], []
    for name, n in sets:
        wl = WORKLOADS[name]
        mom, a, rh, rc = make_inputs(wl, n)
        t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
        inputs.append((t(mom), t(a), t(rh), t(rc)))
        procs.append(pkg.Process(wl.process, device=dev.index))
        outs.append({"me": torch.empty(n, dtype=torch.float64, device=dev),
                     "selhel": torch.empty(n, dtype=torch.int32, device=dev),
                     "selcol": torch.empty(n, dtype=torch.int32, device=dev)})
    total = sum(n for _, n in sets)

    def seq():
        for p, inp, o in zip(procs, inputs, outs):
            p.compute(*inp, stream=stream, out=o)
    ms_seq = _timed(seq, 2, 1, stream)
    b = pkg.Batch(procs)
    bps, epi = b.autotune(inputs, outs)
    side = torch.cuda.Stream(device=dev)           # graphs are captured on a non-default stream
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        b.capture(inputs, outs, side)
        ms_b = _timed(lambda: b.replay(side), 3, 1, side)
    return {"events": total, "batched_graph": {"value": total / (ms_b * 1e-3), "unit": "events/s", "ms": ms_b,
                                               "blocks_per_sm": bps, "events_per_item": dict(zip(
                                                   [name for name, _ in sets], epi))},
            "sequential": {"value": total / (ms_seq * 1e-3), "unit": "events/s", "ms": ms_seq}}


def extra_surrogate(pkg, dev):
    """g g > t t~ g g with cuts: surrogate training, then unweighted events/s plain vs two-stage.
    The two-stage leg takes stage-1 batches of 2^25 events so that the exact |M|^2 of the survivors
    (about 2^18 per batch) runs at a size that fills the GPU; its time is split by phase (CUDA
    events on the stream) and summed over the batches."""
    import torch
    from paper_2503_21935_gb300.surrogate import Unweighter
    U = Unweighter("g g > t t~ g g", 1500.0, [173.0, 173.0, 0.0, 0.0], cut_particles=[4, 5], device=dev.index,
                   seed=5)
    # 32000 steps of 16384: in a measured sweep the exact |M|^2 calls per unweighted event fell from
    # 2.64 (4000 x 8192) to 1.50 (16000 x 16384) and 1.24 (32000 x 16384, 16.5 s of training on the
    # 2^22 events); 64000 steps gave 1.16 for twice the training time
    steps, batch = 32000, 16384
    t0 = time.perf_counter()
    hist = U.train(1 << 22, steps=steps, batch=batch, lr=3e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    U.calibrate(1 << 20)
    torch.cuda.synchronize()
    calib_s = time.perf_counter() - t0
    res = {"training": {"events": 1 << 22, "steps": steps, "batch": batch, "seconds": train_s,
                        "calibration_seconds": calib_s, "loss_first": hist[0][1], "loss_last": hist[-1][1]}}
    # the two-stage leg runs until 10^6 unweighted events; the plain leg (about 8x slower per
    # unweighted event) is timed over a fixed 4 batches of 2^22, its rate being what is compared
    legs = (("plain", lambda b, prof: U.plain(1 << 22, seed=901, first=b << 22), None, 4),
            ("surrogate", lambda b, prof: U.two_stage(1 << 25, seed=901, first=b << 25, profile=prof), 1000000, None))
    for name, fn, target, nbatch in legs:
        fn(1 << 10, False)                         # warm-up (batch index far from the timed ones)
        torch.cuda.synchronize()
        n_unw = gen = calls = 0
        b = 0
        phases = {}
        batch_s = []
        weights = []                                 # for the overweight count after the timed region
        t0 = time.perf_counter()
        while (target is not None and n_unw < target) or (nbatch is not None and b < nbatch):
            tb = time.perf_counter()
            r = None                                 # the previous batch's buffers go back first
            r = fn(b, name == "surrogate")
            n_unw += int(r["weight"].shape[0])
            gen += r["generated"]
            calls += r["exact_calls"]
            weights.append(r["weight"])
            if name == "surrogate" and U.timing:
                for k, v in U.timing.items():
                    phases[k] = phases.get(k, 0.0) + v
            b += 1
            batch_s.append(time.perf_counter() - tb)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        over = sum(int((w > 1).sum().item()) for w in weights)
        res[name] = {"value": n_unw / dt, "unit": "unweighted events/s", "generated": gen,
                     "unweighted": n_unw, "exact_me_calls": calls, "seconds": dt, "batches": b,
                     "overweight_fraction": over / n_unw if n_unw else None,
                     "batch_seconds": [round(x, 4) for x in batch_s]}
        if phases:
            res[name]["phase_ms"] = phases
            res[name]["phase_ms_sum"] = sum(phases.values())
    res["gain"] = res["surrogate"]["value"] / res["plain"]["value"] if res["plain"]["value"] else None
    # the same 10^6 unweighted events with the one-off training and calibration counted in
    sur = res["surrogate"]
    sur["value_including_training"] = sur["unweighted"] / (sur["seconds"] + train_s + calib_s)
    return res


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import numpy as np
    import torch
    rank, world, local = _dist()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    import paper_2503_21935_gb300 as pkg
    from phasespace import WORKLOADS, make_inputs

    def barrier():
        if dist is not None:
            dist.barrier()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:     # the oracle baseline at N = 1 only
        cores = _host_cores()
        per_core = 8 * ORACLE_CHUNK        # about 10 s of oracle work per host process
        rate, n, busy, wall = cpu_oracle_rate(args.workload, per_core, cores)
        r1, n1, busy1, _ = cpu_oracle_rate(args.workload, per_core, 1)
        cpu = {"value": rate, "unit": "events/s", "cores": cores, "kind": "oracle",
               "sample": f"{n} events of the same workload ({per_core} per single-threaded spawn process), "
                         f"{busy:.1f} s busy",
               "single_thread": {"value": r1, "unit": "events/s", "cores": 1,
                                 "sample": f"{n1} events in one single-threaded process, {busy1:.1f} s"}}

    from paper_2503_21935_gb300.dist import event_range, max_over_ranks
    wl = WORKLOADS[args.workload]
    nevt = args.nevt
    mode = pkg.MODES[args.mode]
    first, _ = event_range(rank, world, nevt)
    mom, a, rh, rc = make_inputs(wl, nevt, first=first)          # each rank its own events
    dev = torch.device(f"cuda:{local}")
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    M, A, RH, RC = t(mom), t(a), t(rh), t(rc)
    proc = pkg.Process(wl.process, device=local)
    if args.kernel != "auto":
        proc.set_kernel(KERNELS[args.kernel])
    default_case = args.workload == WORKLOAD and nevt == NEVT and args.kernel == "auto"
    out = {"me": torch.empty(nevt, dtype=torch.float64, device=dev),
           "selhel": torch.empty(nevt, dtype=torch.int32, device=dev),
           "selcol": torch.empty(nevt, dtype=torch.int32, device=dev)}
    stream = torch.cuda.current_stream(dev)

    def step():
        proc.compute(M, A, RH, RC, mode=mode, stream=stream, out=out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for e0, e1 in evs:
            e0.record(stream)
            step()
            e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        wall = time.perf_counter() - t0
    launch_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    total_ms = max_over_ranks(sum(launch_ms), device=dev)
    ms_per_step = total_ms / args.steps
    value = world * nevt / (ms_per_step * 1e-3)

    # end to end through the host-buffer entry point: pinned inputs in, results out, every step
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    hM, hA, hRH, hRC = pin(mom), pin(a), pin(rh), pin(rc)
    hme = torch.empty(nevt, dtype=torch.float64).pin_memory()
    hsh = torch.empty(nevt, dtype=torch.int32).pin_memory()
    hsc = torch.empty(nevt, dtype=torch.int32).pin_memory()
    proc.compute_host(hM, hA, hRH, hRC, hme, hsh, hsc, mode=mode, stream=stream)
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        proc.compute_host(hM, hA, hRH, hRC, hme, hsh, hsc, mode=mode, stream=stream)
    barrier()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, device=dev)
    h2d = sum(x.numel() * x.element_size() for x in (hM, hA, hRH, hRC))
    d2h = sum(x.numel() * x.element_size() for x in (hme, hsh, hsc))

    if rank == 0:
        f32 = args.mode == "float"                              # same arithmetic on the float32 pipe
        flops = proc.fp64_flops_per_event(0 if f32 else mode) * nevt   # algorithmic flops per launch
        insts = proc.fp64_ops_per_event(0 if f32 else mode) * nevt     # instructions per launch
        launch_s = statistics.mean(launch_ms) * 1e-3
        achieved = flops / launch_s / 1e12
        peak = FP32_PEAK_TFLOPS if f32 else FP64_PEAK_TFLOPS
        peak_inst = FP32_PEAK_GINST if f32 else FP64_PEAK_GINST
        per_evt = _traffic_per_event("me_kernel_float" if f32 else "me_kernel", args.workload) \
            if args.mode in ("fp64", "float") and args.kernel in ("auto", "thread") else None
        line = {"metric": METRICS[args.workload].replace("FP64", {"fp64": "FP64", "mixed_fp32": "mixed FP32 colour sum",
                                                   "mixed_tf32": "tcgen05 TF32 colour sum",
                                                   "mixed_bf16x3": "tcgen05 BF16x3 colour sum",
                                                   "float": "FP32"}[args.mode]),
                "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "mixed_fp32": "f64+f32", "mixed_tf32": "f64+tf32", "mixed_bf16x3": "f64+bf16",
                          "float": "f32"}[args.mode], "data": "synthetic",
                # the reference arm prints the same config for the same arguments
                "config": dict(_workload_config(nevt, args.mode, args.workload,
                                                None if default_case else proc.workspace_bytes(nevt, mode)),
                               **({} if args.kernel == "auto" else {"kernel": args.kernel})),
                "process": {"ngood": proc.ngood, "ndiagrams": proc.ndiagrams, "ncol": proc.ncol},
                "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak,
                             "traffic": None if per_evt is None else per_evt * nevt,
                             "kernel": "me_kernel",
                             "peak_source": ("FP32 pipe: 152 SM x 128 FFMA/clk x 2070 MHz (all-fma peak)" if f32 else
                                             "FP64 pipe: 152 SM x 2 DFMA/clk x 2070 MHz (all-fma peak)"),
                             "inst_per_s": insts / launch_s,
                             "pipe_frac": insts / launch_s / 1e9 / peak_inst,
                             "flops_per_event": flops / nevt},
                "e2e": {"value": world * nevt / e2e_s, "unit": "events/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": args.steps * proc.kernel_launches(nevt, mode),
                "clocks": clk.summary(),
                "cpu_baseline": cpu,
                "wall_s_timed": wall}
        if not args.no_extras and world == 1 and default_case:
            extras = {}
            for key, fn in (("ggttgg_modes", lambda: extra_modes(pkg, proc, M, A, RH, RC, nevt, stream)),
                            ("ggttggg", lambda: extra_ggttggg(pkg, dev, stream)),
                            ("small_batches", lambda: extra_small_batches(pkg, dev, stream)),
                            ("eemumu", lambda: extra_eemumu(pkg, dev, stream)),
                            ("batched", lambda: extra_batched(pkg, dev, stream)),
                            ("surrogate_unweighting", lambda: extra_surrogate(pkg, dev)),
                            ("phase_space", lambda: extra_phase_space(pkg, dev))):
                # each workload starts from an empty allocator cache (the previous ones' workspaces,
                # up to 81 GB for g g > t t~ g g g, would otherwise stay reserved)
                gc.collect()
                torch.cuda.empty_cache()
                t0 = time.perf_counter()
                try:
                    extras[key] = fn()
                except Exception as exc:          # a secondary workload must not hide the headline
                    extras[key] = {"error": f"{type(exc).__name__}: {exc}"}
                extras[key]["wall_s"] = time.perf_counter() - t0
            line["extras"] = extras
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
