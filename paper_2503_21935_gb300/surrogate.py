"""Surrogate-driven two-stage unweighting on the GPU (orchestration of library kernels).

A small MLP learns log|M|^2 over phase space from events the exact path evaluates; it then
drives stage 1 of a two-stage unweighting whose stage 2 corrects every surviving event with
its exact |M|^2 (Danziger, Janssen, Schumann, Siegert, arXiv:2109.11964), so the unweighted
sample stays unbiased and the exact |M|^2 has the last word.  Every arithmetic step of the
method runs in the library's kernels (phase space, cuts, matrix elements, network, weights,
accept/reject, compaction); this module sequences the calls and holds device buffers (PyTorch
tensors).

Stage 1 runs on float32 proposals: RAMBO and the cuts (thresholds widened by a small margin, so that
every event the exact cuts accept is proposed) in single precision, the surrogate weight from those
momenta.  Only the stage-1 survivors are regenerated in float64 (the same random numbers, by event
index) for the exact cuts, phase-space weight and |M|^2 of stage 2.  The proposal weight s only has
to be positive wherever the exact weight is, so the unweighted sample stays unbiased.

Data parallelism (one replica per GPU, `dist`): each rank generates and unweights its own
contiguous range of events.  Every random number of the accept/reject steps is keyed by the
event's global index, and the maxima come from the weights of all ranks' calibration events,
so the union of the ranks' unweighted events is exactly the sample one rank would draw from
all the events.  Training is data-parallel too: each rank's gradient comes from its own
training events, the ranks average the gradients (one all-reduce per step) and apply the same
Adam step.
"""
import ctypes

import numpy as np

from . import (Mlp, MgxError, Process, _check, _ptr, _stream, lib, rambo, rambo_f32, rambo_indexed, cuts, cuts_f32,
               uniforms, MGX_FP64, MGX_MOMENTS_LEN)
from . import dist as _dist

# relative widening of the cut thresholds applied to the float32 proposals: far above float32
# rounding of the cut observables (about 1e-6 relative in pT, 1e-3 absolute in eta near |eta| = 5),
# so the proposals' accepted region contains the exact one
PROPOSAL_CUT_MARGIN = 1e-2


class Unweighter:
    """Plain and surrogate two-stage unweighting for one process with generator cuts.

    cut_particles: indices of the final-state particles (in the momentum array) on which
    pT > ptmin, |eta| < etamax and pairwise dR > drmin are required.
    """

    def __init__(self, process, sqrts, final_masses, cut_particles=(), ptmin=20.0, etamax=5.0, drmin=0.4,
                 device=0, mode=MGX_FP64, seed=1):
        import torch
        self.dev = torch.device(f"cuda:{device}")
        self.proc = process if isinstance(process, Process) else Process(process, device=device)
        self.sqrts = float(sqrts)
        self.masses = list(final_masses)
        self.npar = len(self.masses) + 2
        self.cut = (list(cut_particles), ptmin, etamax, drmin)
        self.mode = mode
        self.net = Mlp(seed=seed, device=device)
        self.mean = 0.0
        self.sd = 1.0
        self.exact_calls = 0
        self.timing = None          # per-phase CUDA-event times of the last profiled call

    # ------------------------------------------------------------------ events
    def events(self, n, seed, first=0):
        """Device momenta, phase-space weights and cut mask of events first .. first+n-1."""
        mom, wps = rambo(n, self.sqrts, self.masses, seed, first=first, device=self.dev.index)
        lst, ptmin, etamax, drmin = self.cut
        if lst:
            ok = cuts(mom, lst, ptmin, etamax, drmin)
        else:
            import torch
            ok = torch.ones(n, dtype=torch.uint8, device=self.dev)
        return mom, wps, ok

    def exact_me(self, mom, alpha_s=0.118):
        import torch
        n = mom.shape[0]
        a = torch.full((n,), alpha_s, dtype=torch.float64, device=self.dev)
        self.exact_calls += n
        return self.proc.compute(mom, a, mode=self.mode)["me"]

    def features(self, mom):
        import torch
        n = mom.shape[0]
        ncomp = 4 * self.npar
        if ncomp != 24:
            raise MgxError("the surrogate network takes 24 momentum components (6 particles)")
        x = torch.empty((n, ncomp), dtype=torch.float32, device=self.dev)
        _check(lib().mgx_features(n, ncomp, _ptr(mom), 0.5 * self.sqrts, _ptr(x), _stream(self.dev)), "mgx_features")
        return x

    def _compact(self, keep):
        import torch
        n = keep.shape[0]
        b = ctypes.c_size_t()
        _check(lib().mgx_compact_workspace_bytes(n, ctypes.byref(b)), "mgx_compact_workspace_bytes")
        ws = torch.empty(max(b.value, 256), dtype=torch.uint8, device=self.dev)
        idx = torch.empty(max(n, 1), dtype=torch.int32, device=self.dev)
        cnt = torch.zeros(1, dtype=torch.int32, device=self.dev)
        _check(lib().mgx_compact(n, _ptr(keep), _ptr(idx), _ptr(cnt), _ptr(ws), ws.numel(), _stream(self.dev)),
               "mgx_compact")
        return idx[: int(cnt.item())]

    def _gather(self, idx, src):
        import torch
        m = idx.shape[0]
        row = int(np.prod(src.shape[1:])) if src.dim() > 1 else 1
        dst = torch.empty((m,) + tuple(src.shape[1:]), dtype=torch.float64, device=self.dev)
        _check(lib().mgx_gather(m, _ptr(idx), row, _ptr(src), _ptr(dst), _stream(self.dev)), "mgx_gather")
        return dst

    def _accept(self, w, wref, wmax, r):
        import torch
        n = w.shape[0]
        keep = torch.empty(n, dtype=torch.uint8, device=self.dev)
        over = torch.empty(n, dtype=torch.float64, device=self.dev)
        _check(lib().mgx_accept(n, _ptr(w), _ptr(wref), float(wmax), _ptr(r), _ptr(keep), _ptr(over),
                                _stream(self.dev)), "mgx_accept")
        return keep, over

    def _weights(self, me, wps, ok):
        import torch
        n = me.shape[0]
        w = torch.empty(n, dtype=torch.float64, device=self.dev)
        _check(lib().mgx_exact_weight(n, _ptr(me), _ptr(wps), _ptr(ok), _ptr(w), _stream(self.dev)),
               "mgx_exact_weight")
        return w

    def proposals(self, n, seed, first=0):
        """Float32 momenta, phase-space weights and widened-cut mask of events first .. first+n-1."""
        mom, wps = rambo_f32(n, self.sqrts, self.masses, seed, first=first, device=self.dev.index)
        lst, ptmin, etamax, drmin = self.cut
        if lst:
            ok = cuts_f32(mom, lst, ptmin, etamax, drmin, PROPOSAL_CUT_MARGIN)
        else:
            import torch
            ok = torch.ones(n, dtype=torch.uint8, device=self.dev)
        return mom, wps, ok

    def surrogate_weights(self, mom, wps, ok):
        """s = exp(mean + sd y) wps pass, y the network on the momenta (float64, or float32 proposals)."""
        import torch
        n = mom.shape[0]
        if 4 * self.npar != 24:
            raise MgxError("the surrogate network takes 24 momentum components (6 particles)")
        y = self.net.forward_momenta(mom, 0.5 * self.sqrts)
        s = torch.empty(n, dtype=torch.float64, device=self.dev)
        f = lib().mgx_surrogate_weight_f32 if wps.dtype == torch.float32 else lib().mgx_surrogate_weight
        _check(f(n, _ptr(y), self.mean, self.sd, _ptr(wps), _ptr(ok), _ptr(s), _stream(self.dev)),
               "mgx_surrogate_weight")
        return s

    # ------------------------------------------------------------------ training
    def train(self, ntrain, steps, batch=4096, lr=1e-3, seed=101, lr_decay=0.1):
        """Generate ntrain events (per rank), evaluate them exactly, fit log|M|^2 of those passing
        the cuts.  With several ranks: each rank trains on its own events and the ranks average
        their gradients every step (data-parallel replicas, identical parameters throughout)."""
        import torch
        rank, world = _dist.rank_world()
        mom, wps, ok = self.events(ntrain, seed, first=rank * ntrain)
        me = self.exact_me(mom)
        n0 = me.shape[0]
        logme = torch.empty(n0, dtype=torch.float64, device=self.dev)
        keep = torch.empty(n0, dtype=torch.uint8, device=self.dev)
        _check(lib().mgx_log_targets(n0, _ptr(me), _ptr(ok), _ptr(logme), _ptr(keep), _stream(self.dev)),
               "mgx_log_targets")
        idx = self._compact(keep)
        x = self.features(self._gather(idx, mom))
        y = self._gather(idx, logme)
        n = y.shape[0]
        # standardisation from the moments of all ranks' targets (rank-order sums)
        s1, s2, _ = self._moments(y)
        s1, s2, cnt = _dist.allreduce_sums([s1, s2, n], device=self.dev)
        self.mean = s1 / cnt
        self.sd = float(np.sqrt(max(s2 / cnt - self.mean ** 2, 0.0) * cnt / max(cnt - 1, 1)))
        t = torch.empty(n, dtype=torch.float32, device=self.dev)
        _check(lib().mgx_standardize_f32(n, _ptr(y), self.mean, self.sd, _ptr(t), _stream(self.dev)),
               "mgx_standardize_f32")
        # every step's batch is drawn by the library from the replica's own training set
        key = seed + 7919 * rank
        hist = []
        loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        for step in range(steps):
            rate = lr * (lr_decay ** (step / max(1, steps - 1)))
            if world == 1:
                self.net.train_step_sampled(x, t, batch, key, step, lr=rate, loss_out=loss)
            else:
                grad = self.net.device_gradients_sampled(x, t, batch, key, step, loss_out=loss)
                _dist.allreduce_gradients(grad, batch)
                self.net.adam_step(grad, lr=rate)
            if step % max(1, steps // 20) == 0 or step == steps - 1:
                hist.append((step, float(loss.item())))
        return hist

    def _moments(self, v):
        """(sum, sum of squares, max) of a device float64 vector, in the library's fixed order."""
        import torch
        out = torch.empty(MGX_MOMENTS_LEN, dtype=torch.float64, device=self.dev)
        _check(lib().mgx_moments(v.shape[0], _ptr(v), _ptr(out), _stream(self.dev)), "mgx_moments")
        return tuple(out[:3].tolist())

    # ------------------------------------------------------------------ calibration
    def calibration_sample(self, n, seed, first=0):
        """Exact and surrogate weights (w, s) of events first .. first+n-1 (s as stage 1 computes it,
        from the float32 proposals)."""
        mom, wps, ok = self.events(n, seed, first)
        w = self._weights(self.exact_me(mom), wps, ok)
        s = self.surrogate_weights(*self.proposals(n, seed, first))
        return w, s

    def set_maxima(self, w, s, q=0.999):
        """Reference maxima from calibration weights: w_max (plain), s_max and r_max (two-stage), the
        q-quantiles of w, s and w/s over the events with w > 0 and s > 0 (q = 1: the maxima)."""
        out = (ctypes.c_double * 3)()
        w, s = w.contiguous(), s.contiguous()     # held until the call has copied them back
        _check(lib().mgx_unweighting_maxima(w.shape[0], _ptr(w), _ptr(s), float(q), ctypes.cast(out, ctypes.c_void_p),
                                            _stream(self.dev)), "mgx_unweighting_maxima")
        self.w_max, self.s_max, self.r_max = out[0], out[1], out[2]
        return self.w_max, self.s_max, self.r_max

    def calibrate(self, n, seed=202, q=0.999):
        """Reference maxima from n calibration events per rank; with several ranks the quantiles are
        taken over the weights of all ranks' events (one gather), the same on every rank."""
        rank, world = _dist.rank_world()
        w, s = self.calibration_sample(n, seed, first=rank * n)
        if world > 1:
            w, s = _dist.gather_samples(w), _dist.gather_samples(s)
        return self.set_maxima(w, s, q)

    # ------------------------------------------------------------------ unweighting
    def _stats(self, w):
        """Global (max w, sum w, N) of a batch: one collective across ranks."""
        sw, _, mx = self._moments(w) if w.numel() else (0.0, 0.0, 0.0)
        return _dist.allreduce_weight_stats(mx, sw, int(w.numel()), device=self.dev)

    def _unweighted(self, idx2, idx1, over1, over2, first):
        """Weights and global indices of the unweighted events (mgx_unweighted_out)."""
        import torch
        m = idx2.shape[0]
        weight = torch.empty(m, dtype=torch.float64, device=self.dev)
        index = torch.empty(m, dtype=torch.int64, device=self.dev)
        _check(lib().mgx_unweighted_out(m, _ptr(idx2), _ptr(idx1), _ptr(over1), _ptr(over2), int(first),
                                        _ptr(weight), _ptr(index), _stream(self.dev)), "mgx_unweighted_out")
        return weight, index

    def plain(self, n, seed, first=0):
        """Hit-or-miss on the exact weight of events first .. first+n-1."""
        mom, wps, ok = self.events(n, seed, first)
        calls = self.exact_calls
        w = self._weights(self.exact_me(mom), wps, ok)
        keep, over = self._accept(w, None, self.w_max, uniforms(n, seed, 11, first=first, device=self.dev.index))
        idx = self._compact(keep)
        mx, sw, nn = self._stats(w)
        weight, index = self._unweighted(idx, None, over, None, first)
        return dict(momenta=self._gather(idx, mom), weight=weight, index=index,
                    exact_calls=self.exact_calls - calls, generated=n, all_weights=w, all_momenta=mom,
                    max_w=mx, sum_w=sw, n_events=nn)

    def two_stage(self, n, seed, first=0, profile=False):
        """Stage 1 on the surrogate weight, stage 2 on exact / surrogate for the survivors only, for
        events first .. first+n-1.  Both stages draw their random numbers by global event index.
        profile=True records the time of each phase with CUDA events into self.timing (ms)."""
        import torch
        stream = torch.cuda.current_stream(self.dev)
        marks = []

        def mark(name):
            if profile:
                e = torch.cuda.Event(enable_timing=True)
                e.record(stream)
                marks.append((name, e))
        mark("start")
        mom32, wps32, ok32 = self.proposals(n, seed, first)
        mark("phase space and cuts")
        s = self.surrogate_weights(mom32, wps32, ok32)
        mark("features, network, surrogate weights")
        keep1, over1 = self._accept(s, None, self.s_max, uniforms(n, seed, 12, first=first, device=self.dev.index))
        idx1 = self._compact(keep1)
        # the survivors again in float64: exact momenta, phase-space weight and cuts
        m1, wps1 = rambo_indexed(idx1, first, self.sqrts, self.masses, seed, device=self.dev.index)
        lst, ptmin, etamax, drmin = self.cut
        ok1 = cuts(m1, lst, ptmin, etamax, drmin) if lst else None
        s1 = self._gather(idx1, s)
        r2 = self._gather(idx1, uniforms(n, seed + 7919, 13, first=first, device=self.dev.index))
        mark("stage-1 accept, compaction, float64 survivors")
        calls = self.exact_calls
        me1 = self.exact_me(m1)
        mark("exact |M|^2 of the survivors")
        w1 = self._weights(me1, wps1, ok1)
        keep2, over2 = self._accept(w1, s1, self.r_max, r2)
        idx2 = self._compact(keep2)
        weight, index = self._unweighted(idx2, idx1, over1, over2, first)
        out = dict(momenta=self._gather(idx2, m1), weight=weight, index=index,
                   exact_calls=self.exact_calls - calls, generated=n, stage1=int(idx1.shape[0]))
        mark("stage-2 accept and compaction")
        if profile:
            torch.cuda.synchronize(self.dev)
            self.timing = {name: marks[k - 1][1].elapsed_time(e) for k, (name, e) in enumerate(marks) if k > 0}
        return out
