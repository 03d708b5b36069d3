"""Surrogate-driven two-stage unweighting on the GPU (orchestration of library kernels).

A small MLP learns log|M|^2 over phase space from events the exact path evaluates; it then
drives stage 1 of a two-stage unweighting whose stage 2 corrects every surviving event with
its exact |M|^2 (Danziger, Janssen, Schumann, Siegert, arXiv:2109.11964), so the unweighted
sample stays unbiased and the exact |M|^2 has the last word.  Every arithmetic step runs in the
library's kernels (phase space, cuts, matrix elements, network, weights, accept/reject,
compaction); this module sequences the calls and holds device buffers (PyTorch tensors).
"""
import ctypes
import time

import numpy as np

from . import (Mlp, MgxError, Process, _check, _ptr, _stream, lib, rambo, cuts, uniforms, MGX_FP64)


def _dev_empty(n, dtype, device):
    import torch
    return torch.empty(n, dtype=dtype, device=device)


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

    # ------------------------------------------------------------------ events
    def events(self, n, seed, first=0):
        """Device momenta, phase-space weights and cut mask of n events."""
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

    def _accept(self, w, wref, wmax, seed, stream_id):
        import torch
        n = w.shape[0]
        r = uniforms(n, seed, stream_id, device=self.dev.index)
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

    def surrogate_weights(self, mom, wps, ok):
        import torch
        n = mom.shape[0]
        y = self.net.forward(self.features(mom))
        s = torch.empty(n, dtype=torch.float64, device=self.dev)
        _check(lib().mgx_surrogate_weight(n, _ptr(y), self.mean, self.sd, _ptr(wps), _ptr(ok), _ptr(s),
                                          _stream(self.dev)), "mgx_surrogate_weight")
        return s

    # ------------------------------------------------------------------ training
    def train(self, ntrain, steps, batch=4096, lr=1e-3, seed=101, lr_decay=0.1):
        """Generate ntrain events, evaluate them exactly, fit log|M|^2 of those passing the cuts."""
        import torch
        mom, wps, ok = self.events(ntrain, seed)
        me = self.exact_me(mom)
        keep = ok.bool() & (me > 0)
        x = self.features(mom)[keep].contiguous()
        y = torch.log(me[keep])
        self.mean = float(y.mean().item())
        self.sd = float(y.std().item())
        t = ((y - self.mean) / self.sd).to(torch.float32).contiguous()
        n = x.shape[0]
        g = torch.Generator(device=self.dev)
        g.manual_seed(seed)
        hist = []
        loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        for step in range(steps):
            idx = torch.randint(0, n, (batch,), device=self.dev, generator=g)
            frac = step / max(1, steps - 1)
            rate = lr * (lr_decay ** frac)
            self.net.train_step(x[idx].contiguous(), t[idx].contiguous(), lr=rate, loss_out=loss)
            if step % max(1, steps // 20) == 0 or step == steps - 1:
                hist.append((step, float(loss.item())))
        return hist

    # ------------------------------------------------------------------ calibration
    def calibrate(self, n, seed=202, q=0.999):
        """Reference maxima (high quantiles): w_max (plain), s_max and r_max (two-stage)."""
        mom, wps, ok = self.events(n, seed)
        w = self._weights(self.exact_me(mom), wps, ok)
        s = self.surrogate_weights(mom, wps, ok)
        sel = (w > 0) & (s > 0)
        self.w_max = float(w[sel].quantile(q).item()) if sel.sum() < 2 ** 24 else float(w[sel].max().item())
        self.s_max = float(s[sel].quantile(q).item())
        self.r_max = float((w[sel] / s[sel]).quantile(q).item())
        return self.w_max, self.s_max, self.r_max

    # ------------------------------------------------------------------ unweighting
    def plain(self, n, seed, first=0):
        """Hit-or-miss on the exact weight of every event."""
        import torch
        mom, wps, ok = self.events(n, seed, first)
        calls = self.exact_calls
        w = self._weights(self.exact_me(mom), wps, ok)
        keep, over = self._accept(w, None, self.w_max, seed, 11)
        idx = self._compact(keep)
        return dict(momenta=self._gather(idx, mom), weight=over[idx.long()], exact_calls=self.exact_calls - calls,
                    generated=n, all_weights=w, all_momenta=mom)

    def two_stage(self, n, seed, first=0):
        """Stage 1 on the surrogate weight, stage 2 on exact / surrogate for the survivors only."""
        import torch
        mom, wps, ok = self.events(n, seed, first)
        s = self.surrogate_weights(mom, wps, ok)
        keep1, over1 = self._accept(s, None, self.s_max, seed, 12)
        idx1 = self._compact(keep1)
        m1 = self._gather(idx1, mom)
        calls = self.exact_calls
        me1 = self.exact_me(m1)
        w1 = self._weights(me1, self._gather(idx1, wps), None)
        s1 = self._gather(idx1, s)
        keep2, over2 = self._accept(w1, s1, self.r_max, seed + 7919, 13)
        idx2 = self._compact(keep2)
        weight = over1[idx1.long()][idx2.long()] * over2[idx2.long()]
        return dict(momenta=self._gather(idx2, m1), weight=weight, exact_calls=self.exact_calls - calls,
                    generated=n, stage1=int(idx1.shape[0]))
