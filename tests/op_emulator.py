"""Float64 numpy interpreter of the process compiler's op tables (test infrastructure).

It executes a compiled program (`gen.program.build_program`) with the op semantics the library's
kernels implement: the flat per-event workspace with the compiler's block offsets, op headers
(momenta, propagator prefactors, slash blocks, VVV and VVVV child tables), one current per
helicity state of its own legs (variants addressed by pdep / pext of the leg masks), sum
currents, amplitude groups and runs closed at the root bilinears, colour flows with phases and
first writes, and the colour quadratic form.  All variants of an op, and all helicities of an
amplitude group, are evaluated at once over numpy arrays of events.

It lets the CPU tests check the compiler's output against the oracle without a GPU: a wrong
offset, mask, phase, flow or schedule shows up as a wrong |M|^2 (the workspace starts as NaN, so
a read before the write also shows).  It shares no code with the oracle; physics conventions
(HELAS helicity spinors and polarisation vectors, Feynman rules with all momenta incoming) are
restated here from their definitions.
"""
import math
from collections import Counter

import numpy as np

from paper_2503_21935_gb300.gen import sm
from paper_2503_21935_gb300.gen.program import (
    EXT_EPS_IN, EXT_EPS_OUT, EXT_U, EXT_UBAR, EXT_V, EXT_VBAR, FLOW_FIRST, HEADER, OP_AMP, OP_BIL, OP_EXT,
    OP_FFV_F, OP_FFV_FB, OP_FFV_V, OP_RBIL, OP_SUM, OP_VVV, OP_VVVV, build_program)

# Standard Model inputs (fixed-width propagators; EW scheme {alpha(mZ), G_F, mZ})
PARAMS = {"": 0.0, "mt": 173.0, "wt": 1.4915, "mz": 91.1876, "wz": 2.4414, "mta": 1.777}
ALPHA_EM, G_F = 1.0 / 132.507, 1.16639e-5
METRIC = np.array([1.0, -1.0, -1.0, -1.0])
PHASE = np.array([1.0, 1j, -1.0, -1j])
NAME = {OP_FFV_F: "ffv_f", OP_FFV_FB: "ffv_fb", OP_FFV_V: "ffv_v", OP_VVV: "vvv", OP_VVVV: "vvvv", OP_BIL: "bil",
        OP_RBIL: "rbil"}


def pext(x, mask):
    """Bits of x at the set bits of mask, packed to the low end."""
    r, k = 0, 0
    while mask:
        low = mask & -mask
        if x & low:
            r |= 1 << k
        k += 1
        mask ^= low
    return r


def pdep(v, mask):
    """Low bits of v scattered to the set bits of mask."""
    r, k = 0, 0
    while mask:
        low = mask & -mask
        if (v >> k) & 1:
            r |= low
        k += 1
        mask ^= low
    return r


def nvar(mask):
    return 1 << bin(mask).count("1")


def couplings(P):
    """(cL, cR, chiral) per coupling entry: i g_s (g_s factored out), -i e Q, -i (gL, gR)."""
    e = math.sqrt(4 * math.pi * ALPHA_EM)
    mz2 = PARAMS["mz"] ** 2
    mw2 = 0.5 * mz2 + math.sqrt(0.25 * mz2 * mz2 - math.pi * ALPHA_EM * mz2 / (math.sqrt(2.0) * G_F))
    sw2 = 1.0 - mw2 / mz2
    sw, cw = math.sqrt(sw2), math.sqrt(1.0 - sw2)
    out = []
    for boson, fermion in P.couplings:
        q = sm.charge(fermion) if fermion else 0.0
        t3 = sm.t3(fermion) if fermion else 0.0
        if boson == "g":
            out.append((1j, 1j, False))
        elif boson == "a":
            out.append((-1j * e * q, -1j * e * q, False))
        else:
            gl = e * (t3 - q * sw2) / (sw * cw)
            gr = -e * q * sw2 / (sw * cw)
            out.append((-1j * gl, -1j * gr, True))
    return out


# ---------------------------------------------------------------- external wavefunctions
def _chi(p, pp, lam):
    """Two-component helicity spinor chi_lam(p) ([2, nevt]); along -z and at rest by convention."""
    a = pp + p[3]
    pos = a > 0
    n = np.where(pos, 1.0 / np.sqrt(np.where(pos, 2.0 * pp * a, 1.0)), 0.0)
    pt = p[1] + 1j * p[2]
    down = ~pos & (pp > 0)
    if lam > 0:
        c0 = np.where(pos, a * n, 0.0) + 0j
        c1 = np.where(pos, pt * n, np.where(down, 1.0, 0.0))
        c0 = np.where(pos | down, c0, 1.0)
    else:
        c0 = np.where(pos, -np.conj(pt) * n, np.where(down, -1.0, 0.0))
        c1 = np.where(pos, a * n, np.where(down, 0.0, 1.0)) + 0j
    return np.array([c0, c1])


def _ext_u(p, m, lam):
    pp = np.sqrt(p[1] ** 2 + p[2] ** 2 + p[3] ** 2)
    c = _chi(p, pp, lam)
    if m == 0.0:
        s = np.sqrt(2.0 * p[0])
        wu, wl = (s, 0.0 * s) if lam < 0 else (0.0 * s, s)
    else:
        lp = pp if lam > 0 else -pp
        wu, wl = np.sqrt(np.maximum(p[0] - lp, 0.0)), np.sqrt(np.maximum(p[0] + lp, 0.0))
    return np.array([wu * c[0], wu * c[1], wl * c[0], wl * c[1]])


def _ext_v(p, m, lam):
    pp = np.sqrt(p[1] ** 2 + p[2] ** 2 + p[3] ** 2)
    c = _chi(p, pp, -lam)
    if m == 0.0:
        s = np.sqrt(2.0 * p[0])
        wu, wl = (s, 0.0 * s) if lam > 0 else (0.0 * s, -s)
    else:
        lp = pp if lam > 0 else -pp
        wu, wl = np.sqrt(np.maximum(p[0] + lp, 0.0)), -np.sqrt(np.maximum(p[0] - lp, 0.0))
    return np.array([wu * c[0], wu * c[1], wl * c[0], wl * c[1]])


def _bar(w):
    """psi-bar = psi^dagger gamma^0 in the chiral basis."""
    return np.conj(np.array([w[2], w[3], w[0], w[1]]))


def _ext_eps(k, lam, outgoing):
    """eps^mu(k, lam) = (-lam e1 - i e2)/sqrt2 in the frame of k (upper index); outgoing conjugated."""
    kk = np.sqrt(k[1] ** 2 + k[2] ** 2 + k[3] ** 2)
    pt = np.sqrt(k[1] ** 2 + k[2] ** 2)
    cth = np.where(kk > 0, k[3] / np.where(kk > 0, kk, 1.0), 1.0)
    sth = np.where(kk > 0, pt / np.where(kk > 0, kk, 1.0), 0.0)
    cph = np.where(pt > 0, k[1] / np.where(pt > 0, pt, 1.0), 1.0)
    sph = np.where(pt > 0, k[2] / np.where(pt > 0, pt, 1.0), 0.0)
    r = 1.0 / math.sqrt(2.0)
    eps = np.array([0.0 * kk + 0j, (-lam * cth * cph + 1j * sph) * r, (-lam * cth * sph - 1j * cph) * r,
                    lam * sth * r + 0j])
    return np.conj(eps) if outgoing else eps


# ---------------------------------------------------------------- workspace
class Workspace:
    """Flat float64 workspace [slot][event] with the compiler's offsets (complex = 2 slots).
    With `log` set to a (reads, writes) pair of sets, every slot accessed is recorded."""

    def __init__(self, nslots, nevt):
        self.w = np.full((nslots, nevt), np.nan)
        self.log = None

    def _note(self, which, slots):
        if self.log is not None:
            self.log[which].update(np.ravel(slots).tolist())

    def k(self, off):
        self._note(0, range(off, off + 4))
        return self.w[off:off + 4]

    def set_k(self, off, k):
        self._note(1, range(off, off + 4))
        self.w[off:off + 4] = k

    def set_r(self, off, x):
        self._note(1, [off])
        self.w[off] = x

    def cx(self, off):
        self._note(0, [off, off + 1])
        return self.w[off] + 1j * self.w[off + 1]

    def set_cx(self, off, z):
        self._note(1, [off, off + 1])
        self.w[off], self.w[off + 1] = z.real, z.imag

    def vec(self, base, idx):
        """Complex 4-vectors of variants idx (array) of the block whose variant 0 starts at base:
        [len(idx), 4, nevt]."""
        slots = base + 8 * np.asarray(idx)[:, None] + np.arange(8)[None, :]
        self._note(0, slots)
        x = self.w[slots]
        return x[:, 0::2] + 1j * x[:, 1::2]

    def set_vec(self, base, idx, v):
        slots = base + 8 * np.asarray(idx)[:, None] + np.arange(8)[None, :]
        self._note(1, slots)
        x = np.empty(slots.shape + v.shape[2:])
        x[:, 0::2], x[:, 1::2] = v.real, v.imag
        self.w[slots] = x


def _mdot(a, b):
    """Minkowski product over axis -2 of complex 4-vectors [..., 4, nevt]."""
    return np.einsum("m,...me->...e", METRIC, a * b)


def _slash(V):
    """The four distinct entries of the chiral blocks of Vslash: V0 - V3, V0 + V3, V1 - i V2, V1 + i V2."""
    return np.stack([V[:, 0] - V[:, 3], V[:, 0] + V[:, 3], V[:, 1] - 1j * V[:, 2], V[:, 1] + 1j * V[:, 2]], axis=1)


def _blocks(sl):
    """A = [[a00, a01], [a10, a11]], B likewise, from the slash entries [n, 4, nevt]."""
    s0, s1, s2, s3 = sl[:, 0], sl[:, 1], sl[:, 2], sl[:, 3]
    return (s0, -s2, -s3, s1), (s1, s2, s3, s0)


def _check_wave(logs):
    """No item of a wave may touch a slot that another item of the wave writes."""
    writer = {}
    for it, (_, writes) in logs:
        for s in writes:
            if writer.setdefault(s, it) != it:
                raise AssertionError(f"slot {s} written by items {writer[s]:#x} and {it:#x} of one wave")
    for it, (reads, _) in logs:
        for s in reads:
            if writer.get(s, it) != it:
                raise AssertionError(f"item {it:#x} reads slot {s} that item {writer[s]:#x} of its wave writes")


def _select(w, r):
    """First index whose cumulative weight exceeds r x total (canonical order), else the last."""
    c = np.cumsum(w, axis=1)
    above = c > (r * c[:, -1])[:, None]
    return np.where(above.any(axis=1), above.argmax(axis=1), w.shape[1] - 1)


class Emulator:
    def __init__(self, process):
        self.P = build_program(process)
        P = self.P
        self.cpl = couplings(P)
        self.mass = [(PARAMS[m], PARAMS[w]) for m, w in P.masses]
        self.C = np.array([[float(x) for x in row] for row in P.colour])
        self.nhel = 1 << P.npar
        self.fix, self.bits = 0, 0    # helicity-parallel group: helicity bits `bits` on the legs `fix`

    def _allowed(self, mask):
        """Variants of a current with leg mask `mask` that the current group computes (all of them
        without a group)."""
        free = mask & ~self.fix
        return [pext(pdep(u, free) | (self.bits & mask), mask) for u in range(nvar(free))]

    def evaluate_groups(self, mom, alpha_s, fix, rnd_hel=None, rnd_col=None):
        """The helicity-parallel program: for each of the 2^|fix| groups (helicity bits on the legs in
        `fix`), a fresh NaN workspace in which only the group's current variants, header tables and
        helicity amplitudes are computed; the jamps of each helicity come from its group.  A variant
        or table read that the group did not compute makes the result NaN."""
        P = self.P
        nevt = mom.shape[0]
        pe = np.transpose(mom, (1, 2, 0))
        self.terms, self.flows = P.terms, P.flows
        self.count = Counter()
        out = np.full((self.nhel, P.ncol, nevt), np.nan + 0j)
        k = bin(fix).count("1")
        for g in range(1 << k):
            self.fix, self.bits = fix, pdep(g, fix)
            W = Workspace(P.ws_current_doubles, nevt)
            jamps = np.zeros((self.nhel, P.ncol, nevt), complex) if P.jamp_zero else \
                np.full((self.nhel, P.ncol, nevt), np.nan + 0j)
            for op in P.ops:
                if op[0] == OP_AMP:
                    self._amp(op, W, jamps)
                else:
                    self._header(op, W, pe)
                    self._variants(op, W, pe)
            mine = [h for h in range(self.nhel) if h & fix == self.bits]
            out[mine] = jamps[mine]
        self.fix, self.bits = 0, 0
        return self._finish(out, alpha_s, rnd_hel, rnd_col)

    def evaluate(self, mom, alpha_s, rnd_hel=None, rnd_col=None):
        """me [nevt], per-helicity |M_h|^2 [nevt, nhel] and colour weights [nevt, ncol] for momenta
        [nevt, npar, 4] (every helicity, no filter), and the selections for the given uniforms,
        through the thread-per-event program (ops in order, one current's variants at a time)."""
        P = self.P
        nevt = mom.shape[0]
        pe = np.transpose(mom, (1, 2, 0))                     # [npar, 4, nevt]
        W = Workspace(P.ws_current_doubles, nevt)
        self.terms, self.flows = P.terms, P.flows
        self.count = Counter()      # work executed per event, in the compiler's count names
        # jamps start as NaN unless a flow is never updated: every flow's first update must write
        jamps = np.zeros((self.nhel, P.ncol, nevt), complex) if P.jamp_zero else \
            np.full((self.nhel, P.ncol, nevt), np.nan + 0j)
        for op in P.ops:
            if op[0] == OP_AMP:
                self._amp(op, W, jamps)
            else:
                self._header(op, W, pe)
                self._variants(op, W, pe)
        return self._finish(jamps, alpha_s, rnd_hel, rnd_col)

    def evaluate_parts(self, mom, alpha_s, parts, fix=0, rnd_hel=None, rnd_col=None):
        """The diagram-split program: for each part (op positions in program order) and helicity
        group (bits on the legs in `fix`), a fresh NaN workspace in which only the part's ops run,
        restricted to the group, into zeroed partial jamps that every flow update adds to; the
        partial jamps of the parts are summed.  An op that reads a block its part did not compute
        (or that another op of the part reused) makes the result NaN or wrong."""
        P = self.P
        nevt = mom.shape[0]
        pe = np.transpose(mom, (1, 2, 0))
        self.terms, self.flows = P.terms, P.flows
        self.count = Counter()
        total = np.zeros((self.nhel, P.ncol, nevt), complex)
        k = bin(fix).count("1")
        for g in range(1 << k):
            self.fix, self.bits = fix, pdep(g, fix)
            for part in parts:
                W = Workspace(P.ws_current_doubles, nevt)
                jamps = np.zeros((self.nhel, P.ncol, nevt), complex)
                for i in part:
                    op = P.ops[i]
                    if op[0] == OP_AMP:
                        self._amp(op, W, jamps, first_writes=False)
                    else:
                        self._header(op, W, pe)
                        self._variants(op, W, pe)
                mine = [h for h in range(self.nhel) if h & fix == self.bits]
                total[mine] += jamps[mine]
        self.fix, self.bits = 0, 0
        return self._finish(total, alpha_s, rnd_hel, rnd_col)

    def evaluate_cta(self, mom, alpha_s, rnd_hel=None, rnd_col=None):
        """The same through the block-per-event schedule: waves of (op, header or variant) items
        that a block's threads run in any order, amplitude steps into zeroed jamps.  Raises if an
        item of a wave reads or writes a slot that another item of the same wave writes (a race)."""
        T = self.P.cta
        nevt = mom.shape[0]
        pe = np.transpose(mom, (1, 2, 0))
        W = Workspace(T["store"], nevt)
        self.terms, self.flows = T["terms"], T["flows"]
        self.count = Counter()
        jamps = np.zeros((self.nhel, self.P.ncol, nevt), complex)
        for kind, start, count in T["steps"]:
            if kind == 0:
                logs = []
                for it in T["items"][start:start + count]:
                    op, v = T["ops"][it >> 8], it & 255
                    W.log = (set(), set())
                    if v == 255:
                        self._header(op, W, pe)
                    else:
                        self._variants(op, W, pe, [v])
                    logs.append((it, W.log))
                W.log = None
                _check_wave(logs)
            else:
                for a in range(start, start + count):
                    self._amp(T["ops"][a], W, jamps, first_writes=False)
        return self._finish(jamps, alpha_s, rnd_hel, rnd_col)

    def _finish(self, jamps, alpha_s, rnd_hel, rnd_col):
        P = self.P
        scale = (4 * math.pi * np.asarray(alpha_s)) ** P.gs_power
        mh = np.einsum("hie,ij,hje->eh", np.conj(jamps), self.C, jamps).real * scale[:, None]
        colw = (np.abs(jamps) ** 2).sum(axis=0).T * scale[:, None]
        out = dict(me=mh.sum(axis=1) / P.average_den, mh=mh, colw=colw)
        if rnd_hel is not None:
            out["selhel"] = _select(mh, rnd_hel)
        if rnd_col is not None:
            out["selcol"] = _select(colw, rnd_col)
        return out

    # -------------------------------------------------------------- headers
    def _header(self, op, W, pe):
        code, dst = op[0], op[1]
        if code == OP_SUM:
            return
        if code == OP_EXT:
            sgn = 1.0 if op[11] < self.P.nin else -1.0       # all momenta incoming
            W.set_k(dst, sgn * pe[op[11]])
            return
        if code in (OP_BIL, OP_RBIL):
            cl, cr, chiral = self.cpl[op[9]]
            W.set_cx(dst + 4, np.full(W.w.shape[1], 1.0 if chiral else cl))
            if code == OP_RBIL:
                iv = self._allowed(op[7])
                W.set_vec(dst + 6, iv, _slash(W.vec(op[14], iv)))
                self.count["slash_hdr"] += len(iv)
            return
        k = W.k(op[2]) + W.k(op[3])
        if code == OP_VVVV:
            k = k + W.k(op[4])
            W.set_k(dst, k)
            sv = -1.0 / np.einsum("m,me->e", METRIC, k * k)    # (-i)(-i g_s^2)/P^2 with g_s = 1
            W.set_r(dst + 4, sv)
            base = dst + 6
            for tab, (x, y) in enumerate(self._vvvv_pairs(op[11])):
                nx, ny = nvar(op[6 + x]), nvar(op[6 + y])
                ax, ay = self._allowed(op[6 + x]), self._allowed(op[6 + y])
                ex = W.vec(op[13 + x], ax)
                ey = W.vec(op[13 + y], ay)
                d = (-sv if tab else sv) * _mdot(ex[:, None], ey[None, :])     # [len ax, len ay, nevt]
                for jy, iy in enumerate(ay):
                    for jx, ix in enumerate(ax):
                        W.set_cx(base + 2 * (ix + nx * iy), d[jx, jy])
                base += 2 * nx * ny
                self.count["vvvv_hdr"] += len(ax) * len(ay)
            return
        W.set_k(dst, k)
        k2 = np.einsum("m,me->e", METRIC, k * k)
        if code == OP_VVV:
            ka, kb = W.k(op[2]), W.k(op[3])
            s = -1.0 / k2                                    # -i g_s/P^2 = i s with g_s = 1
            W.set_k(dst + 6, s * (ka - kb))
            q1 = s * (ka + 2 * kb)                           # s (k2 - k3)
            q2 = -s * (2 * ka + kb)                          # s (k3 - k1)
            W.set_k(dst + 10, q1)
            W.set_k(dst + 14, q2)
            n1 = nvar(op[6])
            i1, i2 = self._allowed(op[6]), self._allowed(op[7])
            e1, e2 = W.vec(op[13], i1), W.vec(op[14], i2)
            a1 = np.einsum("m,me,vme->ve", METRIC, q1, e1)
            a2 = np.einsum("m,me,vme->ve", METRIC, q2, e2)
            for j, v in enumerate(i1):
                W.set_cx(dst + 18 + 2 * v, a1[j])
            for j, v in enumerate(i2):
                W.set_cx(dst + 18 + 2 * (n1 + v), a2[j])
            self.count["vvv_hdr"] += len(i1) + len(i2)
            return
        m, w = self.mass[op[10]]
        inv = 1.0 / (k2 - m * m + 1j * m * w)
        pref = -1j * inv if code == OP_FFV_V else 1j * inv   # vector -i/(..), fermion i/(..)
        cl, cr, chiral = self.cpl[op[9]]
        if not chiral:
            pref = pref * cl
        if code == OP_FFV_V:
            W.set_cx(dst + 4, pref)
        else:
            iv = self._allowed(op[7])
            W.set_vec(dst + 6, iv, pref * _slash(W.vec(op[14], iv)))
            self.count["slash_hdr"] += len(iv)
            self.count["slash_pref_hdr"] += len(iv)

    @staticmethod
    def _vvvv_pairs(j):
        """Child pairs whose dot products the colour structure j needs (children 0, 1, 2)."""
        return [((0, 2), (1, 2)), ((0, 1), (1, 2)), ((0, 1), (0, 2))][j]

    # -------------------------------------------------------------- variants
    def _variants(self, op, W, pe, vs=None):
        """Variants vs (default: all) of one op."""
        code, dst, mdst = op[0], op[1], op[5]
        v = np.asarray(self._allowed(mdst)) if vs is None else np.asarray(vs)
        hb = [pdep(x, mdst) for x in v]
        if code in NAME:
            self.count["var_" + NAME[code]] += len(v)
        elif code == OP_SUM:
            self.count["sum_adds"] += (op[12] - 1) * len(v)
        child = lambda s: np.array([pext(h, op[6 + s]) for h in hb])
        if code == OP_EXT:
            p = pe[op[11]]
            m = self.mass[op[10]][0]
            kind = op[12]
            out = []
            for lam in (-1, 1):
                if kind == EXT_U:
                    w = _ext_u(p, m, lam)
                elif kind == EXT_V:
                    w = _ext_v(p, m, lam)
                elif kind == EXT_UBAR:
                    w = _bar(_ext_u(p, m, lam))
                elif kind == EXT_VBAR:
                    w = _bar(_ext_v(p, m, lam))
                else:
                    w = _ext_eps(p, lam, kind == EXT_EPS_OUT)
                out.append(w)
            W.set_vec(dst + 4, v, np.array(out)[v])
            return
        if code == OP_SUM:
            s = 0
            for t in range(op[12]):
                e = self.terms[8 * (op[11] + t):8 * (op[11] + t + 1)]
                s = s + PHASE[e[4]] * W.vec(e[0], v)
            W.set_vec(dst, v, s)
            return
        if code in (OP_FFV_F, OP_FFV_FB):
            psi = W.vec(op[13], child(0))
            A, B = _blocks(W.vec(dst + 6, child(1)))         # prefactor already in the slash entries
            cl, cr, chiral = self.cpl[op[9]]
            k = W.k(dst) if code == OP_FFV_F else -W.k(dst)  # a row current sees -k
            m = self.mass[op[10]][0]
            a00, a11 = k[0] - k[3], k[0] + k[3]
            ka01, ka10 = -k[1] + 1j * k[2], -k[1] - 1j * k[2]
            if code == OP_FFV_F:
                # psi' = (kslash + m) (pref Vslash) (cL PL + cR PR) psi
                u0 = A[0] * psi[:, 2] + A[1] * psi[:, 3]
                u1 = A[2] * psi[:, 2] + A[3] * psi[:, 3]
                l0 = B[0] * psi[:, 0] + B[1] * psi[:, 1]
                l1 = B[2] * psi[:, 0] + B[3] * psi[:, 1]
                if chiral:
                    u0, u1, l0, l1 = cr * u0, cr * u1, cl * l0, cl * l1
                out = [a00 * l0 + ka01 * l1 + m * u0, a11 * l1 + ka10 * l0 + m * u1,
                       a11 * u0 - ka01 * u1 + m * l0, a00 * u1 - ka10 * u0 + m * l1]
            else:
                # psibar' = psibar (pref Vslash) (cL PL + cR PR) (kslash + m)
                xu0 = psi[:, 2] * B[0] + psi[:, 3] * B[2]
                xu1 = psi[:, 2] * B[1] + psi[:, 3] * B[3]
                xl0 = psi[:, 0] * A[0] + psi[:, 1] * A[2]
                xl1 = psi[:, 0] * A[1] + psi[:, 1] * A[3]
                if chiral:
                    xu0, xu1, xl0, xl1 = cl * xu0, cl * xu1, cr * xl0, cr * xl1
                out = [a11 * xl0 - xl1 * ka10 + m * xu0, a00 * xl1 - xl0 * ka01 + m * xu1,
                       a00 * xu0 + xu1 * ka10 + m * xl0, a11 * xu1 + xu0 * ka01 + m * xl1]
            W.set_vec(dst + 6 + 8 * nvar(op[7]), v, np.stack(out, axis=1))
            return
        if code in (OP_FFV_V, OP_BIL):
            r = W.vec(op[13], child(0))
            c = W.vec(op[14], child(1))
            pref = W.cx(dst + 4)
            cl, cr, chiral = self.cpl[op[9]]
            # C^mu = cL rbar_l sigmabar^mu c_l + cR rbar_u sigma^mu c_u (chiral basis)
            R00, R11, R01, R10 = r[:, 0] * c[:, 2], r[:, 1] * c[:, 3], r[:, 0] * c[:, 3], r[:, 1] * c[:, 2]
            L00, L11, L01, L10 = r[:, 2] * c[:, 0], r[:, 3] * c[:, 1], r[:, 2] * c[:, 1], r[:, 3] * c[:, 0]
            Rv = np.stack([R00 + R11, R01 + R10, 1j * (R10 - R01), R00 - R11], axis=1)
            Lv = np.stack([L00 + L11, -(L01 + L10), -1j * (L10 - L01), -(L00 - L11)], axis=1)
            C = cl * Lv + cr * Rv if chiral else Lv + Rv
            M = self.mass[op[10]][0]
            if M > 0:
                k = W.k(dst)
                kC = np.einsum("m,me,vme->ve", METRIC, k, C)
                C = C - k[None] * (kC / (M * M))[:, None]
            W.set_vec(dst + 6, v, pref * C)
            return
        if code == OP_RBIL:
            pb = W.vec(op[13], child(0))
            A, B = _blocks(W.vec(dst + 6, child(1)))
            cl, cr, chiral = self.cpl[op[9]]
            x = [pb[:, 2] * B[0] + pb[:, 3] * B[2], pb[:, 2] * B[1] + pb[:, 3] * B[3],
                 pb[:, 0] * A[0] + pb[:, 1] * A[2], pb[:, 0] * A[1] + pb[:, 1] * A[3]]
            if chiral:
                x = [cl * x[0], cl * x[1], cr * x[2], cr * x[3]]
            W.set_vec(dst + 6 + 8 * nvar(op[7]), v, W.cx(dst + 4) * np.stack(x, axis=1))
            return
        if code == OP_VVV:
            i1, i2 = child(0), child(1)
            n1, n2 = nvar(op[6]), nvar(op[7])
            e1, e2 = W.vec(op[13], i1), W.vec(op[14], i2)
            d = W.k(dst + 6)
            a1 = np.array([W.cx(dst + 18 + 2 * i) for i in i1])
            a2 = np.array([W.cx(dst + 18 + 2 * (n1 + i)) for i in i2])
            s12 = _mdot(e1, e2)
            t = d[None] * s12[:, None] + e2 * a1[:, None] + e1 * a2[:, None]
            W.set_vec(dst + 18 + 2 * (n1 + n2), v, 1j * t)
            return
        if code == OP_VVVV:
            (x0, y0), (x1, y1) = self._vvvv_pairs(op[11])
            nx0, ny0, nx1, ny1 = (nvar(op[6 + s]) for s in (x0, y0, x1, y1))
            t0 = dst + 6
            t1 = t0 + 2 * nx0 * ny0
            X = np.array([W.cx(t0 + 2 * (pext(h, op[6 + x0]) + nx0 * pext(h, op[6 + y0]))) for h in hb])
            Y = np.array([W.cx(t1 + 2 * (pext(h, op[6 + x1]) + nx1 * pext(h, op[6 + y1]))) for h in hb])
            m0, m1 = 3 - x0 - y0, 3 - x1 - y1
            a = W.vec(op[13 + m0], child(m0))
            b = W.vec(op[13 + m1], child(m1))
            W.set_vec(t1 + 2 * nx1 * ny1, v, X[:, None] * a + Y[:, None] * b)
            return
        raise ValueError(f"op code {code}")

    # -------------------------------------------------------------- amplitudes
    def _amp(self, op, W, jamps, first_writes=True):
        """Group amplitude for every helicity: runs of terms sharing a bilinear X, the phased
        other operands summed and closed with one product; then added to the group's flows (a
        flow's first update writes, in the thread-per-event program)."""
        h = np.array([x for x in range(self.nhel) if x & self.fix == self.bits])
        acc = 0
        s = None
        self.count.update(amp=1, amp_terms=op[12], amp_flows=op[10])
        for t in range(op[12]):
            e = self.terms[8 * (op[11] + t):8 * (op[11] + t + 1)]
            self.count["amp_runs"] += e[7]
            Y = W.vec(e[2], [pext(x, e[3]) for x in h])            # [nhel, 4, nevt]
            s = PHASE[e[4]] * Y if e[6] else s + PHASE[e[4]] * Y
            if e[7]:
                X = W.vec(e[0], [pext(x, e[1]) for x in h])
                acc = acc + (_mdot(X, s) if e[5] == 0 else (X * s).sum(axis=1))
        for f in range(op[10]):
            flow, code = self.flows[2 * (op[9] + f):2 * (op[9] + f) + 2]
            j = PHASE[code & 3] * acc
            jamps[h, flow] = j if first_writes and code & FLOW_FIRST else jamps[h, flow] + j
