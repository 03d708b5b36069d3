"""Diagram interpreter: each Feynman-diagram term as an explicit tensor contraction.

For every diagram (split into one term per colour structure of each four-gluon
vertex) the Lorentz part is the einsum of
  * external wavefunctions  u, v, ubar, vbar, eps (lowered index), one helicity axis each,
  * vertex tensors (upper Lorentz indices, couplings included),
  * propagators (lower Lorentz indices),
and the colour part is the einsum of T^a_ij and f^abc over internal colour
indices.  The Feynman rules (Peskin & Schroeder conventions, all momenta
incoming at a vertex):
  q q g  :  i g_s gamma^mu T^a_ij           (i: barred side, j: unbarred side)
  f f a  : -i e Q gamma^mu
  f f z  : -i gamma^mu (gL P_L + gR P_R)
  g g g  :  g_s f^abc [g^mn (k1-k2)^r + g^nr (k2-k3)^m + g^rm (k3-k1)^n]
  gggg   : -i g_s^2 [f^abe f^cde (g^mr g^ns - g^ms g^nr) + f^ace f^bde (g^mn g^rs - g^ms g^nr)
                     + f^ade f^bce (g^mn g^rs - g^mr g^ns)]
  fermion: i (kslash + m) / (k^2 - m^2 + i m Gamma)   (k along fermion-number flow)
  g, a   : -i g_mn / k^2
  z      : -i (g_mn - k_m k_n / mZ^2) / (k^2 - mZ^2 + i mZ GammaZ)
The value of a diagram is i*M; the returned amplitudes are M = -i * contraction.
"""
import itertools
import math

import numpy as np

from . import lorentz as L
from .colour import T as TCOL, F as FCOL
from .diagrams import enumerate_diagrams, parse_process, crossed
from .model import PARTICLES, Params


def _vvv(k1, k2, k3):
    g = L.METRIC
    d12, d23, d31 = k1 - k2, k2 - k3, k3 - k1
    return (np.einsum("mn,er->emnr", g, d12) + np.einsum("nr,em->emnr", g, d23)
            + np.einsum("rm,en->emnr", g, d31)).astype(complex)


def _vvvv_structures():
    g = L.METRIC
    gg = lambda a, b, c, d: np.einsum(f"{a}{b},{c}{d}->mnrs", g, g)
    return [gg("m", "r", "n", "s") - gg("m", "s", "n", "r"),
            gg("m", "n", "r", "s") - gg("m", "s", "n", "r"),
            gg("m", "n", "r", "s") - gg("m", "r", "n", "s")]


VVVV = [x.astype(complex) for x in _vvvv_structures()]
_COLOUR_OPS = {"T": TCOL, "F": FCOL, "D": np.eye(3, dtype=complex)}


def _einsum(*args):
    """np.einsum in sublist form with arbitrary hashable labels (remapped to 0..51)."""
    ops, subs = list(args[0:-1:2]), [list(s) for s in args[1:-1:2]]
    out = list(args[-1])
    names = {}
    for s in subs + [out]:
        for x in s:
            names.setdefault(x, len(names))
    if len(names) > 52:
        raise ValueError("too many einsum labels")
    call = []
    for o, s in zip(ops, subs):
        call += [o, [names[x] for x in s]]
    return np.einsum(*call, [names[x] for x in out], optimize="greedy")


class Process:
    """Oracle process: diagrams, colour decomposition and the amplitude evaluator."""

    def __init__(self, proc, params=None):
        self.proc = proc
        self.params = params or Params()
        self.incoming, self.outgoing = parse_process(proc)
        self.particles = self.incoming + self.outgoing
        self.nin = len(self.incoming)
        self.npar = len(self.particles)
        self.names, self.diagrams = enumerate_diagrams(self.incoming, self.outgoing)
        self.coloured_legs = [i for i, p in enumerate(self.particles) if PARTICLES[p].colour != 1]
        self.gluon_legs = [i for i, p in enumerate(self.particles) if PARTICLES[p].colour == 8]
        quark_legs = [i for i, p in enumerate(self.particles) if abs(PARTICLES[p].colour) == 3]
        self.row_leg = self.col_leg = None
        for i in quark_legs:
            # incoming flavour of the leg: antifermion -> barred (row) end
            if PARTICLES[self.names[i]].is_anti:
                self.row_leg = i
            else:
                self.col_leg = i
        if len(quark_legs) not in (0, 2):
            raise NotImplementedError("only processes with at most one quark line")
        self.terms = []
        for d_index, d in enumerate(self.diagrams):
            self.terms.extend(self._build_terms(d_index, d))

    # ------------------------------------------------------------------ building
    def _build_terms(self, d_index, diagram):
        """Return a list of term descriptions for one diagram."""
        n = self.npar
        lab = itertools.count(1)
        ev = 0
        hel = {i: next(lab) for i in range(n)}
        ops_l = []          # (kind, payload, labels)
        ops_c = []          # (kind, labels) kind in 'T','F'
        ext_l = {}          # external leg -> Lorentz/spinor label
        ext_c = {i: next(lab) for i in self.coloured_legs}
        four_vertices = []  # index into ops placeholders

        def vertex(incident):
            """incident: list of (flav_in, legs_sign, label, colour_label)."""
            flavs = [x[0] for x in incident]
            spins = [PARTICLES[f].spin for f in flavs]
            if len(incident) == 4:
                four_vertices.append(([x[1] for x in incident], [x[2] for x in incident],
                                      [x[3] for x in incident]))
                return
            if spins.count(1) == 2:
                b = spins.index(2)
                fer = [k for k in range(3) if spins[k] == 1]
                row = [k for k in fer if PARTICLES[flavs[k]].is_anti][0]
                col = [k for k in fer if not PARTICLES[flavs[k]].is_anti][0]
                boson = flavs[b]
                fpart = PARTICLES[flavs[col]]
                ops_l.append(("ffv", (boson, fpart.name), (incident[b][2], incident[row][2], incident[col][2])))
                if boson == "g":
                    ops_c.append(("T", (incident[b][3], incident[row][3], incident[col][3])))
                elif abs(fpart.colour) == 3:
                    # colourless boson on a quark line: colour passes through unchanged
                    ops_c.append(("D", (incident[row][3], incident[col][3])))
            else:
                ops_l.append(("vvv", tuple(x[1] for x in incident), tuple(x[2] for x in incident)))
                ops_c.append(("F", tuple(x[3] for x in incident)))

        def walk(line, consumer_label, consumer_colour):
            """Attach `line` whose consumer-side index is consumer_label."""
            if not line.children:
                ext_l[line.leg] = consumer_label
                if line.leg in ext_c:
                    # the external colour label is identified with the consumer-side label
                    subst[consumer_colour] = ext_c[line.leg]
                return
            p_lab = next(lab)
            p_col = consumer_colour
            # propagator between producer and consumer
            fl = line.flav
            part = PARTICLES[fl]
            legs = tuple(sorted(line.legs))
            if part.spin == 2:
                ops_l.append(("vprop", (fl, legs), (p_lab, consumer_label)))
            elif not part.is_anti:
                ops_l.append(("fprop", (fl, legs, +1), (consumer_label, p_lab)))
            else:
                ops_l.append(("fprop", (fl, legs, -1), (p_lab, consumer_label)))
            incident = []
            for c in line.children:
                c_lab = next(lab)
                c_col = next(lab)
                incident.append((c.flav, (tuple(sorted(c.legs)), +1), c_lab, c_col))
                walk(c, c_lab, c_col)
            incident.append((crossed(fl), (legs, -1), p_lab, p_col))
            vertex(incident)

        subst = {}
        incident = []
        for line in diagram.top:
            c_lab = next(lab)
            c_col = next(lab)
            incident.append((line.flav, (tuple(sorted(line.legs)), +1), c_lab, c_col))
            walk(line, c_lab, c_col)
        vertex(incident)

        def sc(x):
            while x in subst:
                x = subst[x]
            return x

        terms = []
        for choice in itertools.product(range(3), repeat=len(four_vertices)):
            tl = list(ops_l)
            tc = list(ops_c)
            for (momenta, labels, cols), j in zip(four_vertices, choice):
                tl.append(("vvvv", j, tuple(labels)))
                e = next(lab)
                a, b, c, d = cols
                pairs = [((a, b, e), (c, d, e)), ((a, c, e), (b, d, e)), ((a, d, e), (b, c, e))][j]
                tc.append(("F", pairs[0]))
                tc.append(("F", pairs[1]))
            tc = [(k, tuple(sc(x) for x in labs)) for k, labs in tc]
            terms.append(dict(diagram=d_index, lorentz=tl, colour=tc, ext_l=dict(ext_l),
                              hel=dict(hel), ext_c=dict(ext_c)))
        return terms

    # ------------------------------------------------------------------ numerics
    def incoming_momenta(self, p):
        """Momenta flowing into the diagram: +p for initial, -p for final legs."""
        q = p.copy()
        q[:, self.nin:] *= -1.0
        return q

    def external_wavefunction(self, i, p):
        name = self.particles[i]
        part = PARTICLES[name]
        m = self.params.mass(part)
        pi = p[:, i]
        initial = i < self.nin
        if part.spin == 2:
            eps = L.polarisation(pi)
            if not initial:
                eps = eps.conj()
            return eps @ L.METRIC  # lowered index
        if initial:
            return L.bar(L.v_spinor(pi, m)) if part.is_anti else L.u_spinor(pi, m)
        return L.v_spinor(pi, m) if part.is_anti else L.bar(L.u_spinor(pi, m))

    def _lorentz_operand(self, op, q, gs):
        kind, payload, labels = op
        prm = self.params
        ev = 0
        if kind == "ffv":
            boson, fname = payload
            fpart = PARTICLES[fname]
            if boson == "g":
                t = 1j * gs[:, None, None, None] * L.GAMMA[None]
            elif boson == "a":
                t = (-1j * prm.ee * fpart.charge * L.GAMMA)[None]
            else:
                gl, gr = prm.z_couplings(fpart)
                t = (-1j * np.einsum("mab,bc->mac", L.GAMMA, gl * L.PL + gr * L.PR))[None]
            if t.shape[0] == 1:
                return t[0], list(labels)
            return t, [ev] + list(labels)
        if kind == "vvv":
            ks = [sign * sum(q[:, i] for i in legs) for legs, sign in payload]
            return gs[:, None, None, None] * _vvv(*ks), [ev] + list(labels)
        if kind == "vvvv":
            return -1j * (gs * gs)[:, None, None, None, None] * VVVV[payload][None], [ev] + list(labels)
        if kind == "vprop":
            fl, legs = payload
            k = sum(q[:, i] for i in legs)
            k2 = L.minkowski(k, k)
            part = PARTICLES[fl]
            if fl == "z":
                m, w = prm.mz, prm.wz
                klow = k @ L.METRIC
                num = L.METRIC[None] - np.einsum("em,en->emn", klow, klow) / (m * m)
                return -1j * num / (k2 - m * m + 1j * m * w)[:, None, None], [ev] + list(labels)
            return (-1j * L.METRIC[None] / k2[:, None, None]).astype(complex), [ev] + list(labels)
        if kind == "fprop":
            fl, legs, orient = payload
            k = orient * sum(q[:, i] for i in legs)
            part = PARTICLES[fl]
            m, w = prm.mass(part), prm.width(part)
            k2 = L.minkowski(k, k)
            num = L.slash(k) + m * np.eye(4)[None]
            return 1j * num / (k2 - m * m + 1j * m * w)[:, None, None], [ev] + list(labels)
        raise ValueError(kind)

    def term_amplitudes(self, p, alpha_s, gauge_leg=None):
        """A[t, nevt, 2**npar] for every term t (canonical helicity order).

        gauge_leg: replace that external vector's polarisation by its momentum
        (lowered index) in both helicity slots -- the Ward-identity check.
        """
        nevt = p.shape[0]
        q = self.incoming_momenta(p)
        gs = np.sqrt(4.0 * math.pi * np.asarray(alpha_s, dtype=float)) * np.ones(nevt)
        wf = [self.external_wavefunction(i, p) for i in range(self.npar)]
        if gauge_leg is not None:
            k = (p[:, gauge_leg] @ L.METRIC).astype(complex)
            wf[gauge_leg] = np.stack([k, k], axis=1)
        out = np.zeros((len(self.terms), nevt, 2 ** self.npar), dtype=complex)
        for t, term in enumerate(self.terms):
            args = []
            for i in range(self.npar):
                args += [wf[i], [0, term["hel"][i], term["ext_l"][i]]]
            for op in term["lorentz"]:
                arr, labs = self._lorentz_operand(op, q, gs)
                args += [arr, labs]
            outl = [0] + [term["hel"][i] for i in range(self.npar)]
            r = _einsum(*args, outl)
            out[t] = -1j * r.reshape(nevt, -1)
        return out

    def term_colour(self, term, configs=None):
        """Colour tensor of a term: dense [8|3, ...] over coloured legs, or at configs [R, ncl]."""
        args = []
        ext = [term["ext_c"][i] for i in self.coloured_legs]
        if configs is None:
            for kind, labs in term["colour"]:
                args += [_COLOUR_OPS[kind], list(labs)]
            if not args:
                return np.ones(())
            return _einsum(*args, ext)
        R = configs.shape[0]
        batch = 10 ** 6
        pos = {lab: k for k, lab in enumerate(ext)}
        for kind, labs in term["colour"]:
            arr = _COLOUR_OPS[kind].astype(complex)
            new_labs = []
            fixed = [(ax, pos[l]) for ax, l in enumerate(labs) if l in pos]
            if fixed:
                # gather the external indices per configuration
                idx = [slice(None)] * arr.ndim
                for ax, k in fixed:
                    idx[ax] = configs[:, k]
                # advanced indexing moves the gathered axes to the front when they are separated
                sel = np.moveaxis(arr, [ax for ax, _ in fixed], list(range(len(fixed))))
                sel = sel[tuple(configs[:, k] for _, k in fixed)]
                new_labs = [batch] + [l for l in labs if l not in pos]
                args += [sel, new_labs]
            else:
                args += [arr, list(labs)]
        if not args:
            return np.ones(R, dtype=complex)
        return _einsum(*args, [batch])
