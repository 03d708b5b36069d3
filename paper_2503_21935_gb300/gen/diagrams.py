"""Tree diagrams as off-shell currents rooted at one external leg.

The root is the barred end of the (single) fermion line: the external antifermion
in the all-incoming picture (an outgoing fermion's ubar, or an incoming
antifermion's vbar).  Every other external subset S gets the list of distinct
off-shell currents over S (one per distinct subtree), built bottom-up by
popcount; a diagram term is the root vertex closing the root leg with currents
covering the remaining legs.  Each four-gluon vertex contributes three currents,
one per colour structure, so a diagram with k such vertices gives 3^k terms.

Colour: with the root at the barred quark end no gluon current contains a quark,
so every current carries its colour as a polynomial in ordered gluon words
(f^{xyz} T^z = -i [T^x, T^y] applied recursively); a fermion current carries the
ordered word of the gluons attached between it and the unbarred end.
"""
from dataclasses import dataclass, field

from . import sm


@dataclass
class Current:
    id: int
    mask: int
    flav: str           # particle entering the consumer vertex from this subtree
    op: str             # EXT, FFV_F (column spinor), FFV_FB (row spinor), FFV_V, VVV, VVVV
    children: tuple = ()
    struct: int = -1    # four-gluon colour structure 0..2
    leg: int = -1
    colour: dict = field(default_factory=dict)   # word (tuple of gluon legs) -> complex


@dataclass
class Term:
    diagram: int
    row: int            # root external (row spinor) current id
    col: int            # column-spinor current id
    vec: int            # vector current id
    colour: dict


def _mul(a, b):
    out = {}
    for wa, ca in a.items():
        for wb, cb in b.items():
            w = wa + wb
            out[w] = out.get(w, 0) + ca * cb
    return {w: c for w, c in out.items() if c != 0}


def _add(a, b, s=1):
    out = dict(a)
    for w, c in b.items():
        out[w] = out.get(w, 0) + s * c
    return {w: c for w, c in out.items() if c != 0}


def _comm(a, b):
    """-i [a, b]"""
    return {w: -1j * c for w, c in _add(_mul(a, b), _mul(b, a), -1).items()}


def _scale(a, s):
    return {w: s * c for w, c in a.items()}


class Diagrams:
    def __init__(self, incoming, outgoing, ew=None):
        self.incoming = list(incoming)
        self.outgoing = list(outgoing)
        names = self.incoming + self.outgoing
        self.npar = len(names)
        self.nin = len(self.incoming)
        # all-incoming flavours
        self.flav_in = [p if i < self.nin else sm.anti(p) for i, p in enumerate(names)]
        fermion_legs = [i for i, f in enumerate(self.flav_in) if sm.kind(f) == "F"]
        bar = [i for i in fermion_legs if sm.is_anti(self.flav_in[i])]
        quark_lines = [i for i in fermion_legs if abs(sm.colour(self.flav_in[i])) == 3]
        if len(quark_lines) > 2:
            raise NotImplementedError("at most one quark line is supported")
        if not bar:
            raise NotImplementedError("processes without an external fermion line are not supported")
        qbar = [i for i in bar if abs(sm.colour(self.flav_in[i])) == 3]
        self.root = qbar[0] if qbar else bar[0]
        self.gluons = [i for i, f in enumerate(self.flav_in) if f == "g"]
        coloured = any(sm.colour(f) != 1 for f in self.flav_in)
        if ew is None:
            ew = any(sm.kind(f) == "F" and sm.colour(f) == 1 for f in self.flav_in)
        self.ew = ew
        self.qcd = coloured
        self.currents = []
        self.by_mask = {}
        self._build()

    # ------------------------------------------------------------ vertices
    def _bosons_for(self, fermion):
        out = []
        if abs(sm.colour(fermion)) == 3 and self.qcd:
            out.append("g")
        if self.ew:
            if sm.charge(fermion) != 0.0:
                out.append("a")
            out.append("z")
        return out

    def _combine2(self, c1, c2):
        """Currents produced by joining c1, c2 at a three-point vertex."""
        f1, f2 = c1.flav, c2.flav
        k1, k2 = sm.kind(f1), sm.kind(f2)
        out = []
        if k1 == "V" and k2 == "V":
            if f1 == "g" and f2 == "g":
                out.append(("VVV", "g", (c1, c2), _comm(c1.colour, c2.colour)))
            return out
        if k1 == "F" and k2 == "F":
            if sm.anti(f1) != f2:
                return out
            row, col = (c1, c2) if sm.is_anti(f1) else (c2, c1)
            base = row.flav if not sm.is_anti(row.flav) else sm.anti(row.flav)
            for b in self._bosons_for(base):
                if b == "g":
                    raise NotImplementedError("quark pair into a gluon needs a second colour line")
                out.append(("FFV_V", b, (row, col), _mul(row.colour, col.colour)))
            return out
        ferm, vec = (c1, c2) if k1 == "F" else (c2, c1)
        base = ferm.flav if not sm.is_anti(ferm.flav) else sm.anti(ferm.flav)
        if vec.flav not in self._bosons_for(base):
            return out
        if sm.is_anti(ferm.flav):
            out.append(("FFV_FB", ferm.flav, (ferm, vec), _mul(ferm.colour, vec.colour)))
        else:
            out.append(("FFV_F", ferm.flav, (ferm, vec), _mul(vec.colour, ferm.colour)))
        return out

    def _new(self, mask, flav, op, children=(), struct=-1, leg=-1, colour=None):
        c = Current(len(self.currents), mask, flav, op, tuple(x.id for x in children), struct, leg,
                    colour if colour is not None else {(): 1})
        self.currents.append(c)
        self.by_mask.setdefault(mask, []).append(c)
        return c

    def _build(self):
        n = self.npar
        for i in range(n):
            if i == self.root:
                continue
            f = self.flav_in[i]
            self._new(1 << i, f, "EXT", leg=i, colour={(i,): 1} if f == "g" else {(): 1})
        # the root's external wavefunction is a current too (not offered to subtree building)
        self.root_current = Current(len(self.currents), 1 << self.root, self.flav_in[self.root], "EXT",
                                    leg=self.root)
        self.currents.append(self.root_current)
        full = ((1 << n) - 1) & ~(1 << self.root)
        masks = sorted((m for m in range(1, full + 1) if m & full == m), key=lambda m: (bin(m).count("1"), m))
        for S in masks:
            if bin(S).count("1") < 2:
                continue
            low = S & -S
            # two-way splits: S1 holds the lowest leg
            sub = (S - 1) & S
            while sub:
                if sub & low and sub != S:
                    S1, S2 = sub, S ^ sub
                    for c1 in list(self.by_mask.get(S1, [])):
                        for c2 in list(self.by_mask.get(S2, [])):
                            for op, flav, ch, col in self._combine2(c1, c2):
                                self._new(S, flav, op, ch, colour=col)
                sub = (sub - 1) & S
            # three-way splits through the four-gluon vertex
            for S1 in self._submasks_with(S, low):
                R1 = S ^ S1
                if not R1:
                    continue
                low2 = R1 & -R1
                for S2 in self._submasks_with(R1, low2):
                    S3 = R1 ^ S2
                    if not S3:
                        continue
                    for a in self.by_mask.get(S1, []):
                        if a.flav != "g":
                            continue
                        for b in self.by_mask.get(S2, []):
                            if b.flav != "g":
                                continue
                            for c in self.by_mask.get(S3, []):
                                if c.flav != "g":
                                    continue
                                Wa, Wb, Wc = a.colour, b.colour, c.colour
                                cols = [_scale(_comm(_comm(Wa, Wb), Wc), 1),
                                        _scale(_comm(_comm(Wa, Wc), Wb), 1),
                                        _scale(_comm(_comm(Wb, Wc), Wa), 1)]
                                for j in range(3):
                                    self._new(S, "g", "VVVV", (a, b, c), struct=j, colour=cols[j])
        # root terms
        self.terms = []
        rf = self.flav_in[self.root]
        base = sm.anti(rf)
        diag_of = {}
        sub = (full - 1) & full
        low = full & -full
        while sub:
            if sub & low:
                S1, S2 = sub, full ^ sub
                for c1 in self.by_mask.get(S1, []):
                    for c2 in self.by_mask.get(S2, []):
                        pair = [c1, c2]
                        ferm = [c for c in pair if sm.kind(c.flav) == "F"]
                        vec = [c for c in pair if sm.kind(c.flav) == "V"]
                        if len(ferm) != 1 or len(vec) != 1:
                            continue
                        if ferm[0].flav != base or vec[0].flav not in self._bosons_for(base):
                            continue
                        colour = _mul(vec[0].colour, ferm[0].colour)
                        key = self._diagram_key(ferm[0]), self._diagram_key(vec[0])
                        d = diag_of.setdefault(key, len(diag_of))
                        self.terms.append(Term(d, -1, ferm[0].id, vec[0].id, colour))
            sub = (sub - 1) & full
        self.ndiagrams = len(diag_of)

    @staticmethod
    def _submasks_with(S, bit):
        out = []
        sub = S
        while sub:
            if sub & bit:
                out.append(sub)
            sub = (sub - 1) & S
        return out

    def _diagram_key(self, c):
        """Identity of the subtree with four-gluon colour structures merged."""
        if c.op == "EXT":
            return ("E", c.leg)
        kids = tuple(self._diagram_key(self.currents[k]) for k in c.children)
        op = c.op
        return (op, c.flav, kids)
