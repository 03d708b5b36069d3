"""Brute-force enumeration of tree-level Feynman diagrams.

Every external particle is treated as incoming (an outgoing particle X enters as
its antiparticle).  A diagram is grown by repeatedly merging two or three open
lines at an allowed vertex into one new line; it is complete when the open lines
meet at a single vertex.  Different merge orders reach the same tree, so trees
are identified by their set of internal lines, each written as (set of external
legs on the side without the last leg, effective particle entering from that
side) -- a tree is fixed by its splits and their particle types.

The vertex set is the SM one restricted to the particles that occur:
  {q~ q g}, {g g g}, {g g g g}          (QCD)
  {f~ f a} for charged f, {f~ f z}      (electroweak neutral currents)
"""
import itertools
from dataclasses import dataclass, field

from .model import PARTICLES


def crossed(name):
    return PARTICLES[name].anti


@dataclass(frozen=True)
class Line:
    """An open line: external leg (legs of size 1) or a merged subtree."""
    flav: str                 # particle entering the rest of the diagram from this subtree
    legs: frozenset
    children: tuple = ()      # child Lines (empty for an external leg)
    leg: int = -1             # external leg index when external

    def internal_lines(self):
        out = set()
        for c in self.children:
            out |= c.internal_lines()
        if self.children:
            out.add((self.legs, self.flav))
        return out


@dataclass
class Diagram:
    """A tree: the lines meeting at the final vertex (each itself a subtree)."""
    top: tuple
    key: frozenset = field(default=None)


def vertex_set(flavours, ew):
    """Allowed vertices as sorted tuples of incoming particle names."""
    fermions = sorted({f for f in flavours if PARTICLES[f].spin == 1 and not PARTICLES[f].is_anti})
    has_gluon = any(PARTICLES[f].colour == 8 for f in flavours) or any(PARTICLES[f].colour == 3 for f in fermions)
    verts = set()
    for f in fermions:
        p = PARTICLES[f]
        if p.colour == 3:
            verts.add(tuple(sorted((p.anti, f, "g"))))
        if ew:
            if p.charge != 0.0:
                verts.add(tuple(sorted((p.anti, f, "a"))))
            verts.add(tuple(sorted((p.anti, f, "z"))))
    if has_gluon:
        verts.add(("g", "g", "g"))
        verts.add(("g", "g", "g", "g"))
    return verts


def _normalise(legs, flav, n):
    last = n - 1
    if last in legs:
        comp = frozenset(range(n)) - legs
        return (comp, crossed(flav))
    return (legs, flav)


def enumerate_diagrams(incoming, outgoing, ew=None):
    """All distinct tree diagrams for `incoming > outgoing` (lists of particle names).

    Returns a list of Diagram objects in a deterministic order (sorted by key).
    """
    names = list(incoming) + [crossed(p) for p in outgoing]
    n = len(names)
    if ew is None:
        ew = not any(PARTICLES[p].colour != 1 for p in names)
        ew = ew or any(PARTICLES[p].colour == 1 and PARTICLES[p].spin == 1 for p in names)
    verts = vertex_set(set(names) | {crossed(x) for x in names}, ew)
    three = {v for v in verts if len(v) == 3}
    four = {v for v in verts if len(v) == 4}
    lines0 = tuple(Line(names[i], frozenset([i]), (), i) for i in range(n))
    found = {}
    seen = set()

    def key_of(lines):
        s = set()
        for L in lines:
            for (legs, fl) in L.internal_lines():
                s.add(_normalise(legs, fl, n))
        return frozenset(s)

    def state_key(lines):
        return frozenset((L.legs, L.flav, frozenset(_normalise(a, b, n) for a, b in L.internal_lines()))
                         for L in lines)

    def rec(lines):
        sk = state_key(lines)
        if sk in seen:
            return
        seen.add(sk)
        m = len(lines)
        flavs = [L.flav for L in lines]
        # completion at a single vertex
        if (m == 3 and tuple(sorted(flavs)) in three) or (m == 4 and tuple(sorted(flavs)) in four):
            k = key_of(lines)
            if k not in found:
                found[k] = Diagram(tuple(lines), k)
        if m <= 3 and not (m == 4):
            if m <= 3:
                pass
        # merge two lines through a 3-vertex
        for i, j in itertools.combinations(range(m), 2):
            for v in three:
                rest = list(v)
                ok = True
                for f in (flavs[i], flavs[j]):
                    if f in rest:
                        rest.remove(f)
                    else:
                        ok = False
                        break
                if not ok:
                    continue
                new = Line(crossed(rest[0]), lines[i].legs | lines[j].legs, (lines[i], lines[j]))
                if len(new.legs) == n or m - 1 < 3:
                    continue
                rec(tuple(L for t, L in enumerate(lines) if t not in (i, j)) + (new,))
        # merge three lines through a 4-vertex
        for i, j, k in itertools.combinations(range(m), 3):
            for v in four:
                rest = list(v)
                ok = True
                for f in (flavs[i], flavs[j], flavs[k]):
                    if f in rest:
                        rest.remove(f)
                    else:
                        ok = False
                        break
                if not ok:
                    continue
                new = Line(crossed(rest[0]), lines[i].legs | lines[j].legs | lines[k].legs,
                           (lines[i], lines[j], lines[k]))
                if m - 2 < 3:
                    continue
                rec(tuple(L for t, L in enumerate(lines) if t not in (i, j, k)) + (new,))

    rec(lines0)
    diags = [found[k] for k in sorted(found, key=lambda k: sorted((sorted(a), b) for a, b in k))]
    return names, diags


def parse_process(proc):
    lhs, rhs = proc.split(">")
    return lhs.split(), rhs.split()
