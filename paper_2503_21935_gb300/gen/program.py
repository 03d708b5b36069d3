"""Emit the op table ("program") executed by the generic CUDA amplitude kernel.

One program per process.  Each op is 16 int32 fields:
  0 code  1 dst  2 a  3 b  4 c  5 mask_dst  6 mask_a  7 mask_b  8 mask_c
  9 coupling  10 mass/width entry  11 aux  12 aux2  13..15 reserved
Offsets (fields 1-4) are in doubles inside a per-event workspace block:
  block = [k0 k1 k2 k3 | variant 0: 4 complex | variant 1 | ...]
where k is the current's incoming momentum and variant v holds the current for
the helicities pdep(v, mask) of the legs in `mask` (leg p <-> bit npar-1-p, the
bit of the canonical helicity index).  A current is computed once per helicity
state of its own legs (helicity recycling) and its block is freed after its last
use.  AMP ops close a diagram term at the root vertex for every good helicity
and add it, times a phase in {1, i, -1, -i}, to the term's colour flows.
"""
import itertools
import math
from dataclasses import dataclass, field
from fractions import Fraction

from . import sm
from .colour import colour_matrix
from .diagrams import Diagrams

OP_EXT, OP_FFV_F, OP_FFV_FB, OP_FFV_V, OP_VVV, OP_VVVV, OP_AMP = 1, 2, 3, 4, 5, 6, 7
EXT_U, EXT_V, EXT_UBAR, EXT_VBAR, EXT_EPS_IN, EXT_EPS_OUT = 0, 1, 2, 3, 4, 5
NFIELD = 16

# coupling flags
C_GS = 1        # multiply by the per-event strong coupling g_s
C_CHIRAL = 2    # left and right couplings differ

_PHASE = {1: 0, 1j: 1, -1: 2, -1j: 3}


@dataclass
class Program:
    process: str
    npar: int
    nin: int
    root: int
    ops: list
    flows: list                 # flattened (flow, phase code) pairs
    perms: list
    colour: list                # exact Fractions
    couplings: list             # (kind, fermion) specs resolved at process creation
    masses: list                # mass/width parameter names per table entry
    ext_mass: list
    ws_current_doubles: int
    ndiagrams: int
    nterms: int
    average_den: int            # 1 / average factor
    flop_counts: dict = field(default_factory=dict)

    @property
    def ncol(self):
        return len(self.perms)


def _bit(npar, leg):
    return 1 << (npar - 1 - leg)


def build_program(process):
    lhs, rhs = process.split(">")
    inc, out = lhs.split(), rhs.split()
    D = Diagrams(inc, out)
    npar = D.npar
    cur = D.currents

    def hmask(m):
        # convert a leg bitmask (bit leg) to helicity-bit positions (bit npar-1-leg)
        return sum(_bit(npar, p) for p in range(npar) if m >> p & 1)

    # ---- mass / coupling tables
    masses = [("", "")]
    def mass_index(flav):
        key = (sm.mass_param(flav), sm.width_param(flav))
        if key == ("", ""):
            return 0
        if key not in masses:
            masses.append(key)
        return masses.index(key)

    couplings = []
    def coupling_index(boson, fermion):
        base = fermion if not sm.is_anti(fermion) else sm.anti(fermion)
        spec = (boson, base if boson != "g" else "")
        if spec not in couplings:
            couplings.append(spec)
        return couplings.index(spec)

    # ---- schedule: depth-first from each term
    order = []
    done = set()
    def emit(i):
        if i in done:
            return
        for k in cur[i].children:
            emit(k)
        done.add(i)
        order.append(("C", i))
    for ti, t in enumerate(D.terms):
        emit(t.col)
        emit(t.vec)
        order.append(("A", ti))
    ROOT = -1
    order.insert(0, ("C", ROOT))

    def uses(item):
        kind, x = item
        if kind == "C":
            return [] if x == ROOT else list(cur[x].children)
        t = D.terms[x]
        return [ROOT, t.col, t.vec]

    last = {}
    for pos, item in enumerate(order):
        for u in uses(item):
            last[u] = pos

    def nvar(i):
        m = D.root_current.mask if i == ROOT else cur[i].mask
        return 1 << bin(m).count("1")

    # ---- first-fit allocation of current blocks
    free = []          # list of (start, size)
    top = 0
    offset = {}

    def alloc(size):
        nonlocal top
        for k, (s, z) in enumerate(free):
            if z >= size:
                if z == size:
                    free.pop(k)
                else:
                    free[k] = (s + size, z - size)
                return s
        s = top
        top += size
        return s

    def release(s, size):
        free.append((s, size))
        free.sort()
        merged = []
        for a, z in free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + z)
            else:
                merged.append((a, z))
        free[:] = merged

    def blocksize(i):
        return 4 + 8 * nvar(i)

    ops = []
    flows = []
    ext_mass = [0] * npar
    counts = dict(ext=0, ffv_f=0, ffv_fb=0, ffv_v=0, vvv=0, vvvv=0, amp=0, amp_flows=0,
                  var_ffv_f=0, var_ffv_fb=0, var_ffv_v=0, var_vvv=0, var_vvvv=0)
    for pos, item in enumerate(order):
        kind, x = item
        op = [0] * NFIELD
        if kind == "C":
            c = D.root_current if x == ROOT else cur[x]
            off = alloc(blocksize(x))
            offset[x] = off
            op[1] = off
            op[5] = hmask(c.mask)
            if c.op == "EXT":
                leg = c.leg
                f = c.flav                      # all-incoming flavour
                initial = leg < D.nin
                if sm.kind(f) == "V":
                    etype = EXT_EPS_IN if initial else EXT_EPS_OUT
                else:
                    phys = D.incoming[leg] if initial else D.outgoing[leg - D.nin]
                    anti = sm.is_anti(phys)
                    etype = ({(True, False): EXT_U, (True, True): EXT_VBAR,
                              (False, False): EXT_UBAR, (False, True): EXT_V})[(initial, anti)]
                mi = mass_index(f)
                ext_mass[leg] = mi
                op[0] = OP_EXT
                op[10] = mi
                op[11] = leg
                op[12] = etype
                counts["ext"] += 1
            else:
                ch = [cur[k] for k in c.children]
                for slot, k in enumerate(c.children):
                    op[2 + slot] = offset[k]
                    op[6 + slot] = hmask(cur[k].mask)
                nv = nvar(x)
                if c.op == "FFV_F":
                    ferm, vec = ch
                    op[0] = OP_FFV_F
                    op[9] = coupling_index(vec.flav, ferm.flav)
                    op[10] = mass_index(c.flav)
                    counts["ffv_f"] += 1
                    counts["var_ffv_f"] += nv
                elif c.op == "FFV_FB":
                    ferm, vec = ch
                    op[0] = OP_FFV_FB
                    op[9] = coupling_index(vec.flav, ferm.flav)
                    op[10] = mass_index(c.flav)
                    counts["ffv_fb"] += 1
                    counts["var_ffv_fb"] += nv
                elif c.op == "FFV_V":
                    row, col = ch
                    op[0] = OP_FFV_V
                    op[9] = coupling_index(c.flav, col.flav)
                    op[10] = mass_index(c.flav)
                    counts["ffv_v"] += 1
                    counts["var_ffv_v"] += nv
                elif c.op == "VVV":
                    op[0] = OP_VVV
                    counts["vvv"] += 1
                    counts["var_vvv"] += nv
                elif c.op == "VVVV":
                    op[0] = OP_VVVV
                    op[11] = c.struct
                    counts["vvvv"] += 1
                    counts["var_vvvv"] += nv
                else:
                    raise ValueError(c.op)
        else:
            t = D.terms[x]
            col, vec = cur[t.col], cur[t.vec]
            op[0] = OP_AMP
            op[2], op[3], op[4] = offset[ROOT], offset[t.col], offset[t.vec]
            op[6], op[7], op[8] = hmask(D.root_current.mask), hmask(col.mask), hmask(vec.mask)
            op[9] = coupling_index(vec.flav, col.flav)
            op[11] = len(flows) // 2
            nf = 0
            for word, coeff in sorted(t.colour.items()):
                full = complex(coeff) * (-1j)          # M = -i * (diagram value)
                fl = D_perm_index(D, word)
                key = complex(round(full.real), round(full.imag))
                if abs(full - key) > 1e-12 or key not in _PHASE:
                    raise ValueError(f"unexpected colour coefficient {coeff}")
                flows += [fl, _PHASE[key]]
                nf += 1
            op[12] = nf
            counts["amp"] += 1
            counts["amp_flows"] += nf
        ops.append(op)
        for u in set(uses(item)):
            if last[u] == pos:
                release(offset[u], blocksize(u))

    perms = _perms(D)
    C = colour_matrix(perms) if D.gluons or any(abs(sm.colour(f)) == 3 for f in D.flav_in) else [[Fraction(1)]]
    ncol_in = 1
    for p in inc:
        ncol_in *= abs(sm.colour(p)) if sm.colour(p) != 1 else 1
    ident = 1
    for p in set(out):
        ident *= math.factorial(out.count(p))
    return Program(process=" ".join(inc) + " > " + " ".join(out), npar=npar, nin=D.nin, root=D.root,
                   ops=ops, flows=flows, perms=perms, colour=C, couplings=couplings, masses=masses,
                   ext_mass=ext_mass, ws_current_doubles=top, ndiagrams=D.ndiagrams, nterms=len(D.terms),
                   average_den=4 * ncol_in * ident, flop_counts=counts)


def _perms(D):
    if not D.gluons and not any(abs(sm.colour(f)) == 3 for f in D.flav_in):
        return [()]
    return [tuple(p) for p in itertools.permutations(D.gluons)]


def D_perm_index(D, word):
    idx = getattr(D, "_perm_index", None)
    if idx is None:
        idx = D._perm_index = {p: i for i, p in enumerate(_perms(D))}
    return idx[tuple(word)]
