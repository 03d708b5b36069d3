"""Emit the op table ("program") executed by the generic CUDA amplitude kernel.

One program per process.  Each op is 16 int32 fields:
  0 code  1 dst  2 a  3 b  4 c  5 mask_dst  6 mask_a  7 mask_b  8 mask_c
  9 coupling  10 mass/width entry  11 aux  12 aux2  13..15 variant bases of children a, b, c
Offsets (fields 1-4) are in doubles inside a per-event workspace block:
  block = [k0 k1 k2 k3 | variant 0: 4 complex | variant 1 | ...]
where k is the current's incoming momentum and variant v holds the current for
the helicities pdep(v, mask) of the legs in `mask` (leg p <-> bit npar-1-p, the
bit of the canonical helicity index).  A current is computed once per helicity
state of its own legs (helicity recycling) and its block is freed after its last
use.  Every diagram term is closed at the root vertex through a root bilinear (column
Q.V or row R.psi, chosen by an exact minimum vertex cover); terms with one colour
vector up to a phase form a group; terms of a group sharing a bilinear form a run
whose other operands are summed by a SUM op (once per helicity state of their legs).
AMP ops take one product per run and good helicity and add the group amplitude,
times a phase in {1, i, -1, -i}, to the group's colour flows.  Where it is cheaper, the
single-run groups of one bilinear are closed flow-major instead: one summed current per colour
flow they reach and one AMP op per flow (see _flow_major_bilinears).
"""
import itertools
import math
from dataclasses import dataclass, field
from fractions import Fraction

from . import sm
from .colour import colour_matrix
from .diagrams import Diagrams, Current

OP_EXT, OP_FFV_F, OP_FFV_FB, OP_FFV_V, OP_VVV, OP_VVVV, OP_AMP, OP_BIL, OP_RBIL, OP_SUM = 1, 2, 3, 4, 5, 6, 7, 8, 9, 10
EXT_U, EXT_V, EXT_UBAR, EXT_VBAR, EXT_EPS_IN, EXT_EPS_OUT = 0, 1, 2, 3, 4, 5
NFIELD = 16
FLOW_FIRST = 4                  # flow entry phase-code bit: first update of that flow (write, not add)
CHILD_HEADER = ("VVV", "VVVV", "FFV_F", "FFV_FB", "RBIL")   # headers that read child variants

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
    flows: list                 # flattened (flow, phase code) pairs of the AMP groups
    terms: list                 # flattened 8-int term entries of the AMP groups
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


HEADER = {"EXT": 4, "FFV_F": 6, "FFV_FB": 6, "FFV_V": 6, "VVV": 18, "VVVV": 6, "BIL": 6, "RBIL": 6, "SUM": 0}
# float64 instructions per variant of the two root bilinears (column: Q = psibar gamma psi_col;
# row: R = psibar Vslash), used to choose between them
BIL_COST = {"BIL": 56, "RBIL": 40}
SMEM_STORE_BUDGET = 96 * 1024     # bytes of shared memory for one event's current store


class _Allocator:
    """First-fit allocator over a linear range of doubles; frees merge with neighbours."""

    def __init__(self):
        self.free = []
        self.top = 0

    def alloc(self, size):
        for k, (s, z) in enumerate(self.free):
            if z >= size:
                if z == size:
                    self.free.pop(k)
                else:
                    self.free[k] = (s + size, z - size)
                return s
        s = self.top
        self.top += size
        return s

    def release(self, s, size):
        self.free.append((s, size))
        self.free.sort()
        merged = []
        for a, z in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + z)
            else:
                merged.append((a, z))
        self.free = merged


class _Builder:
    """Common encoding of ops for both schedules."""

    def __init__(self, D):
        self.D = D
        self.npar = D.npar
        self.masses = [("", "")]
        self.couplings = []
        self.ext_mass = [0] * D.npar
        self.ROOT = D.root_current.id
        self._add_bilinears()

    def _add_bilinears(self):
        """Close every diagram term at the root vertex through a bilinear.  A term (column current C,
        vector current V) is psibar_root Vslash (cL PL + cR PR) psi_C; it is evaluated either as
        Q_C . V with the column bilinear Q_C^mu = psibar gamma^mu (..) psi_C (one per C and coupling,
        2^(1+|C|) variants) or as R_V . psi_C with the row bilinear R_V = psibar Vslash (..) (one per V
        and coupling, 2^(1+|V|) variants).  The set of bilinears is a minimum-weight vertex cover of
        the bipartite (C, V) graph of the terms (exact, by max-flow / min-cut), so the cheaper side
        is built wherever a current is shared by many terms."""
        D = self.D
        nb = lambda m: bin(m).count("1")
        info = []
        for t in D.terms:
            col, vec = D.currents[t.col], D.currents[t.vec]
            info.append((t, (t.col, self.coupling_index(vec.flav, col.flav)), (t.vec, self.coupling_index(vec.flav, col.flav))))
        Cs = sorted({c for _, c, _ in info})
        Vs = sorted({v for _, _, v in info})
        wC = {c: BIL_COST["BIL"] * 2 ** (1 + nb(D.currents[c[0]].mask)) for c in Cs}
        wV = {v: BIL_COST["RBIL"] * 2 ** (1 + nb(D.currents[v[0]].mask)) for v in Vs}
        cover_C, cover_V = _bipartite_min_cover(Cs, Vs, {(c, v) for _, c, v in info}, wC, wV)
        made = {}
        for t, c, v in info:
            if c in cover_C:
                key, kind, other = ("BIL", c), "BIL", t.vec
            else:
                key, kind, other = ("RBIL", v), "RBIL", t.col
            if key not in made:
                src = t.col if kind == "BIL" else t.vec
                node = Current(len(D.currents), D.root_current.mask | D.currents[src].mask, kind, kind,
                               children=(self.ROOT, src))
                node.cpl = key[1][1]
                D.currents.append(node)
                made[key] = node.id
            t.bil = made[key]
            t.other = other
            t.kind = 0 if kind == "BIL" else 1

    def hmask(self, m):
        return sum(_bit(self.npar, p) for p in range(self.npar) if m >> p & 1)

    def mass_index(self, flav):
        key = (sm.mass_param(flav), sm.width_param(flav))
        if key == ("", ""):
            return 0
        if key not in self.masses:
            self.masses.append(key)
        return self.masses.index(key)

    def coupling_index(self, boson, fermion):
        base = fermion if not sm.is_anti(fermion) else sm.anti(fermion)
        spec = (boson, base if boson != "g" else "")
        if spec not in self.couplings:
            self.couplings.append(spec)
        return self.couplings.index(spec)

    def cur(self, i):
        return self.D.currents[i]

    def nvar(self, i):
        return 1 << bin(self.cur(i).mask).count("1")

    # VVVV colour structures: the two child pairs whose dot products each one needs
    VVVV_PAIRS = {0: ((0, 2), (1, 2)), 1: ((0, 1), (1, 2)), 2: ((0, 1), (0, 2))}

    def header(self, i):
        """Header slots of current i.  VVV and VVVV headers also hold, per event, the dot
        products that depend on only one child (VVV: (k-combination . e) per child variant) or one
        pair of children (VVVV: e_x . e_y per pair of variants), and fermion-vector vertices hold
        the slash blocks of each variant of their vector child, so that the variants, which
        range over all children's helicities, do not recompute them."""
        c = self.cur(i)
        h = HEADER[c.op]
        if c.op in ("FFV_F", "FFV_FB", "RBIL"):
            h += 8 * self.nvar(c.children[1])          # slash blocks per vector variant
        elif c.op == "VVV":
            h += 2 * (self.nvar(c.children[0]) + self.nvar(c.children[1]))
        elif c.op == "VVVV":
            for x, y in self.VVVV_PAIRS[c.struct]:
                h += 2 * self.nvar(c.children[x]) * self.nvar(c.children[y])
        return h

    def blocksize(self, i):
        return self.header(i) + 8 * self.nvar(i)

    def varbase(self, i, offset):
        return offset[i] + self.header(i)

    def current_row(self, i, offset, terms=None):
        D = self.D
        c = self.cur(i)
        op = [0] * NFIELD
        op[1] = offset[i]
        op[5] = self.hmask(c.mask)
        if c.op == "SUM":
            # sum of phased currents over the same legs: list entries (base, mask, -, -, phase, ...)
            # in the term table; variant v of every summand is its variant v
            op[0], op[11], op[12] = OP_SUM, len(terms) // 8, len(c.children)
            for k, ph in zip(c.children, c.phases):
                terms += [self.varbase(k, offset), self.hmask(D.currents[k].mask), 0, 0, ph, 0, 0, 0]
            return op
        if c.op == "EXT":
            leg = c.leg
            f = c.flav
            initial = leg < D.nin
            if sm.kind(f) == "V":
                etype = EXT_EPS_IN if initial else EXT_EPS_OUT
            else:
                phys = D.incoming[leg] if initial else D.outgoing[leg - D.nin]
                anti = sm.is_anti(phys)
                etype = ({(True, False): EXT_U, (True, True): EXT_VBAR,
                          (False, False): EXT_UBAR, (False, True): EXT_V})[(initial, anti)]
            mi = self.mass_index(f)
            self.ext_mass[leg] = mi
            op[0], op[10], op[11], op[12] = OP_EXT, mi, leg, etype
            return op
        ch = [D.currents[k] for k in c.children]
        for slot, k in enumerate(c.children):
            op[2 + slot] = offset[k]
            op[6 + slot] = self.hmask(D.currents[k].mask)
            op[13 + slot] = self.varbase(k, offset)
        if c.op == "FFV_F":
            op[0], op[9], op[10] = OP_FFV_F, self.coupling_index(ch[1].flav, ch[0].flav), self.mass_index(c.flav)
        elif c.op == "FFV_FB":
            op[0], op[9], op[10] = OP_FFV_FB, self.coupling_index(ch[1].flav, ch[0].flav), self.mass_index(c.flav)
        elif c.op == "FFV_V":
            op[0], op[9], op[10] = OP_FFV_V, self.coupling_index(c.flav, ch[1].flav), self.mass_index(c.flav)
        elif c.op == "VVV":
            op[0] = OP_VVV
        elif c.op == "VVVV":
            op[0], op[11] = OP_VVVV, c.struct
        elif c.op == "BIL":
            op[0], op[9] = OP_BIL, c.cpl
        elif c.op == "RBIL":
            op[0], op[9] = OP_RBIL, c.cpl
        else:
            raise ValueError(c.op)
        return op

    def amp_row(self, runs, fl, offset, flows, terms):
        """One AMP row per term group: term table entries (bil base, bil mask, other base, other mask,
        phase, kind, run start, run end) and the group's (flow, phase) list.  `runs` lists
        (bilinear, kind, [(other current, phase), ...]): terms closing on the same bilinear, whose
        phased other operands the kernel sums first and closes with one product (distributivity)."""
        op = [0] * NFIELD
        op[0] = OP_AMP
        op[11] = len(terms) // 8
        op[12] = sum(len(items) for _, _, items in runs)
        for x, kind, items in runs:
            for k, (y, ph) in enumerate(items):
                terms += [self.varbase(x, offset), self.hmask(self.cur(x).mask), self.varbase(y, offset),
                          self.hmask(self.cur(y).mask), ph, kind, int(k == 0), int(k == len(items) - 1)]
        op[9] = len(flows) // 2
        op[10] = len(fl)
        for f, ph in fl:
            flows += [f, ph]
        return op


def _runs(D, group):
    """The group's terms as runs: (bilinear, kind, [(other current, phase), ...]) per bilinear."""
    tis, phases, _ = group
    out = {}
    for ti, ph in zip(tis, phases):
        t = D.terms[ti]
        out.setdefault((t.bil, t.kind), []).append((t.other, ph))
    return [(x, kind, items) for (x, kind), items in sorted(out.items())]


def _bipartite_min_cover(left, right, edges, wl, wr):
    """Minimum-weight vertex cover of a bipartite graph (every edge needs one endpoint chosen):
    the source side of a minimum s-t cut with capacities wl (source -> left), wr (right -> sink)
    and infinite left -> right edges (Konig / max-flow min-cut).  Edmonds-Karp max flow."""
    import collections
    S, T = ("s",), ("t",)
    cap = collections.defaultdict(float)
    adj = collections.defaultdict(set)

    def link(a, b, c):
        cap[(a, b)] += c
        adj[a].add(b)
        adj[b].add(a)
    inf = float("inf")
    for x in left:
        link(S, ("L", x), wl[x])
    for y in right:
        link(("R", y), T, wr[y])
    for x, y in edges:
        link(("L", x), ("R", y), inf)
    while True:
        parent = {S: None}
        q = collections.deque([S])
        while q and T not in parent:
            u = q.popleft()
            for w in adj[u]:
                if w not in parent and cap[(u, w)] > 0:
                    parent[w] = u
                    q.append(w)
        if T not in parent:
            break
        f, w = inf, T
        while parent[w] is not None:
            f = min(f, cap[(parent[w], w)])
            w = parent[w]
        w = T
        while parent[w] is not None:
            cap[(parent[w], w)] -= f
            cap[(w, parent[w])] += f
            w = parent[w]
    reach = set(parent)          # residual-reachable from the source after the last search
    cover_left = {x for x in left if ("L", x) not in reach}
    cover_right = {y for y in right if ("R", y) in reach}
    for x, y in edges:
        if x not in cover_left and y not in cover_right:
            raise RuntimeError("vertex cover does not cover every term")
    return cover_left, cover_right


def _term_groups(D):
    """Group diagram terms whose colour vectors agree up to a phase in {1, i, -1, -i}: a group's
    terms are summed with their phases first and the sum is added to the flows once.
    Returns [(terms, [(phase code per term)], [(flow, phase code)])] in first-occurrence order."""
    groups = {}
    order = []
    for ti, t in enumerate(D.terms):
        items = sorted(t.colour.items())
        c0 = complex(items[0][1])
        key = tuple((w, complex(c) / c0) for w, c in items)
        if key not in groups:
            groups[key] = []
            order.append(key)
        groups[key].append((ti, c0 * (-1j)))          # M = -i * (diagram value)
    out = []
    for key in order:
        phases = []
        for ti, ph in groups[key]:
            k = complex(round(ph.real), round(ph.imag))
            if abs(ph - k) > 1e-12 or k not in _PHASE:
                raise ValueError(f"unexpected colour coefficient {ph}")
            phases.append(_PHASE[k])
        fl = []
        for w, r in key:
            k = complex(round(r.real), round(r.imag))
            if abs(r - k) > 1e-12 or k not in _PHASE:
                raise ValueError(f"unexpected colour ratio {r}")
            fl.append((D_perm_index(D, w), _PHASE[k]))
        out.append(([ti for ti, _ in groups[key]], phases, fl))
    return out


def _closure(D, ti):
    out = set()
    st = [D.terms[ti].bil, D.terms[ti].other]
    while st:
        x = st.pop()
        if x in out:
            continue
        out.add(x)
        st.extend(D.currents[x].children)
    return out


def _flow_major_bilinears(B, groups, gruns):
    """Bilinears whose single-run groups are cheaper closed flow by flow.  Group-major (the default)
    costs, per good helicity, one product X . Y_g per group plus a jamp add per (group, flow);
    flow-major costs one product and one jamp add per colour flow the groups reach and helicity,
    plus, per helicity state of the other legs, a 4-vector add per further (group, flow) entry to
    form the flow's summed current.  A bilinear shared by many groups that reach few flows
    (a row bilinear over the root and one gluon: 15 groups on 6 flows in g g > t t~ g g) gains.
    Costs are float64 instructions of the kernels with 2^npar helicities.  Returns {(X, kind):
    [group indices]} for the bilinears to close flow-major."""
    nhel = 1 << B.npar
    byx = {}
    for gi, eff in enumerate(gruns):
        if len(eff) == 1 and len(eff[0][2]) == 1:
            byx.setdefault(eff[0][:2], []).append(gi)
    out = {}
    for key, gis in byx.items():
        nvar_y = B.nvar(gruns[gis[0]][0][2][0][0])
        entries = sum(len(groups[g][2]) for g in gis)
        nflows = len({f for g in gis for f, _ in groups[g][2]})
        group_major = nhel * (16 * len(gis) + 2 * entries)
        flow_major = nhel * 18 * nflows + 8 * nvar_y * (entries - nflows)
        if flow_major < group_major:
            out[key] = gis
    return out


def _dfs_schedule(B):
    """Thread-per-event schedule: ops in depth-first order, blocks freed after last use."""
    D = B.D
    cur = D.currents
    ROOT = B.ROOT
    order = [("C", ROOT)]
    done = {ROOT}

    def emit(i):
        if i in done:
            return
        for k in cur[i].children:
            emit(k)
        done.add(i)
        order.append(("C", i))
    groups = _term_groups(D)

    def sum_node(items):
        mask = cur[items[0][0]].mask
        if any(cur[y].mask != mask for y, _ in items):
            raise ValueError("summands cover different legs")
        node = Current(len(cur), mask, cur[items[0][0]].flav, "SUM", children=tuple(y for y, _ in items))
        node.phases = [ph for _, ph in items]
        cur.append(node)
        return node.id
    # a run of several terms closing on one bilinear gets a sum current: the phased sum of its
    # other operands (all over the same legs), computed once per helicity state of those legs
    # instead of once per full helicity inside the amplitude row
    gruns = []
    for g in groups:
        gruns.append([(x, kind, [(sum_node(items), 0)] if len(items) > 1 else items)
                      for x, kind, items in _runs(D, g)])
    flow_major = _flow_major_bilinears(B, groups, gruns)
    amps = []                       # (runs, flows) of each AMP row
    handled = set()
    for gi, g in enumerate(groups):
        if gi in handled:
            continue
        eff = gruns[gi]
        key = eff[0][:2] if len(eff) == 1 else None
        if key in flow_major:
            # flow-major closure of every single-run group on this bilinear X: per colour flow f,
            # T_f = sum over the groups g entering f of (flow phase x term phase) Y_g, a current
            # over the legs X does not cover (once per helicity state of those legs), then one
            # product X . T_f per good helicity into flow f alone.  The Y_g are made first, then
            # every T_f (one sum op per flow), then the products.
            x, kind = key
            gis = flow_major[key]
            handled.update(gis)
            emit(x)
            per_flow = {}
            for gj in gis:
                ((_, _, ((y, ph),)),) = gruns[gj]
                emit(y)
                for f, fph in groups[gj][2]:
                    per_flow.setdefault(f, []).append((y, (ph + fph) % 4))
            for f, items in per_flow.items():
                if len(items) > 1:
                    t = sum_node(items)
                    emit(t)
                    items = [(t, 0)]
                amps.append(([(x, kind, items)], [(f, 0)]))
                order.append(("A", len(amps) - 1))
            continue
        for x, _, items in eff:
            emit(x)
            for y, _ in items:
                emit(y)
        amps.append((eff, g[2]))
        order.append(("A", len(amps) - 1))

    def uses(item):
        kind, x = item
        if kind == "C":
            return list(cur[x].children)
        out = []
        for b, _, items in amps[x][0]:
            out += [b] + [y for y, _ in items]
        return out
    last = {}
    for pos, item in enumerate(order):
        for u in uses(item):
            last[u] = pos
    A = _Allocator()
    offset = {}
    ops, flows, terms = [], [], []
    for pos, item in enumerate(order):
        kind, x = item
        if kind == "C":
            offset[x] = A.alloc(B.blocksize(x))
            ops.append(B.current_row(x, offset, terms))
        else:
            ops.append(B.amp_row(amps[x][0], amps[x][1], offset, flows, terms))
        for u in set(uses(item)):
            if last[u] == pos:
                A.release(offset[u], B.blocksize(u))
    # the first update of each flow in program order writes instead of adding (phase code bit 2),
    # so the jamps need no zeroing beforehand; a flow that no group updates stays unwritten, in
    # which case every jamp is zeroed first (flag returned with the tables)
    seen = set()
    for op in ops:
        if op[0] != OP_AMP:
            continue
        for k in range(op[9], op[9] + op[10]):
            if flows[2 * k] not in seen:
                seen.add(flows[2 * k])
                flows[2 * k + 1] |= FLOW_FIRST
    B.all_flows_written = len(seen) == len(B.D_perms)
    # positions of the ops each op reads (children of a current; bilinears and other operands of a
    # group), for the diagram split
    pos_of = {x: pos for pos, (kind, x) in enumerate(order) if kind == "C"}
    deps = [sorted({pos_of[u] for u in uses(item)}) for item in order]
    return ops, flows, terms, A.top, deps


# float64 instructions per variant of each current kind (the work model of the roofline), and per
# helicity of an amplitude group: one closing product per run and an add per flow
_VAR_COST = {OP_EXT: 24, OP_FFV_F: 64, OP_FFV_FB: 64, OP_FFV_V: 72, OP_VVV: 56, OP_VVVV: 32, OP_BIL: 56, OP_RBIL: 32}


def _op_cost(op, nhel):
    if op[0] == OP_AMP:
        return nhel * (16 * op[12] + 2 * op[10])
    w = _VAR_COST.get(op[0], 8 * max(0, op[12] - 1))        # OP_SUM: a 4-vector add per further summand
    return w << bin(op[5]).count("1")


def _diagram_parts(ops, deps, nparts, nhel):
    """Diagram split: the amplitude groups, in program order, cut into at most `nparts` contiguous
    segments; each part is its groups plus every op they need (closure over the ops they read), in
    program order.  The cut minimises the largest part's cost (binary search on a cap with a greedy
    sweep).  Executing a part's ops in program order is valid with the thread program's block
    offsets: a block is reused only after the last op that reads it, and a part holds every reader
    it needs.  Returns the op positions of each part."""
    cost = [_op_cost(op, nhel) for op in ops]
    clos = {}

    def closure(i):
        if i not in clos:
            out = {i}
            for d in deps[i]:
                out |= closure(d)
            clos[i] = out
        return clos[i]
    amps = [i for i, op in enumerate(ops) if op[0] == OP_AMP]

    def sweep(cap):
        parts, cur, c = [], set(), 0
        for a in amps:
            new = cur | closure(a)
            cn = sum(cost[i] for i in new)
            if cur and cn > cap:
                parts.append(cur)
                cur = set(closure(a))
            else:
                cur = new
        parts.append(cur)
        return parts
    lo = max(sum(cost[i] for i in closure(a)) for a in amps)
    hi = sum(cost)
    while lo < hi:
        mid = (lo + hi) // 2
        if len(sweep(mid)) <= nparts:
            hi = mid
        else:
            lo = mid + 1
    return [sorted(p) for p in sweep(lo)]


def _wave_schedule(B, chunk):
    """CTA-per-event schedule: terms in chunks; each chunk computes the currents it still
    needs level by level in waves of independent (current, variant) items, then closes its
    terms.  Returns (ops, flows, items, steps, store_doubles)."""
    D = B.D
    cur = D.currents
    ROOT = B.ROOT
    level = {}

    def lv(i):
        if i not in level:
            c = cur[i]
            level[i] = 0 if c.op == "EXT" else 1 + max(lv(k) for k in c.children)
        return level[i]
    
    groups = _term_groups(D)
    chunks = []                       # lists of group indices holding about `chunk` terms
    cur_chunk, nt = [], 0
    for gi, g in enumerate(groups):
        cur_chunk.append(gi)
        nt += len(g[0])
        if nt >= chunk:
            chunks.append(cur_chunk)
            cur_chunk, nt = [], 0
    if cur_chunk:
        chunks.append(cur_chunk)
    gneed = [set().union(*[_closure(D, ti) for ti in g[0]]) for g in groups]
    last_chunk = {ROOT: len(chunks) - 1}
    for ci, ch in enumerate(chunks):
        for gi in ch:
            for x in gneed[gi]:
                last_chunk[x] = ci
    A = _Allocator()
    offset = {}
    row_of = {}
    ops, flows, items, steps, terms = [], [], [], [], []
    done = set()
    live = set()
    for ci, ch in enumerate(chunks):
        want = set().union(*[gneed[gi] for gi in ch]) - done
        if ci == 0:
            want.add(ROOT)
        for x in sorted(want, key=lambda i: (lv(i), i)):
            offset[x] = A.alloc(B.blocksize(x))
            live.add(x)
        for x in sorted(want, key=lambda i: (lv(i), i)):
            row_of[x] = len(ops)
            ops.append(B.current_row(x, offset))
        bylev = {}
        for x in want:
            bylev.setdefault(lv(x), []).append(x)
        if bylev:
            lo, hi = min(bylev), max(bylev)
            waves = [[(row_of[x], 255) for x in sorted(bylev.get(lo, []))]]
            for l in range(lo, hi + 1):
                w = []
                for x in sorted(bylev.get(l, []), key=lambda i: (cur[i].op, i)):
                    w += [(row_of[x], v) for v in range(B.nvar(x))]
                # headers of the next level; headers that read their children's variants (dot
                # products, slash blocks) wait for a wave of their own
                nxt = sorted(bylev.get(l + 1, []))
                w += [(row_of[x], 255) for x in nxt if cur[x].op not in CHILD_HEADER]
                waves.append(w)
                waves.append([(row_of[x], 255) for x in nxt if cur[x].op in CHILD_HEADER])
            for w in waves:
                if w:
                    steps.append((0, len(items), len(w)))
                    items.extend((r << 8) | v for r, v in w)
        done |= want
        first = len(ops)
        for gi in ch:
            ops.append(B.amp_row(_runs(D, groups[gi]), groups[gi][2], offset, flows, terms))
        steps.append((1, first, len(ch)))
        for x in list(live):
            if last_chunk[x] == ci:
                A.release(offset[x], B.blocksize(x))
                live.discard(x)
    return ops, flows, terms, items, steps, A.top


def gs_power(D):
    """Power of g_s carried by every tree amplitude of the process (one per q q g or g g g
    vertex, two per g g g g vertex); all diagram terms of a process share it, so the kernel
    evaluates the vertices with g_s = 1 and multiplies |M|^2 by g_s^(2p) = (4 pi alpha_s)^p."""
    cur = D.currents

    def gp(i):
        c = cur[i]
        if c.op == "EXT":
            return 0
        own = {"VVV": 1, "VVVV": 2}.get(c.op, 0)
        if c.op in ("FFV_F", "FFV_FB", "FFV_V"):
            own = 1 if any(cur[k].flav == "g" for k in c.children) or c.flav == "g" else 0
        return own + sum(gp(k) for k in c.children)
    powers = {gp(t.col) + gp(t.vec) + (1 if cur[t.vec].flav == "g" else 0) for t in D.terms}
    if len(powers) != 1:
        raise ValueError(f"diagram terms carry different powers of g_s: {powers}")
    return powers.pop()


def build_program(process, smem_budget=SMEM_STORE_BUDGET):
    lhs, rhs = process.split(">")
    inc, out = lhs.split(), rhs.split()
    D = Diagrams(inc, out)
    gsp = gs_power(D)
    npar = D.npar
    B = _Builder(D)
    B.D_perms = _perms(D)
    ops, flows, terms, top, deps = _dfs_schedule(B)
    counts = dict(ext=0, ffv_f=0, ffv_fb=0, ffv_v=0, vvv=0, vvvv=0, bil=0, rbil=0, amp=0, amp_flows=0,
                  var_ffv_f=0, var_ffv_fb=0, var_ffv_v=0, var_vvv=0, var_vvvv=0, var_bil=0, var_rbil=0)
    name = {OP_EXT: "ext", OP_FFV_F: "ffv_f", OP_FFV_FB: "ffv_fb", OP_FFV_V: "ffv_v", OP_VVV: "vvv",
            OP_VVVV: "vvvv", OP_AMP: "amp", OP_BIL: "bil", OP_RBIL: "rbil", OP_SUM: "sum"}
    counts["sum"] = counts["sum_adds"] = counts["vvv_hdr"] = counts["vvvv_hdr"] = counts["slash_hdr"] = 0
    counts["slash_pref_hdr"] = 0
    for op in ops:
        k = name[op[0]]
        counts[k] += 1
        if op[0] == OP_AMP:
            counts["amp_flows"] += op[10]
            counts["amp_terms"] = counts.get("amp_terms", 0) + op[12]
            counts["amp_runs"] = counts.get("amp_runs", 0) + sum(terms[8 * (op[11] + k) + 6] for k in range(op[12]))
        elif op[0] == OP_SUM:
            counts["sum_adds"] += (op[12] - 1) << bin(op[5]).count("1")     # 4-vector adds
        elif op[0] != OP_EXT:
            counts["var_" + k] += 1 << bin(op[5]).count("1")
        if op[0] in (OP_FFV_F, OP_FFV_FB, OP_RBIL):
            counts["slash_hdr"] += 1 << bin(op[7]).count("1")
        if op[0] in (OP_FFV_F, OP_FFV_FB):
            counts["slash_pref_hdr"] += 1 << bin(op[7]).count("1")
        if op[0] == OP_VVV:
            counts["vvv_hdr"] += (1 << bin(op[6]).count("1")) + (1 << bin(op[7]).count("1"))
        elif op[0] == OP_VVVV:
            nv = [1 << bin(op[6 + j]).count("1") for j in range(3)]
            counts["vvvv_hdr"] += sum(nv[x] * nv[y] for x, y in _Builder.VVVV_PAIRS[op[11]])
    # CTA schedule: largest chunk whose store fits the shared-memory budget
    cta = None
    nterm = len(D.terms)
    for chunk in sorted({min(nterm, c) for c in (8, 16, 24, 32, 48, 64, 96, 128, 192, 256, nterm)}, reverse=True):
        res = _wave_schedule(B, chunk)   # same builder: coupling/mass indices shared
        if res[5] * 8 <= smem_budget:
            cta = dict(zip(("ops", "flows", "terms", "items", "steps", "store"), res), chunk=chunk)
            break
    perms = _perms(D)
    C = colour_matrix(perms) if D.gluons or any(abs(sm.colour(f)) == 3 for f in D.flav_in) else [[Fraction(1)]]
    ncol_in = 1
    for p in inc:
        ncol_in *= abs(sm.colour(p)) if sm.colour(p) != 1 else 1
    ident = 1
    for p in set(out):
        ident *= math.factorial(out.count(p))
    prog = Program(process=" ".join(inc) + " > " + " ".join(out), npar=npar, nin=D.nin, root=D.root,
                   ops=ops, flows=flows, terms=terms, perms=perms, colour=C, couplings=B.couplings, masses=B.masses,
                   ext_mass=B.ext_mass, ws_current_doubles=top, ndiagrams=D.ndiagrams, nterms=len(D.terms),
                   average_den=4 * ncol_in * ident, flop_counts=counts)
    prog.cta = cta
    prog.deps = deps
    # diagram splits into 2, 4 and 8 parts (fewer when the program has fewer amplitude groups)
    prog.splits = {n: _diagram_parts(ops, deps, n, 1 << npar) for n in (2, 4, 8)}
    prog.gs_power = gsp
    prog.jamp_zero = 0 if B.all_flows_written else 1
    # integer scaling of the colour matrix for the tensor-core colour sum (exact in tf32)
    den = 1
    for row in C:
        for x in row:
            den = math.lcm(den, Fraction(x).denominator)
    for row in C:
        for x in row:
            v = abs(int(x * den))
            while v and v % 2 == 0:
                v //= 2
            if v.bit_length() > 11:
                raise ValueError("scaled colour matrix not exact in tf32")
    prog.col_den = den
    return prog


def _perms(D):
    if not D.gluons and not any(abs(sm.colour(f)) == 3 for f in D.flav_in):
        return [()]
    return [tuple(p) for p in itertools.permutations(D.gluons)]


def D_perm_index(D, word):
    idx = getattr(D, "_perm_index", None)
    if idx is None:
        idx = D._perm_index = {p: i for i, p in enumerate(_perms(D))}
    return idx[tuple(word)]
