"""Exact colour matrix of the quark-line flow basis by symbolic SU(N) algebra.

C_st = sum_colours conj(b_s) b_t with b_s = (T^{s1} ... T^{sn})_{ij} equals the
single trace Tr(T^{sn} ... T^{s1} T^{t1} ... T^{tn}) with every adjoint label
summed.  Labels are eliminated one at a time with the completeness relation
T^a_ij T^a_kl = 1/2 (d_il d_kj - 1/N d_ij d_kl):
  Tr(a X a Y)      = 1/2 Tr(X) Tr(Y) - 1/(2N) Tr(X Y)
  Tr(a X) Tr(a Y)  = 1/2 Tr(X Y)     - 1/(2N) Tr(X) Tr(Y)
with Tr() = N.  Results are exact Fractions.
"""
from fractions import Fraction
from functools import lru_cache
import itertools

N = 3


def _canon(traces):
    """Canonical form: relabel in order of first appearance after rotating each trace
    to its lexicographically smallest rotation, then sort traces."""
    best = None
    # small inputs: try every ordering of traces / rotation choice greedily
    def rot_min(t):
        if not t:
            return t
        return min(t[i:] + t[:i] for i in range(len(t)))
    ts = [tuple(t) for t in traces]
    for perm in itertools.permutations(range(len(ts))) if len(ts) <= 4 else [range(len(ts))]:
        relabel = {}
        out = []
        for k in perm:
            t = ts[k]
            # choose rotation after relabelling greedily: relabel with current map + fresh labels
            cands = []
            for i in range(max(1, len(t))):
                r = t[i:] + t[:i]
                m = dict(relabel)
                rr = []
                for x in r:
                    if x not in m:
                        m[x] = len(m)
                    rr.append(m[x])
                cands.append((tuple(rr), m))
            rr, m = min(cands, key=lambda z: z[0])
            relabel = m
            out.append(rr)
        key = tuple(out)
        if best is None or key < best:
            best = key
    return best


@lru_cache(maxsize=None)
def _trace_product(key):
    """Value of a product of traces (tuple of tuples of labels, each label twice)."""
    traces = [list(t) for t in key]
    # drop empty traces: Tr() = N
    val_mult = Fraction(1)
    rest = []
    for t in traces:
        if not t:
            val_mult *= N
        else:
            rest.append(t)
    if not rest:
        return val_mult
    for t in rest:
        if len(t) == 1:
            return Fraction(0)          # traceless generators
    a = rest[0][0]
    # locate the second occurrence of a
    loc = None
    for ti, t in enumerate(rest):
        for pi, x in enumerate(t):
            if x == a and not (ti == 0 and pi == 0):
                loc = (ti, pi)
                break
        if loc:
            break
    ti, pi = loc
    half = Fraction(1, 2)
    invn = Fraction(1, 2 * N)
    if ti == 0:
        t = rest[0]
        X = t[1:pi]
        Y = t[pi + 1:]
        others = rest[1:]
        v1 = _eval(others + [X, Y])
        v2 = _eval(others + [X + Y])
        return val_mult * (half * v1 - invn * v2)
    t0 = rest[0]
    t1 = rest[ti]
    X = t0[1:]
    Y = t1[pi + 1:] + t1[:pi]
    others = [t for k, t in enumerate(rest) if k not in (0, ti)]
    v1 = _eval(others + [X + Y])
    v2 = _eval(others + [X, Y])
    return val_mult * (half * v1 - invn * v2)


def _eval(traces):
    return _trace_product(_canon(traces))


def colour_matrix(perms):
    """Exact C[s][t] (list of lists of Fraction) for the flow strings `perms`."""
    n = len(perms)
    C = [[None] * n for _ in range(n)]
    for s in range(n):
        for t in range(s, n):
            word = tuple(reversed(perms[s])) + tuple(perms[t])
            v = _eval([list(word)]) if perms[s] or perms[t] else Fraction(N)
            C[s][t] = C[t][s] = v
    return C
