"""Write the built-in process programs as a C include file for the library build."""
import os

from .program import build_program

BUILTIN = [
    "e+ e- > mu+ mu-",
    "g g > t t~",
    "g g > t t~ g",
    "g g > t t~ g g",
    "g g > t t~ g g g",
    "g u~ > ta+ ta- g g u~",
]

_PARAM_ID = {"": 0, "mt": 1, "wt": 2, "mz": 3, "wz": 4, "mta": 5}
_BOSON_ID = {"g": 0, "a": 1, "z": 2}


def _arr(ctype, name, vals, per_line=16):
    vals = list(vals)
    body = []
    for i in range(0, len(vals), per_line):
        body.append("  " + ", ".join(vals[i:i + per_line]) + ",")
    if not vals:
        body.append("  0")
    return f"static const {ctype} {name}[] = {{\n" + "\n".join(body) + "\n};\n"


def emit(path):
    from . import sm
    out = ["/* generated by paper_2503_21935_gb300.gen.emit -- do not edit */\n"]
    entries = []
    for k, proc in enumerate(BUILTIN):
        P = build_program(proc)
        pre = f"mgx_p{k}"
        out.append(_arr("int32_t", pre + "_ops", (str(x) for op in P.ops for x in op)))
        out.append(_arr("int32_t", pre + "_flows", (str(x) for x in P.flows)))
        out.append(_arr("int32_t", pre + "_terms", (str(x) for x in P.terms)))
        out.append(_arr("double", pre + "_colour",
                        (repr(float(x)) for row in P.colour for x in row), per_line=8))
        spec = []
        for boson, fermion in P.couplings:
            q = sm.charge(fermion) if fermion else 0.0
            t3 = sm.t3(fermion) if fermion else 0.0
            spec += [str(_BOSON_ID[boson]), repr(q), repr(t3)]
        out.append(_arr("double", pre + "_coupl", spec, per_line=9))
        out.append(_arr("int32_t", pre + "_mass",
                        (str(_PARAM_ID[x]) for pair in P.masses for x in pair)))
        out.append(_arr("int32_t", pre + "_extmass", (str(x) for x in P.ext_mass)))
        split_init = []
        for n in (2, 4, 8):
            parts = P.splits[n]
            out.append(_arr("int32_t", f"{pre}_split{n}_ops", (str(i) for part in parts for i in part)))
            starts = [0]
            for part in parts:
                starts.append(starts[-1] + len(part))
            out.append(_arr("int32_t", f"{pre}_split{n}_start", (str(x) for x in starts)))
            split_init.append(f"{{{len(parts)}, {pre}_split{n}_ops, {pre}_split{n}_start}}")
        c = P.flop_counts
        cta = P.cta
        if cta is not None:
            out.append(_arr("int32_t", pre + "_cta_ops", (str(x) for op in cta["ops"] for x in op)))
            out.append(_arr("int32_t", pre + "_cta_flows", (str(x) for x in cta["flows"])))
            out.append(_arr("int32_t", pre + "_cta_terms", (str(x) for x in cta["terms"])))
            out.append(_arr("int32_t", pre + "_cta_items", (str(x) for x in cta["items"])))
            out.append(_arr("int32_t", pre + "_cta_steps", (str(x) for st in cta["steps"] for x in st)))
            cta_init = (f'{{{len(cta["ops"])}, {pre}_cta_ops, {len(cta["flows"]) // 2}, {pre}_cta_flows, '
                        f'{len(cta["terms"]) // 8}, {pre}_cta_terms, '
                        f'{len(cta["items"])}, {pre}_cta_items, {len(cta["steps"])}, {pre}_cta_steps, '
                        f'{cta["store"]}, {cta["chunk"]}}}')
        else:
            cta_init = "{0, nullptr, 0, nullptr, 0, nullptr, 0, nullptr, 0, nullptr, 0, 0}"
        entries.append(
            f'  {{"{P.process}", {P.npar}, {P.nin}, {P.root}, {len(P.ops)}, {pre}_ops, '
            f'{len(P.flows) // 2}, {pre}_flows, {len(P.terms) // 8}, {pre}_terms, {P.ncol}, {pre}_colour, {len(P.couplings)}, {pre}_coupl, '
            f'{len(P.masses)}, {pre}_mass, {pre}_extmass, {P.ws_current_doubles}, {P.ndiagrams}, '
            f'{P.nterms}, {P.average_den}, {P.gs_power}, {P.col_den}, {P.jamp_zero}, '
            f'{{{c["var_ffv_f"]}, {c["var_ffv_fb"]}, {c["var_ffv_v"]}, {c["var_vvv"]}, {c["var_vvvv"]}, {c["var_bil"]}, {c["var_rbil"]}, '
            f'{c["ffv_f"] + c["ffv_fb"] + c["ffv_v"] + c["vvv"] + c["vvvv"] + c["bil"] + c["rbil"]}, {c["amp_terms"]}, {c["amp_flows"]}, {c["amp"]}, {c["amp_runs"]}, {c["sum_adds"]}, {c["vvv_hdr"]}, {c["vvvv_hdr"]}, {c["slash_hdr"]}, {c["slash_pref_hdr"]}}}, '
            f'{cta_init}, {{{", ".join(split_init)}}}}},')
    out.append("static const mgx_program_desc mgx_programs[] = {\n" + "\n".join(entries) + "\n};\n")
    out.append(f"static const int mgx_num_programs = {len(BUILTIN)};\n")
    text = "\n".join(out)
    os.makedirs(os.path.dirname(path), exist_ok=True)
    old = open(path).read() if os.path.exists(path) else None
    if old != text:
        with open(path, "w") as f:
            f.write(text)
    return path


if __name__ == "__main__":
    import sys
    emit(sys.argv[1])
