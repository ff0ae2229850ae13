"""Profiling diagnostics of a spaQR factorisation, after the paper's
profiling figures (Section 4): per level the fronts and interfaces, their
sizes before and after sparsification, the decay of the CPQR pivots
|R_kk| / |R_11| that sets the ranks, and the time of each phase; across grid
sizes the factorisation time, the factor's device memory and the size of the
top separator against N.

Everything comes from the factor through the C ABI (spaqr_factor_level,
spaqr_factor_pivots, spaqr_factor_ranks, spaqr_factor_info); the plan report
comes from the ordering alone (spaqr_ordering_get).  The inputs are the
seeded synthetic matrices of synth.convdiff.

    python -m paper_2010_06807_gb300.diagnostics --kind 3d_uniform_a \\
        --sizes 16 32 48 64 --eps 1e-2 [--scaling 0] [--json out.json]

The symbolic plan alone (host only, no GPU): front and interface sizes per
level before sparsification and the atom counts, for the geometric ordering
or, with --permute SEED, the grid-free ordering of the permuted matrix:

    python -m paper_2010_06807_gb300.diagnostics --plan-only --kind 2d_lognormal \\
        --sizes 128 256 [--permute 11 [--matching max_product]]
"""
import argparse
import json
import time

import numpy as np

import paper_2010_06807_gb300 as sq

PHASES = ("factorize", "scale", "sparsify", "merge")
DECAY_AT = (1, 2, 4, 8, 16, 32, 64)


def pivot_decay(norms_list, at=DECAY_AT):
    """Median over interfaces of |R_kk| / |R_11| at step k (1-based) for
    the k in `at` that at least one interface reached; None where none did."""
    out = {}
    for k in at:
        vals = [nm[k - 1] / nm[0] for nm in norms_list if len(nm) >= k and nm[0] > 0]
        out[k] = float(np.median(vals)) if vals else None
    return out


def plan_report(ordering):
    """Host-only summary of an ordering's symbolic plan (no factorisation, no
    GPU): per level (0 = leaves) the fronts (count, sizes |s|, heights = the
    summed sizes of their row clusters) and the interfaces left after them
    (count, sizes), all before sparsification; plus the atom counts.
    Cluster sizes come from the atoms: an active cluster spans the atoms from
    its first one up to the next active cluster of the same node (the
    clusters of a node partition its atoms at every level)."""
    arr = ordering.arrays()
    atom_ptr, atom_node = arr["atom_ptr"], arr["atom_node"]
    na = atom_node.shape[0]
    node_end = {}
    for a in range(na):
        node_end[int(atom_node[a])] = a + 1
    leaf_level = int(arr["node_level"].max()) if arr["node_level"].size else 1
    sep_atoms = np.array([atom_ptr[a + 1] - atom_ptr[a] for a in range(na)
                          if arr["node_level"][atom_node[a]] < leaf_level], dtype=np.int64)
    rows = []
    for k, st in enumerate(ordering.plan()):
        cl = sorted(st["clusters"])
        size = {}
        for i, c in enumerate(cl):
            nd = int(atom_node[c])
            end = node_end[nd]
            if i + 1 < len(cl) and int(atom_node[cl[i + 1]]) == nd:
                end = cl[i + 1]
            size[c] = int(atom_ptr[end] - atom_ptr[c])
        fronts = [f["id"] for f in st["fronts"]]
        fs = set(fronts)
        s_sizes = [size[f] for f in fronts]
        heights = [sum(size[r] for r in f["R"]) for f in st["fronts"]]
        inter = [size[c] for c in cl if c not in fs]
        rows.append({"level": k, "clusters": len(cl), "n_fronts": len(fronts),
                     "front_cols": int(sum(s_sizes)), "max_front": max(s_sizes) if s_sizes else 0,
                     "max_front_rows": max(heights) if heights else 0,
                     "n_interfaces": len(inter), "interface_cols": int(sum(inter)),
                     "max_interface": max(inter) if inter else 0,
                     "median_interface": float(np.median(inter)) if inter else 0.0})
    return {"n": int(ordering.n), "levels": ordering.L, "atoms": int(na),
            "separator_atoms": int(sep_atoms.size),
            "separator_atom_median": float(np.median(sep_atoms)) if sep_atoms.size else 0.0,
            "separator_atoms_le2": int((sep_atoms <= 2).sum()), "per_level": rows}


def plan_markdown(rep, title):
    """Table of a plan_report result."""
    lines = [f"### {title}", "",
             f"N = {rep['n']}, {rep['levels']} levels, {rep['atoms']} atoms ({rep['separator_atoms']} in "
             f"separators: median {rep['separator_atom_median']:g} columns, {rep['separator_atoms_le2']} of at "
             "most 2)", "",
             "| level | clusters | fronts | front columns | largest front (rows x cols) | interfaces after |"
             " interface columns | largest / median interface |",
             "|---|---|---|---|---|---|---|---|"]
    for r in rep["per_level"]:
        lines.append(f"| {r['level']} | {r['clusters']} | {r['n_fronts']} | {r['front_cols']} | "
                     f"{r['max_front_rows']} x {r['max_front']} | {r['n_interfaces']} | {r['interface_cols']} | "
                     f"{r['max_interface']} / {r['median_interface']:g} |")
    return "\n".join(lines)


def level_report(F):
    """One dict per level (0 = leaves)."""
    info = sq.spaqr_factor_info(F)
    rows = []
    for k in range(info["nlevels"]):
        d = sq.spaqr_factor_level(F, k)
        pairs, _ = sq.spaqr_factor_ranks(F, k)
        piv = sq.spaqr_factor_pivots(F, k)
        d["level"] = k
        d["rank_fraction"] = (float(pairs[:, 1].sum()) / float(pairs[:, 0].sum())) if len(pairs) else None
        d["pivot_decay"] = pivot_decay(piv) if piv else {}
        rows.append(d)
    return rows


def factor_problem(p, eps, scaling=1, precision="fp64", skip=2, device=None):
    """Order and factor one synthetic problem on the device; returns
    (ordering, factor, csr tensors, factor wall ms by CUDA events)."""
    import torch
    dev = device or torch.device("cuda:0")
    A = [torch.from_numpy(x).to(dev) for x in (p.rowptr, p.colind, p.val)]
    o = sq.spaqr_order(p.rowptr, p.colind, p.dims)
    st = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    F = sq.spaqr_factor(o, *A, eps=eps, skip=skip, scaling=scaling, precision=precision)
    e1.record(st)
    e1.synchronize()
    return o, F, A, e0.elapsed_time(e1)


def scaling_study(kind, sizes, eps, scaling=1, precision="fp64", gmres=True, device=None, apply_rhs=0):
    """Factor time, device memory, ranks and GMRES iterations per grid side;
    with apply_rhs > 0 also the time of one application of the factor to that
    many right-hand sides (spaqr_solve; the first application warms up)."""
    import torch
    from synth.convdiff import config_problem, rhs
    dev = device or torch.device("cuda:0")
    out = []
    for n in sizes:
        p = config_problem(kind, n=n)
        # warm-up factorisation (first-call attribute setup, memory pool growth)
        _, F, _, _ = factor_problem(p, eps, scaling, precision, device=dev)
        del F
        o, F, A, ms = factor_problem(p, eps, scaling, precision, device=dev)
        info = sq.spaqr_factor_info(F)
        row = {"n_side": n, "N": p.n, "nnz": p.nnz, "levels": info["nlevels"], "factor_ms": ms,
               "factor_bytes": info["factor_bytes"], "bytes_per_unknown": info["factor_bytes"] / p.n,
               "top_separator": info["top_size"], "rank_sum": info["rank_sum"], "size_sum": info["size_sum"],
               "phase_ms": dict(zip(PHASES, info["phase_ms"])), "levels_detail": level_report(F)}
        if apply_rhs > 0:
            Bq = torch.from_numpy(np.ascontiguousarray(rhs(p, apply_rhs).T)).to(dev).T
            sq.spaqr_solve(F, Bq)
            st = torch.cuda.current_stream(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            sq.spaqr_solve(F, Bq)
            e1.record(st)
            e1.synchronize()
            row.update(apply_rhs=apply_rhs, apply_ms=e0.elapsed_time(e1))
        if gmres:
            b = torch.from_numpy(np.ascontiguousarray(rhs(p, 1).T)).to(dev).T
            t0 = time.perf_counter()
            _, it, rr, hist = sq.spaqr_gmres(F, *A, b, tol=1e-12, history=True)
            torch.cuda.synchronize(dev)
            row.update(gmres_iters=int(it[0]), gmres_relres=float(rr[0]),
                       gmres_ms=(time.perf_counter() - t0) * 1e3,
                       gmres_history=[float(x) for x in hist[0]])
        del F
        out.append(row)
    return out


def markdown(study, title):
    """Tables of a scaling_study result."""
    lines = [f"### {title}", "",
             "| side | N | levels | factor ms | MB | B/unknown | top sep. | ranks / sizes | GMRES it |",
             "|---|---|---|---|---|---|---|---|---|"]
    for r in study:
        lines.append(f"| {r['n_side']} | {r['N']} | {r['levels']} | {r['factor_ms']:.1f} | "
                     f"{r['factor_bytes'] / 2 ** 20:.0f} | {r['bytes_per_unknown']:.0f} | {r['top_separator']} | "
                     f"{r['rank_sum']} / {r['size_sum']} | {r.get('gmres_iters', '')} |")
    for r in study:
        if r.get("apply_ms") is not None:
            lines.append(f"\nside {r['n_side']}: one application to {r['apply_rhs']} right-hand sides "
                         f"{r['apply_ms']:.2f} ms")
    hist = [r for r in study if r.get("gmres_history")]
    if hist:
        lines += ["", "GMRES residual estimates ||b - A x_j|| / ||b|| (iterations 1, 2, ...):", ""]
        for r in hist:
            lines.append(f"- side {r['n_side']}: " + " ".join(f"{x:.1e}" for x in r["gmres_history"]))
    for r in study:
        lines += ["", f"Per level, side {r['n_side']} (level 0 = leaves):", "",
                  "| level | fronts | max front (rows x cols) | interfaces | max interface | size before -> after |"
                  " median \\|R_kk\\|/\\|R_11\\| at k = 1,2,4,8,16,32,64 | ms factorize / scale / sparsify / merge |",
                  "|---|---|---|---|---|---|---|---|"]
        for d in r["levels_detail"]:
            pd = {int(k): v for k, v in d["pivot_decay"].items()}   # int keys, also after a JSON round trip
            dec = " ".join("-" if pd.get(k) is None else f"{pd[k]:.1e}" for k in DECAY_AT) if pd else ""
            ph = " / ".join(f"{x:.1f}" for x in d["phase_ms"])
            lines.append(f"| {d['level']} | {d['n_fronts']} | {d['max_front_rows']} x {d['max_front_cols']} | "
                         f"{d['n_interfaces']} | {d['max_interface']} | {d['remaining_size']} -> "
                         f"{d['interface_after']} | {dec} | {ph} |")
    return "\n".join(lines)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--kind", default="3d_uniform_a")
    ap.add_argument("--sizes", type=int, nargs="+", default=[16, 32, 48, 64])
    ap.add_argument("--eps", type=float, default=1e-2)
    ap.add_argument("--scaling", type=int, default=1)
    ap.add_argument("--precision", default="fp64")
    ap.add_argument("--no-gmres", action="store_true")
    ap.add_argument("--apply-rhs", type=int, default=0, metavar="N",
                    help="also time one application of the factor to N right-hand sides")
    ap.add_argument("--json")
    ap.add_argument("--plan-only", action="store_true",
                    help="host only: the symbolic plan of each size's ordering, no factorisation")
    ap.add_argument("--permute", type=int, default=None, metavar="SEED",
                    help="with --plan-only: permute rows and columns and use the grid-free ordering")
    ap.add_argument("--matching", default="max_product", help="row matching of the grid-free ordering")
    a = ap.parse_args(argv)
    if a.plan_only:
        from synth.convdiff import config_problem, permuted
        reps = []
        for n in a.sizes:
            p = config_problem(a.kind, n=n)
            if a.permute is None:
                o = sq.spaqr_order(p.rowptr, p.colind, p.dims)
                how = "geometric ordering"
            else:
                p = permuted(p, a.permute)
                o = sq.spaqr_order(p.rowptr, p.colind, None, val=p.val, matching=a.matching)
                how = f"rows and columns permuted (seed {a.permute}), grid-free ordering, {a.matching} matching"
            rep = plan_report(o)
            reps.append(rep)
            print(plan_markdown(rep, f"{a.kind}, side {n}: {how}"))
            print()
        if a.json:
            with open(a.json, "w") as f:
                json.dump(reps, f, indent=1)
        return 0
    study = scaling_study(a.kind, a.sizes, a.eps, a.scaling, a.precision, gmres=not a.no_gmres,
                          apply_rhs=a.apply_rhs)
    if a.json:
        with open(a.json, "w") as f:
            json.dump(study, f, indent=1)
    print(markdown(study, f"{a.kind}, eps {a.eps:g}, scaling {a.scaling}, {a.precision}"))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
