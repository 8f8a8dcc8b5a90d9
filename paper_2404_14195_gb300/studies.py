"""Parameter studies of the paper around the two solvers: the porosity sweep
(section "Permeability and drag coefficient for various porosities"), the
node-placement spread over seeds ("Node placement sensitivity"), the
refinement-parameter and stencil-size studies ("Influence of the refinement
parameters and the stencil size", Eq. refinement_error) and the grid
convergence index of the appendix (Eqs. gci_convergence_study,
relative_error_convergence_study, pairwise_relative_error_convergence_study).

Orchestration only: every solve runs through `crossval.cross_validate` or
`crossval.run_to_steady` in the library's kernels; the host evaluates the
scalar formulas of the studies.
"""
from __future__ import annotations

import time

import numpy as np

from . import RBF_FP32, RBF_FP32C, RBF_FP32R, RBF_FP64, RbfError
from . import crossval

# the radii of the paper's porosity sweep run over r in [0.04, 0.69]
SWEEP_RADII = (0.04, 0.062, 0.1, 0.15, 0.2, 0.25, 0.3, 0.35, 0.4, 0.45, 0.49, 0.55, 0.6, 0.6526, 0.69)


# ---------------------------------------------------------------- GCI
def apparent_order(h, X, h_ref: float | None = None) -> float:
    """p_X of the appendix: slope of the least-squares line through
    (log h, log e_X(h)) with e_X(h) = |X(h) - X(h_ref)| / X(h_ref) (Eq.
    relative_error_convergence_study), h_ref the finest h by default; the point
    h_ref itself (e = 0) is left out."""
    h = np.asarray(h, np.float64)
    X = np.asarray(X, np.float64)
    iref = int(np.argmin(h)) if h_ref is None else int(np.nonzero(h == h_ref)[0][0])
    e = np.abs(X - X[iref]) / abs(X[iref])
    use = (np.arange(len(h)) != iref) & (e > 0)
    if use.sum() < 2:
        raise ValueError("apparent_order needs two coarser points with a nonzero error")
    slope, _ = np.polyfit(np.log(h[use]), np.log(e[use]), 1)
    return float(slope)


def gci(h, X, F_s: float = 1.3, h_ref: float | None = None, p: float | None = None):
    """Grid convergence index of Eq. gci_convergence_study for every pair of
    successive discretisations, assigned to the finer one of the pair:
    GCI = F_s |eps| / (r^p - 1), eps = |X_coarser - X_finer| / X_finer (Eq.
    pairwise_relative_error_convergence_study), r = h_coarser / h_finer > 1, p
    from apparent_order unless given.  Returns (p, {h_finer: GCI})."""
    h = np.asarray(h, np.float64)
    X = np.asarray(X, np.float64)
    o = np.argsort(-h)  # coarse to fine
    h, X = h[o], X[o]
    if p is None:
        p = apparent_order(h, X, h_ref)
    out = {}
    for i in range(1, len(h)):
        r = h[i - 1] / h[i]
        eps = abs(X[i - 1] - X[i]) / abs(X[i])
        out[float(h[i])] = F_s * eps / (r ** p - 1.0)
    return p, out


def refinement_error(K, K_ref) -> float:
    """E of Eq. refinement_error: |K - K_ref| / K_ref, K_ref the value on the
    uniform discretisation (h_max / h_min = 1)."""
    return abs(K - K_ref) / abs(K_ref)


# ---------------------------------------------------------------- ranks
def dist_env():
    """(dist or None, rank, world size, local rank) from the torchrun environment.
    With more than one rank, a gloo process group carries the results to every
    rank; the solves themselves share nothing (one independent cell per run)."""
    import os
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1, 0
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group("gloo")
    return dist, dist.get_rank(), ws, int(os.environ.get("LOCAL_RANK", "0"))


# where each finished run is appended as one JSON line (set by main's --progress), so
# that a long study that is stopped keeps the runs it finished
PROGRESS_PATH = None


def _record(i, item, result):
    if PROGRESS_PATH is None:
        return
    import json
    with open(PROGRESS_PATH, "a") as f:
        f.write(json.dumps(crossval._jsonable(dict(index=i, item=item, result=result))) + "\n")


def run_sharded(fn, items, dist=None, rank: int = 0, world: int = 1):
    """fn(item) for the items i with i % world == rank, then every rank gets all
    results in item order (all_gather_object of the per-rank lists)."""
    mine = []
    for i, x in enumerate(items):
        if i % world == rank:
            mine.append((i, fn(x)))
            _record(i, x, mine[-1][1])
    if dist is None or world == 1:
        return [r for _, r in mine]
    parts = [None] * world
    dist.all_gather_object(parts, mine)
    merged = sorted((p for part in parts for p in part), key=lambda p: p[0])
    return [r for _, r in merged]


# ---------------------------------------------------------------- runs
def _run(r, h_min, seed=2, h_ratio=2.0, eps=0.295, n_l=25, v_ref="auto", **kw):
    import synth
    case = synth.gaussian_cell(r=r, h_min=h_min, h_max=h_ratio * h_min, eps=eps, seed=seed)
    t = time.perf_counter()
    res = dict(r=r, h_min=h_min, seed=seed, h_ratio=h_ratio, eps=eps, n_l=n_l, n=case.n)
    try:
        out = crossval.cross_validate(case, n_l=n_l, v_ref=v_ref, **kw)
    except RbfError as e:  # a set-up the library rejects (e.g. too few fluid nodes for the wall stencils)
        nan = float("nan")
        res.update(error=str(e), wall_s=time.perf_counter() - t, delta_median=nan, delta_l2=nan)
        for nm in ("mlbm", "mns"):
            res[nm] = dict(k=nan, K=nan, steps=0, converged=False, time=0.0, wall_s=0.0, v_ref=None)
        return res
    res["wall_s"] = time.perf_counter() - t
    for nm in ("mlbm", "mns"):
        x = out[nm]
        res[nm] = dict(k=x["k_over_d2"], K=x["K"], steps=x["steps"], converged=x["converged"],
                       time=x["time"], wall_s=x["wall_s"], v_ref=x.get("v_ref"))
    res["delta_median"] = out["delta_summary"]["median"]
    res["delta_l2"] = out["delta_summary"]["l2_rel"]
    return res


def porosity_sweep(radii=SWEEP_RADII, h_min: float = 0.02, seed: int = 2, solid_check_above: float | None = None,
                   _ranks=(), **kw):
    """k/d^2 and K of both solvers over the radii (one cross-validation per
    radius, same nodes for both solvers).  solid_check_above: radius from which
    the MLBM uses the solid-check bounce-back rule (the paper switches to it
    near and past the touching limit).  _ranks: (dist, rank, world) to spread
    the radii over ranks (run_sharded)."""
    def one(r):
        rule = 1 if (solid_check_above is not None and r >= solid_check_above) else 0
        x = _run(r, h_min, seed=seed, unknown_rule=rule, **kw)
        x["unknown_rule"] = rule
        return x
    return run_sharded(one, list(radii), *_ranks)


def seed_spread(radii, h_min: float = 0.02, seeds=(1, 2, 3, 4, 5), _ranks=(), **kw):
    """Node-placement sensitivity: per radius, the standard deviation of k/d^2
    and K over node sets that differ only in the generator's seed, normalised
    by the mean (only converged runs count)."""
    pairs = [(r, sd) for r in radii for sd in seeds]
    allruns = run_sharded(lambda p: _run(p[0], h_min, seed=p[1], **kw), pairs, *_ranks)
    out = []
    for i, r in enumerate(radii):
        runs = allruns[i * len(seeds):(i + 1) * len(seeds)]
        row = dict(r=r, runs=runs)
        for nm in ("mlbm", "mns"):
            for q in ("k", "K"):
                v = np.array([x[nm][q] for x in runs if x[nm]["converged"] and np.isfinite(x[nm][q])])
                row[f"{nm}_{q}_spread"] = float(v.std(ddof=1) / v.mean()) if len(v) > 1 else float("nan")
                row[f"{nm}_{q}_n"] = int(len(v))
        out.append(row)
    return out


def convergence_study(r, h_list, **kw):
    """Both solvers at each h_min, then p and GCI of k/d^2 and K per solver."""
    runs = [_run(r, h, **kw) for h in h_list]
    res = dict(r=r, runs=runs)
    hs = [x["h_min"] for x in runs]
    for nm in ("mlbm", "mns"):
        for q in ("k", "K"):
            vals = [x[nm][q] for x in runs]
            try:
                p, g = gci(hs, vals)
            except ValueError:
                p, g = float("nan"), {}
            res[f"{nm}_{q}_p"] = p
            res[f"{nm}_{q}_gci"] = g
    return res


def refinement_parameter_study(r, h_min: float = 0.01, ratios=(1.0, 2.0, 3.0, 4.0), eps_list=(0.1, 0.2, 0.3),
                               **kw):
    """E(h_max/h_min, eps) of Eq. refinement_error for both solvers, against the
    uniform discretisation (ratio 1)."""
    ref = _run(r, h_min, h_ratio=1.0, eps=1.0, **kw)
    rows = []
    for ratio in ratios:
        if ratio == 1.0:
            continue
        for e in eps_list:
            x = _run(r, h_min, h_ratio=ratio, eps=e, **kw)
            for nm in ("mlbm", "mns"):
                x[nm]["E"] = refinement_error(x[nm]["K"], ref[nm]["K"]) if x[nm]["converged"] else float("nan")
            rows.append(x)
    return dict(r=r, reference=ref, rows=rows)


def stencil_size_study(r, n_l_list=(15, 20, 25, 30, 35, 40), h_min: float = 0.01, h_ratio: float = 3.0,
                       eps: float = 0.3, **kw):
    """K of both solvers against the stencil size N_L (the paper's stencil-size
    figure: r = 0.6526, h_max / h_min = 3)."""
    return [_run(r, h_min, h_ratio=h_ratio, eps=eps, n_l=n, **kw) for n in n_l_list]


def single_solver_trace(r, h_min, solver: str, chunk: int, chunks: int, seed: int = 2, n_l: int = 25,
                        v_ref=0.01, unknown_rule: int = 0, precision: int = RBF_FP64, tune: bool = True,
                        device: int = 0):
    """One solver alone on a Gaussian-refined cell, stepped in `chunks` chunks of
    `chunk` steps from rest: (steps, k/d^2, F_x) after every chunk, stopping at
    the first non-finite k.  For transients that the rate criterion of Eq.
    stopCrit cannot see (the MNS pressure relaxation at low porosity, reading its
    dependence on v_ref) and for MLBM stability under the two bounce-back rules."""
    import synth
    from . import RBF_SOLVER_ACM, RBF_SOLVER_LBM
    case = synth.gaussian_cell(r=r, h_min=h_min, seed=seed)
    if solver == "mlbm":
        s, _ = crossval._solver(case, n_l, 3, 2, RBF_SOLVER_LBM, 15, 0.5 * h_min,
                                dict(precision=precision, nu=1.0, g=(1.0, 0.0, 0.0), tau_plus=1.0, magic=1.0), device)
        if unknown_rule:
            s.lbm_set_unknown_rule(unknown_rule)
        if tune:
            s.autotune(20)
    else:
        s, v_ref = crossval._solver(case, n_l, 3, 2, RBF_SOLVER_ACM, 15, 0.0,
                                    dict(precision=precision, nu=1.0, g=(1.0, 0.0, 0.0), v_ref=v_ref, beta=10.0),
                                    device)
        if tune:
            s.autotune_persistent(200)
    trace = []
    t = time.perf_counter()
    for i in range(chunks):
        if solver == "mlbm":
            s.step(chunk)
        else:
            s.solve(chunk, 1e-300, check_every=chunk)
        k, _ = s.permeability(32)
        F, _ = s.drag(32)
        trace.append((chunk * (i + 1), k, F[0]))
        if not np.isfinite(k):
            break
    out = dict(r=r, h_min=h_min, solver=solver, n=case.n, n_l=n_l, v_ref=v_ref, unknown_rule=unknown_rule,
               dt=s.time_step(), trace=trace, wall_s=time.perf_counter() - t)
    s.close()
    return out


def main(argv=None):
    """Command line: one study, JSON to stdout (and --out).  Under torchrun the
    porosity sweep and the seed spread spread their runs over the ranks, one GPU
    per rank (LOCAL_RANK), and rank 0 prints the merged result."""
    import argparse
    import json

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("study", choices=("porosity", "spread", "convergence", "refinement", "stencil", "trace"))
    ap.add_argument("--radii", default=None, help="comma-separated radii")
    ap.add_argument("--h-min", type=float, default=0.02)
    ap.add_argument("--h-list", default="0.028,0.02,0.014,0.01")
    ap.add_argument("--seeds", default="1,2,3,4,5")
    ap.add_argument("--n-l-list", default="15,20,25,30,35,40")
    ap.add_argument("--window", type=int, default=10_000)
    ap.add_argument("--max-steps", type=int, default=4_000_000)
    ap.add_argument("--precision-acm", choices=("fp64", "fp32c"), default="fp32c")
    ap.add_argument("--precision-lbm", choices=("fp64", "fp32", "fp32r"), default="fp64",
                    help="MLBM populations: fp32r keeps FP32 steps on an FP64 base (RBF_FP32R)")
    ap.add_argument("--n-l-lbm", type=int, default=None, help="MLBM stencil size (default: --n-l)")
    ap.add_argument("--v-ref", default="auto", help='MNS reference speed: a number or "auto"')
    ap.add_argument("--solid-check-above", type=float, default=None)
    ap.add_argument("--solver", choices=("mlbm", "mns"), default="mns", help="trace: the solver")
    ap.add_argument("--v-ref-list", default="0.01", help="trace (MNS): comma-separated v_ref values")
    ap.add_argument("--unknown-rules", default="0", help="trace (MLBM): comma-separated rules")
    ap.add_argument("--n-l", type=int, default=25)
    ap.add_argument("--chunk", type=int, default=50_000)
    ap.add_argument("--chunks", type=int, default=4)
    ap.add_argument("--out", default=None)
    ap.add_argument("--progress", default=None,
                    help="append each finished run of a porosity sweep or seed spread here as a JSON line "
                         "(per rank: the rank number is added to the name)")
    a = ap.parse_args(argv)
    radii = tuple(float(x) for x in a.radii.split(",")) if a.radii else SWEEP_RADII
    dist, rank, world, local = dist_env()
    ranks = (dist, rank, world)
    global PROGRESS_PATH
    if a.progress:
        PROGRESS_PATH = a.progress if world == 1 else f"{a.progress}.{rank}"
    kw = dict(window_steps=a.window, max_steps=a.max_steps, tune=True, device=local,
              precision_acm=RBF_FP32C if a.precision_acm == "fp32c" else RBF_FP64,
              precision_lbm={"fp64": RBF_FP64, "fp32": RBF_FP32, "fp32r": RBF_FP32R}[a.precision_lbm],
              n_l_lbm=a.n_l_lbm, v_ref=a.v_ref if a.v_ref == "auto" else float(a.v_ref))
    if a.study in ("porosity", "spread"):
        kw["n_l"] = a.n_l
    t = time.perf_counter()
    if a.study == "porosity":
        res = porosity_sweep(radii, a.h_min, solid_check_above=a.solid_check_above, _ranks=ranks, **kw)
    elif a.study == "spread":
        res = seed_spread(radii, a.h_min, seeds=tuple(int(x) for x in a.seeds.split(",")), _ranks=ranks, **kw)
    elif a.study == "convergence":
        res = [convergence_study(r, [float(x) for x in a.h_list.split(",")], **kw) for r in radii]
    elif a.study == "refinement":
        res = [refinement_parameter_study(r, a.h_min, **kw) for r in radii]
    elif a.study == "stencil":
        res = [stencil_size_study(r, tuple(int(x) for x in a.n_l_list.split(",")), a.h_min, **kw) for r in radii]
    else:
        prec = RBF_FP32C if (a.solver == "mns" and a.precision_acm == "fp32c") else RBF_FP64
        variants = ([dict(v_ref=float(v)) for v in a.v_ref_list.split(",")] if a.solver == "mns"
                    else [dict(unknown_rule=int(u)) for u in a.unknown_rules.split(",")])
        res = [single_solver_trace(r, a.h_min, a.solver, a.chunk, a.chunks, n_l=a.n_l, precision=prec,
                                   device=local, **v) for r in radii for v in variants]
    txt = json.dumps(crossval._jsonable(dict(study=a.study, args=vars(a), ranks=world,
                                             wall_s=time.perf_counter() - t, result=res)))
    if rank != 0:
        return
    print(txt)
    if a.out:
        with open(a.out, "w") as f:
            f.write(txt + "\n")


if __name__ == "__main__":
    main()
