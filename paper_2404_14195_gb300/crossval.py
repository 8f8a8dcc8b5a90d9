"""Cross-validation of the two solvers on identical nodes (the section
"Pointwise comparison of the meshless solvers"): the MLBM and the MNS (ACM)
solver run on the same node set to the steady state of Eq. stopCrit; then the
permeability k/d^2 (Eq. k_definition), the drag coefficient K (Eq.
K_definition) and the pointwise velocity difference delta(x) of Eq.
pointwise_error are compared.

Orchestration only: stepping, probes, drag and the pointwise difference run in
the library's kernels (rbf_step / rbf_solve, rbf_permeability, rbf_drag,
rbf_pointwise_difference); the host evaluates the scalar stopping rule between
windows and summarises the per-node arrays.
"""
from __future__ import annotations

import time

import numpy as np

from . import (RBF_EDIVERGED, RBF_FP64, RBF_SOLVER_ACM, RBF_SOLVER_LBM, RbfError, Solver, pointwise_difference)

# isocontour levels of delta drawn in the paper's pointwise comparison figure
ISO_LEVELS = {0.062: (0.1, 0.05, 0.01), 0.6526: (1.0, 0.25, 0.05)}


def stop_rate(k_now: float, k_prev: float, window: float) -> float:
    """|Delta|_{k/d^2} of Eq. stopCrit: relative change of k/d^2 over the last
    window, per unit physical time."""
    return abs(k_now - k_prev) / (abs(k_now) * window)


def run_to_steady(s: Solver, tol: float = 1e-2, window_steps: int = 10_000, max_steps: int = 2_000_000,
                  m_p: int = 32, min_windows: int = 2):
    """Step `s` in windows of `window_steps` until the stopping rule of Eq.
    stopCrit holds (rate below `tol` per unit time; the paper: 10^4 steps and
    10^-2), or `max_steps`.  ACM windows run in one persistent launch each, LBM
    windows as graph-captured steps.  Returns steps, physical time, the (step,
    k/d^2) history, the last rate, converged flag and the wall time."""
    dt = s.time_step()
    hist, rate, k_prev = [], float("inf"), None
    steps = 0
    t0 = time.perf_counter()
    converged = False
    while steps < max_steps:
        n = int(min(window_steps, max_steps - steps))
        try:
            if s.solver == RBF_SOLVER_ACM:
                s.solve(n, 1e-300, check_every=n, m_p=m_p)
            else:
                s.step(n)
        except RbfError as e:  # the persistent driver reports non-finite fields itself
            if e.code != RBF_EDIVERGED:
                raise
            steps += n
            hist.append((steps, float("nan")))
            break
        steps += n
        k, _ = s.permeability(m_p)
        hist.append((steps, k))
        if not np.isfinite(k):
            break
        if k_prev is not None:
            rate = stop_rate(k, k_prev, n * dt)
            if rate < tol and len(hist) >= min_windows:
                converged = True
                break
        k_prev = k
    return dict(steps=steps, time=steps * dt, dt=dt, history=hist, rate=rate, converged=converged,
                wall_s=time.perf_counter() - t0)


def auto_v_ref(h_min: float, nu: float = 1.0, beta: float = 10.0, cfl: float = 0.1, courant: float = 0.01) -> float:
    """v_ref that puts the artificial sound speed C = beta v_ref at an acoustic
    Courant number C dt / h_min = `courant`, with dt = cfl h_min^2 / (2 nu) the
    MNS time step (h_min the smallest internodal distance).  A build choice, not
    the paper's: the steady state does not depend on C, and a C this large lets
    the pressure relax within ~10^5 steps also in low-porosity cells (0.01 is
    about a tenth of the Courant number at which r = 0.6526 went unstable)."""
    return courant * 2.0 * nu / (beta * cfl * h_min)


def _solver(case, n_l, k, m, solver, q, dx, init_kw, device):
    s = Solver(device)
    s.set_case(case)
    s.build_stencils(n_l)
    rep = s.compute_weights(k=k, m=m, solver=solver, q=q, dx=dx)
    kw = dict(init_kw)
    if kw.get("v_ref") == "auto":
        kw["v_ref"] = auto_v_ref(rep["h_min"], kw.get("nu", 1.0), kw.get("beta", 10.0))
    s.init(**kw)
    return s, kw.get("v_ref")


def line_profile(case, v_a, v_b, half_width: float | None = None, y0: float = 0.5, z0: float = 0.5):
    """Fluid nodes in a tube around the line y = y0, z = z0 (the paper's line
    plot), sorted by x: x, |v_a|, |v_b|, |v_a - v_b| (Eq. pointwise_error's
    Delta v) and ||v_a| - |v_b|| (the difference of magnitudes the line plot
    shows)."""
    xyz = np.asarray(case["xyz"])
    hw = case["h_min"] if half_width is None else half_width
    dy = np.abs((xyz[:, 1] - y0 + 0.5) % 1.0 - 0.5)
    dz = np.abs((xyz[:, 2] - z0 + 0.5) % 1.0 - 0.5)
    sel = np.nonzero((dy < hw) & (dz < hw) & (np.asarray(case["type"]) == 0))[0]
    sel = sel[np.argsort(xyz[sel, 0])]
    na = np.sqrt((v_a[sel] ** 2).sum(1))
    nb = np.sqrt((v_b[sel] ** 2).sum(1))
    dv = np.sqrt(((v_a[sel] - v_b[sel]) ** 2).sum(1))
    return dict(x=xyz[sel, 0], node=sel, speed_a=na, speed_b=nb, dv=dv, dspeed=np.abs(na - nb))


def delta_summary(case, delta, dv, v_b_speed, levels=(1.0, 0.25, 0.1, 0.05, 0.01)):
    """Statistics of delta over fluid nodes where it is defined: percentiles,
    the fraction of nodes above each isocontour level, and the velocity-weighted
    relative difference sqrt(sum dv^2 / sum |v_b|^2)."""
    fl = (np.asarray(case["type"]) == 0) & np.isfinite(delta)
    d = delta[fl]
    if d.size == 0:  # a diverged solution leaves no finite delta
        return dict(n_fluid=0, median=float("nan"), mean=float("nan"), p90=float("nan"), p99=float("nan"),
                    max=float("nan"), frac_above={float(l): float("nan") for l in levels}, l2_rel=float("nan"))
    out = dict(n_fluid=int(fl.sum()),
               median=float(np.median(d)), mean=float(d.mean()),
               p90=float(np.percentile(d, 90)), p99=float(np.percentile(d, 99)), max=float(d.max()),
               frac_above={float(l): float((d > l).mean()) for l in levels},
               l2_rel=float(np.sqrt((dv[fl] ** 2).sum() / (v_b_speed[fl] ** 2).sum())))
    return out


def cross_validate(case, n_l: int = 25, k: int = 3, m: int = 2, q: int = 15, dx: float | None = None,
                   tau_plus: float = 1.0, magic: float = 1.0, nu: float = 1.0, g=(1.0, 0.0, 0.0),
                   v_ref: float | str = 0.01, beta: float = 10.0, precision_lbm: int = RBF_FP64,
                   precision_acm: int = RBF_FP64, tol: float = 1e-2, window_steps: int = 10_000,
                   window_steps_lbm: int | None = None, max_steps: int = 2_000_000, m_p: int = 32,
                   device: int = 0, keep_fields: bool = False, unknown_rule: int = 0, n_l_lbm: int | None = None,
                   tune: bool = False):
    """Both solvers on `case`'s nodes, each to the steady state of Eq. stopCrit,
    then k/d^2, K and Eq. pointwise_error with a = MLBM, b = MNS.  The MLBM
    defaults are the paper's: D3Q15, TRT with Lambda = 1 and tau+ = 1, streaming
    distance dx = h_min / 2.  unknown_rule selects the MLBM bounce-back rule
    (rbf_lbm_set_unknown_rule: 0 wall normal, 1 solid check); n_l_lbm a separate
    MLBM stencil size (the paper enlarges it near the touching limit).  tune:
    pick the step schedules first (rbf_autotune_persistent for the MNS,
    rbf_autotune for the MLBM; both restore the state after their trials).
    v_ref sets the artificial sound speed C = beta max(max|v|, v_ref) of Eq.
    MNS_C.  It does not change the steady state, only how fast the pressure
    relaxes: in low-porosity cells (r = 0.6526) the default 0.01 leaves a
    transient so slow that the rate criterion of Eq. stopCrit fires long before
    k/d^2 has settled, and a v_ref of order 10 is needed.  v_ref = "auto" takes
    auto_v_ref of the cell's smallest internodal distance.
    Returns a dict with per-solver results, the delta summary, the line profile
    and (keep_fields) the velocity fields."""
    dx = 0.5 * case["h_min"] if dx is None else dx
    t0 = time.perf_counter()
    lbm, _ = _solver(case, n_l_lbm or n_l, k, m, RBF_SOLVER_LBM, q, dx,
                     dict(precision=precision_lbm, nu=nu, g=g, tau_plus=tau_plus, magic=magic), device)
    try:
        acm, v_ref_used = _solver(case, n_l, k, m, RBF_SOLVER_ACM, q, 0.0,
                                  dict(precision=precision_acm, nu=nu, g=g, v_ref=v_ref, beta=beta), device)
    except Exception:
        lbm.close()
        raise
    try:
        return _compare(case, lbm, acm, v_ref_used, time.perf_counter() - t0, dx, unknown_rule, tune, tol,
                        window_steps, window_steps_lbm, max_steps, m_p, keep_fields)
    finally:
        lbm.close()
        acm.close()


def _compare(case, lbm, acm, v_ref_used, setup_s, dx, unknown_rule, tune, tol, window_steps, window_steps_lbm,
             max_steps, m_p, keep_fields):
    out = dict(n=case.n, n_wall=int((np.asarray(case["type"]) == 1).sum()), dx=dx, setup_s=setup_s)
    for name, s, w in (("mlbm", lbm, window_steps_lbm or window_steps), ("mns", acm, window_steps)):
        if name == "mlbm" and unknown_rule:
            s.lbm_set_unknown_rule(unknown_rule)
        if tune:  # both tuners restore the state after their trials
            if name == "mns":
                s.autotune_persistent(200)
            else:
                s.autotune(20)
        r = run_to_steady(s, tol=tol, window_steps=w, max_steps=max_steps, m_p=m_p)
        kk, qq = s.permeability(m_p)
        F, K = s.drag(m_p)
        r.update(k_over_d2=kk, q=qq, F=F, K=K)
        if name == "mns":
            r["v_ref"] = v_ref_used
        out[name] = r
    delta, dv = pointwise_difference(lbm, acm)
    fa, fb = lbm.get_fields(), acm.get_fields()
    va, vb = fa[:, :3], fb[:, :3]
    out["delta_summary"] = delta_summary(case, delta, dv, np.sqrt((vb * vb).sum(1)))
    out["line"] = line_profile(case, va, vb)
    out["diverged"] = [nm for nm in ("mlbm", "mns") if not np.isfinite(out[nm]["k_over_d2"])]
    out["k_rel_diff"] = abs(out["mlbm"]["k_over_d2"] - out["mns"]["k_over_d2"]) / abs(out["mns"]["k_over_d2"])
    out["K_rel_diff"] = abs(out["mlbm"]["K"] - out["mns"]["K"]) / abs(out["mns"]["K"])
    if keep_fields:
        out.update(delta=delta, dv=dv, fields_mlbm=fa, fields_mns=fb)
    return out


def _jsonable(x):
    if isinstance(x, dict):
        return {str(k): _jsonable(v) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [_jsonable(v) for v in x]
    if isinstance(x, np.ndarray):
        return _jsonable(x.tolist())
    if isinstance(x, (np.floating, float)):
        return float(x) if np.isfinite(x) else None
    if isinstance(x, (np.integer,)):
        return int(x)
    return x


def main(argv=None):
    """Command line: one cross-validation run on a Gaussian-refined cell; prints
    one JSON object (per-solver steps, times, k/d^2, K; delta statistics; the
    line profile thinned to at most 64 points)."""
    import argparse
    import json

    from . import RBF_FP32, RBF_FP32C, RBF_FP64
    import synth  # the seeded node generators beside the package

    prec = {"fp64": RBF_FP64, "fp32": RBF_FP32, "fp32c": RBF_FP32C}
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--r", type=float, default=0.062)
    ap.add_argument("--h-min", type=float, default=0.02)
    ap.add_argument("--h-ratio", type=float, default=2.0, help="h_max / h_min")
    ap.add_argument("--eps", type=float, default=0.295)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--n-l", type=int, default=25)
    ap.add_argument("--q", type=int, default=15)
    ap.add_argument("--tau-plus", type=float, default=1.0)
    ap.add_argument("--magic", type=float, default=1.0)
    ap.add_argument("--n-l-lbm", type=int, default=None)
    ap.add_argument("--unknown-rule", type=int, default=0, choices=(0, 1))
    ap.add_argument("--v-ref", default="0.01", help='a number, or "auto"')
    ap.add_argument("--tune", action="store_true")
    ap.add_argument("--tol", type=float, default=1e-2)
    ap.add_argument("--window", type=int, default=10_000)
    ap.add_argument("--max-steps", type=int, default=4_000_000)
    ap.add_argument("--precision-lbm", choices=sorted(prec), default="fp64")
    ap.add_argument("--precision-acm", choices=sorted(prec), default="fp64")
    ap.add_argument("--out", default=None, help="also write the JSON here")
    a = ap.parse_args(argv)
    case = synth.gaussian_cell(r=a.r, h_min=a.h_min, h_max=a.h_ratio * a.h_min, eps=a.eps, seed=a.seed)
    out = cross_validate(case, n_l=a.n_l, q=a.q, tau_plus=a.tau_plus, magic=a.magic, tol=a.tol,
                         window_steps=a.window, max_steps=a.max_steps, precision_lbm=prec[a.precision_lbm],
                         precision_acm=prec[a.precision_acm], unknown_rule=a.unknown_rule, n_l_lbm=a.n_l_lbm,
                         v_ref=a.v_ref if a.v_ref == "auto" else float(a.v_ref), tune=a.tune)
    line = out.pop("line")
    step = max(1, len(line["x"]) // 64)
    out["line"] = {k: v[::step] for k, v in line.items() if k != "node"}
    for name in ("mlbm", "mns"):
        h = out[name]["history"]
        out[name]["history"] = h[-5:]
    out["args"] = vars(a)
    txt = json.dumps(_jsonable(out))
    print(txt)
    if a.out:
        with open(a.out, "w") as f:
            f.write(txt + "\n")


if __name__ == "__main__":
    main()
