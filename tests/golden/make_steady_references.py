"""Writes tests/golden/steady_references.json: steady permeability k/d^2 (Eq.
k_definition) and drag coefficient K (Eqs. integration_force, K_definition) of
the FP64 oracle on the seeded cells that the steady-state parity tests and the
time-to-steady measurement compare against.  Calls only oracle/ and synth/.

Each entry runs the oracle from rest (MNS: v = p = 0; MLBM: f = f_eq(1, 0)) in
windows of `window` steps until k and K change by less than `tol` relative over
one window, and records k, K, the steps taken and the last window's change.

  python tests/golden/make_steady_references.py [name ...]   (default: all)

Each entry records the CPU seconds it took: the config-2 MLBM entry 3.4 hours on
8 cores, each held-out entry of the warm-start experiment 4-16 minutes, the
config-4-family entry under 4 minutes.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(HERE, "steady_references.json")


def _mns(case, n_l, v_ref, m_p, window, tol, max_steps, k=3, m=2):
    idx = oracle.knn(case["xyz"], case["xyz"], n_l, grid=case.n > 20000 or None)
    w4 = oracle.acm_weights(case["xyz"], idx, k, m)
    wl, idxb = oracle.neumann_stencils(case, n_l)
    wgb = oracle.neumann_weights(case, idxb, k, m)
    h_min = np.linalg.norm(oracle.min_image(case["xyz"][idx[:, 1]] - case["xyz"]), axis=1).min()
    dt = oracle.acm_dt(h_min, 1.0)
    pr = oracle.probe_setup(case["xyz"], case["centre"], case["radius"], m_p, n_l, k, m)
    f = np.zeros((case.n, 4))
    steps, prev = 0, None
    while True:
        f, _ = oracle.acm_run(case, idx, w4, idxb, wgb, f, window, dt=dt, v_ref=v_ref)
        steps += window
        k, q = oracle.permeability(pr, f[:, 0], 1.0, 1.0)
        F = oracle.drag(case, idx, w4[wl][:, :3], f, 1.0)
        K = oracle.drag_coefficient(F[0], case["radius"], q, 1.0)
        if prev is not None:
            ck, cK = abs(k - prev[0]) / abs(k), abs(K - prev[1]) / abs(K)
            print(f"  {steps} k={k:.12e} K={K:.10e} dk={ck:.1e} dK={cK:.1e}", flush=True)
            if (ck < tol and cK < tol) or steps >= max_steps:
                return dict(k_over_d2=k, K=K, steps=steps, last_window_change_k=ck, last_window_change_K=cK,
                            dt=dt, h_min=h_min)
        prev = (k, K)


def _mlbm(case, n_l, q, dx, m_p, window, tol, max_steps, tau_plus=0.8, magic=3.0 / 16.0):
    idx = oracle.knn(case["xyz"], case["xyz"], n_l, grid=case.n > 20000 or None)
    h_min = np.linalg.norm(oracle.min_image(case["xyz"][idx[:, 1]] - case["xyz"]), axis=1).min()
    dx = dx if dx > 0 else h_min / -dx
    u = oracle.lbm_units(1.0, tau_plus, dx, (1.0, 0.0, 0.0))
    wk = oracle.lbm_weights(case["xyz"], idx, q, dx)
    tm = oracle.tau_minus(tau_plus, magic)
    wall = np.nonzero(case["type"] == 1)[0]
    wg = oracle.rbf_weights(case["xyz"], case["xyz"][wall], idx[wall], 3, 2, oracle.ACM_OPS[:3])
    pr = oracle.probe_setup(case["xyz"], case["centre"], case["radius"], m_p, n_l)
    f = oracle.lbm_equilibrium(q, np.ones(case.n), np.zeros((case.n, 3)))
    steps, prev = 0, None
    while True:
        f = oracle.lbm_run(f, q, case, idx, wk, tau_plus, tm, u["g_lb"], window)
        steps += window
        fld = oracle.lbm_fields(f, q, u)
        k, qq = oracle.permeability(pr, fld[:, 0], 1.0, 1.0)
        F = oracle.drag(case, idx, wg, fld, 1.0)
        K = oracle.drag_coefficient(F[0], case["radius"], qq, 1.0)
        if prev is not None:
            ck, cK = abs(k - prev[0]) / abs(k), abs(K - prev[1]) / abs(K)
            print(f"  {steps} k={k:.12e} K={K:.10e} dk={ck:.1e} dK={cK:.1e}", flush=True)
            if (ck < tol and cK < tol) or steps >= max_steps:
                return dict(k_over_d2=k, K=K, steps=steps, last_window_change_k=ck, last_window_change_K=cK,
                            dx=dx, dt=u["dt"], h_min=h_min)
        prev = (k, K)


ENTRIES = {
    # MLBM on a 1,511-node jittered cell with dx = h_min / 8: the ratio of the
    # steady lattice velocity to the per-step forcing (~ k / (nu_lb dx^2), the
    # momentum relaxation time in steps) is ~6,600, like the 150k-node cell's
    # ~8,300, so per-step rounding in reduced precision weighs as much as there
    "mlbm_small_dx8": dict(
        case=dict(kind="jittered", r=0.35, n_axis=12, seed=7),
        run=lambda c: _mlbm(c, 30, 19, -8.0, 24, 10000, 1e-9, 600000)),
    # MNS on the 6,857-node jittered cell (h = 1/20, r = 0.35, N_L = 25), v_ref = 2
    "mns_config1_vref2": dict(
        case=dict(kind="jittered", r=0.35, n_axis=20, seed=1),
        run=lambda c: _mns(c, 25, 2.0, 32, 2000, 1e-10, 100000)),
    # MLBM D3Q19 TRT on the 149,640-node h-refined cell (r = 0.4, h(d) = 0.008 +
    # 0.032 min(1, d / 0.2), seed 2), N_L = 30, dx = 0.004, tau+ = 0.8, Lambda = 3/16
    "mlbm_config2": dict(
        case=dict(kind="refined", r=0.4, h_min=0.008, h_max=0.04, ramp=0.2, seed=2),
        run=lambda c: _mlbm(c, 30, 19, 0.004, 32, 10000, 2e-8, 600000)),
}

# Held-out cells of the warm-start experiment at the configured node counts:
# jittered grid h = 1/40 (41k-58k nodes), five radii inside the training range
# and not drawn for it, MNS at v_ref = 2.  (Radii below ~0.25 relax with time
# constants of ~2e4 steps at this resolution; their oracle runs take hours.)
HELDOUT_RADII = (0.29, 0.33, 0.37, 0.41, 0.45)
for _i, _r in enumerate(HELDOUT_RADII):
    ENTRIES[f"mns_c5_heldout_{_i}"] = dict(
        case=dict(kind="jittered", r=_r, n_axis=40, seed=900 + _i),
        run=lambda c: _mns(c, 25, 2.0, 32, 4000, 1e-8, 400000))

# The family of the large mixed-precision ACM cell (r = 0.45, PHS r^5 + order-3
# monomials, N_L = 40) at a resolution the oracle can take to its steady state
# (h 0.02 at the wall to 0.03, 52,941 nodes; the 3M-node cell at h 0.003..0.02
# needs ~1e6 steps), MNS at v_ref = 2.
ENTRIES["mns_config4_family"] = dict(
    case=dict(kind="refined", r=0.45, h_min=0.02, h_max=0.03, ramp=0.32, seed=4),
    run=lambda c: _mns(c, 40, 2.0, 32, 4000, 1e-8, 400000, k=5, m=3))


def make_case(spec):
    s = dict(spec)
    kind = s.pop("kind")
    return synth.jittered_cell(**s) if kind == "jittered" else synth.refined_cell(**s)


def main(names):
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        e = ENTRIES[name]
        case = make_case(e["case"])
        print(name, case.n, "nodes", flush=True)
        t0 = time.time()
        rec = e["run"](case)
        rec.update(case=e["case"], nodes=int(case.n), cpu_seconds=time.time() - t0,
                   written_by="tests/golden/make_steady_references.py (FP64 oracle)")
        data[name] = rec
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
        print(name, rec, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(ENTRIES))
