"""The parameter-study drivers (studies.seed_spread, studies.convergence_study)
on the GPU, each run checked against the oracle on the same nodes.

A study run is a cross-validation: the MLBM (the paper's D3Q15, Lambda = 1,
tau+ = 1, dx = h_min / 2) and the MNS each step to the stopping rule of Eq.
stopCrit, then k/d^2 (Eq. k_definition) and K (Eq. K_definition) are read.  The
oracle replays each solver for exactly the number of steps the driver took
(and, for the MNS, with the v_ref it used), so k/d^2 and K must agree to FP64
parity; the studies' own statistics (spread over seeds, apparent order, GCI)
are host arithmetic on those values, pinned in test_studies_host.py.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import gpu_or_skip, oracle_acm_setup

pytestmark = pytest.mark.gpu

KW = dict(window_steps=2000, v_ref=2.0, n_l=25)


@pytest.fixture(scope="module")
def rbf():
    return gpu_or_skip()


def _oracle_run(r, h_min, seed, run, m_p=32):
    case = synth.gaussian_cell(r=r, h_min=h_min, h_max=2.0 * h_min, eps=0.295, seed=seed)
    assert case.n == run["n"]
    o = oracle_acm_setup(case, 25)
    pr = oracle.probe_setup(case["xyz"], case["centre"], case["radius"], m_p, 25)
    wg = o["w4"][o["wl"]][:, :3]
    out = {}
    # MNS: the driver's time step (cfl h_min^2 / (2 nu), h_min the smallest
    # internodal distance) and its v_ref
    dt = oracle.acm_dt(o["h_min"], 1.0)
    f, _ = oracle.acm_run(case, o["idx"], o["w4"], o["idxb"], o["wgb"], np.zeros((case.n, 4)), run["mns"]["steps"],
                          dt=dt, v_ref=run["mns"]["v_ref"])
    k, q = oracle.permeability(pr, f[:, 0], 1.0, 1.0)
    out["mns"] = (k, oracle.drag_coefficient(oracle.drag(case, o["idx"], wg, f, 1.0)[0], r, q, 1.0))
    # MLBM: D3Q15, Lambda = 1, tau+ = 1, dx = h_min / 2 of the generator
    qn, dx = 15, 0.5 * h_min
    u = oracle.lbm_units(1.0, 1.0, dx, (1.0, 0.0, 0.0))
    wk = oracle.lbm_weights(case["xyz"], o["idx"], qn, dx)
    fl = oracle.lbm_run(oracle.lbm_equilibrium(qn, np.ones(case.n), np.zeros((case.n, 3))), qn, case, o["idx"], wk,
                        1.0, oracle.tau_minus(1.0, 1.0), u["g_lb"], run["mlbm"]["steps"])
    fld = oracle.lbm_fields(fl, qn, u)
    k, q = oracle.permeability(pr, fld[:, 0], 1.0, 1.0)
    out["mlbm"] = (k, oracle.drag_coefficient(oracle.drag(case, o["idx"], wg, fld, 1.0)[0], r, q, 1.0))
    return out


def _check(run, want):
    for nm in ("mns", "mlbm"):
        assert run[nm]["converged"], (nm, run[nm])
        k, K = want[nm]
        assert abs(run[nm]["k"] - k) <= 1e-8 * abs(k), (nm, run[nm]["k"], k)
        assert abs(run[nm]["K"] - K) <= 1e-8 * abs(K), (nm, run[nm]["K"], K)


def test_seed_spread_runs_match_the_oracle(rbf):
    from paper_2404_14195_gb300 import studies
    r, h_min = 0.3, 0.05
    rows = studies.seed_spread([r], h_min=h_min, seeds=(1, 2), **KW)
    assert len(rows) == 1 and len(rows[0]["runs"]) == 2
    for run, seed in zip(rows[0]["runs"], (1, 2)):
        _check(run, _oracle_run(r, h_min, seed, run))
    # the spread is the host statistic of the two runs' values
    ks = np.array([x["mns"]["k"] for x in rows[0]["runs"]])
    assert abs(rows[0]["mns_k_spread"] - ks.std(ddof=1) / ks.mean()) <= 1e-12


def test_convergence_study_runs_match_the_oracle(rbf):
    from paper_2404_14195_gb300 import studies
    r = 0.25
    res = studies.convergence_study(r, [0.06, 0.05, 0.042], **KW)
    assert len(res["runs"]) == 3
    for run in res["runs"]:
        _check(run, _oracle_run(r, run["h_min"], run["seed"], run))
    for nm in ("mns", "mlbm"):
        assert np.isfinite(res[f"{nm}_k_p"]) and len(res[f"{nm}_k_gci"]) == 2
