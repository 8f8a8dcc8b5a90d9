"""Reduced precision against the FP64 oracle at the steady state.

The oracle runs the MNS and the MLBM from rest until k/d^2 (Eq. k_definition)
and K (Eqs. integration_force, K_definition) no longer change, on a 1,511-node
cell.  The GPU then solves the same cell through rbf_solve to a stopping
criterion, in FP64, in compensated FP32 (RBF_FP32C) and in plain FP32, and its
permeability and drag coefficient must agree with the oracle's converged values:
FP64 to 1e-9, the FP32 forms to 1e-4 relative (the reduced-precision bar).

ACM runs at v_ref = 2 (Eq. MNS_C): with C = beta v_ref = 20 the artificial
sound waves relax faster than viscous diffusion, so the steady state is reached
in ~10^4 steps; both sides use the same v_ref.  The FP32 forms cannot take the
relative velocity change per step below ~1.5e-8 (rounding of FP32 stencil sums),
so their criterion is 3e-8; FP64 stops at 1e-13.  The MLBM criterion is the
relative change of k/d^2 between checks 500 steps apart.

A second MLBM case uses dx = h_min / 8: there the steady lattice velocity is
~6,600 times the per-step forcing (as on the 150k-node cell), so a relative
error of 1e-8 per step in the populations or the interpolation would shift k by
~1e-4.  Its oracle values come from tests/golden/steady_references.json
(written by tests/golden/make_steady_references.py, FP64 oracle; 230,000
steps), and the GPU runs the same number of steps.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_common import gpu_or_skip, oracle_acm_setup

pytestmark = pytest.mark.gpu

M_P = 24
V_REF = 2.0


@pytest.fixture(scope="module")
def rbf():
    return gpu_or_skip()


@pytest.fixture(scope="module")
def cell():
    return synth.jittered_cell(r=0.35, n_axis=12, seed=7)


@pytest.fixture(scope="module")
def acm_ref(cell):
    """Oracle MNS from rest to its steady state: (k/d^2, K, dt)."""
    o = oracle_acm_setup(cell, 25)
    dt = oracle.acm_dt(o["h_min"], 1.0)
    pr = oracle.probe_setup(cell["xyz"], cell["centre"], cell["radius"], M_P, 25)
    f, res = oracle.acm_run(cell, o["idx"], o["w4"], o["idxb"], o["wgb"], np.zeros((cell.n, 4)), 14000, dt=dt,
                            v_ref=V_REF)
    k1, q1 = oracle.permeability(pr, f[:, 0], 1.0, 1.0)
    f, res = oracle.acm_run(cell, o["idx"], o["w4"], o["idxb"], o["wgb"], f, 2000, dt=dt, v_ref=V_REF)
    k, q = oracle.permeability(pr, f[:, 0], 1.0, 1.0)
    F = oracle.drag(cell, o["idx"], o["w4"][o["wl"]][:, :3], f, 1.0)
    K = oracle.drag_coefficient(F[0], cell["radius"], q, 1.0)
    assert res[-1] < 1e-14 and abs(k - k1) <= 1e-13 * k  # converged
    return k, K, dt


@pytest.fixture(scope="module")
def lbm_ref(cell):
    """Oracle MLBM (D3Q19 TRT, tau+ = 0.8, Lambda = 3/16, dx = h_min / 2) from
    rest to its steady state: (k/d^2, K, dx)."""
    q, n_l = 19, 30
    idx = oracle.knn(cell["xyz"], cell["xyz"], n_l)
    dx = np.linalg.norm(oracle.min_image(cell["xyz"][idx[:, 1]] - cell["xyz"]), axis=1).min() / 2.0
    u = oracle.lbm_units(1.0, 0.8, dx, (1.0, 0.0, 0.0))
    wk = oracle.lbm_weights(cell["xyz"], idx, q, dx)
    tm = oracle.tau_minus(0.8, 3.0 / 16.0)
    f = oracle.lbm_equilibrium(q, np.ones(cell.n), np.zeros((cell.n, 3)))
    pr = oracle.probe_setup(cell["xyz"], cell["centre"], cell["radius"], M_P, n_l)
    wall = np.nonzero(cell["type"] == 1)[0]
    wg = oracle.rbf_weights(cell["xyz"], cell["xyz"][wall], idx[wall], 3, 2, oracle.ACM_OPS[:3])
    out = []
    for nsteps in (20000, 2000):
        f = oracle.lbm_run(f, q, cell, idx, wk, 0.8, tm, u["g_lb"], nsteps)
        uvwp = oracle.lbm_fields(f, q, u)
        k, qq = oracle.permeability(pr, uvwp[:, 0], 1.0, 1.0)
        F = oracle.drag(cell, idx, wg, uvwp, 1.0)
        out.append((k, oracle.drag_coefficient(F[0], cell["radius"], qq, 1.0)))
    (k1, K1), (k, K) = out
    assert abs(k - k1) <= 1e-10 * k and abs(K - K1) <= 1e-9 * K  # converged
    return k, K, dx


def _acm(rbf, cell, prec, dt):
    s = rbf.Solver(0)
    s.set_case(cell)
    s.build_stencils(25)
    s.compute_weights(solver=rbf.RBF_SOLVER_ACM)
    s.init(precision=prec, dt=dt, v_ref=V_REF)
    return s


@pytest.mark.parametrize("prec,tol,bar", [("fp64", 1e-13, 1e-9), ("fp32c", 3e-8, 1e-4), ("fp32", 3e-8, 1e-4)])
@pytest.mark.parametrize("code", [256, 4128])  # persistent schedule: one node per lane; four lanes per node
def test_acm_steady_k_and_K_against_oracle(rbf, cell, acm_ref, prec, tol, bar, code):
    k_o, K_o, dt = acm_ref
    p = {"fp64": rbf.RBF_FP64, "fp32": rbf.RBF_FP32, "fp32c": rbf.RBF_FP32C}[prec]
    s = _acm(rbf, cell, p, dt)
    s.set_persistent_block(code)
    r = s.solve(60000, tol, check_every=100, m_p=M_P)
    assert r["converged"], r
    k, _ = s.permeability(M_P)
    F, K = s.drag(M_P)
    assert abs(k - k_o) <= bar * k_o, (prec, k, k_o)
    assert abs(K - K_o) <= bar * K_o, (prec, K, K_o)
    s.close()


def test_acm_compensated_fp32_long_run_stays_on_the_oracle(rbf, cell, acm_ref):
    """Past the criterion, 20,000 more compensated FP32 steps neither stall nor
    drift: k/d^2 and K stay within 1e-5 of the oracle's steady values."""
    k_o, K_o, dt = acm_ref
    s = _acm(rbf, cell, rbf.RBF_FP32C, dt)
    s.solve(30000, 1e-300, check_every=1000, m_p=M_P)
    k, _ = s.permeability(M_P)
    F, K = s.drag(M_P)
    assert abs(k - k_o) <= 1e-5 * k_o and abs(K - K_o) <= 1e-5 * K_o, (k / k_o - 1, K / K_o - 1)
    s.close()


LBM_PREC = {"fp64": 0, "fp32": 1, "fp32r": 3}


@pytest.mark.parametrize("prec,variant,tol,bar", [("fp64", 1, 1e-12, 1e-8), ("fp32", 1, 2e-6, 1e-4),
                                                  ("fp32", 6, 2e-6, 1e-4), ("fp32r", 1, 1e-9, 1e-7),
                                                  ("fp32r", 6, 1e-9, 1e-7)])
def test_lbm_steady_k_and_K_against_oracle(rbf, cell, lbm_ref, prec, variant, tol, bar):
    k_o, K_o, dx = lbm_ref
    s = rbf.Solver(0)
    s.set_case(cell)
    s.build_stencils(30)
    s.compute_weights(solver=rbf.RBF_SOLVER_LBM, q=19, dx=dx)
    s.init(precision=LBM_PREC[prec], g=(1.0, 0.0, 0.0))
    s.set_kernel_variant(variant)
    r = s.solve(60000, tol, check_every=500, m_p=M_P)
    assert r["converged"], r
    k, _ = s.permeability(M_P)
    F, K = s.drag(M_P)
    assert abs(k - k_o) <= bar * k_o, (prec, k, k_o)
    assert abs(K - K_o) <= bar * K_o, (prec, K, K_o)
    s.close()


def _golden(name):
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "steady_references.json")
    return json.load(open(here))[name]


@pytest.mark.parametrize("prec,variant,bar", [("fp64", 1, 1e-8), ("fp32r", 1, 1e-6), ("fp32r", 6, 1e-6)])
def test_lbm_steady_small_dx_against_oracle(rbf, cell, prec, variant, bar):
    """FP64 and refined FP32 reach the oracle's steady state where the per-step
    forcing is ~1.5e-4 of the populations' deviation; plain FP32 is measured
    (test below) but carries a rounding bias of ~3e-4 there."""
    ref = _golden("mlbm_small_dx8")
    assert ref["nodes"] == cell.n
    s = rbf.Solver(0)
    s.set_case(cell)
    s.build_stencils(30)
    s.compute_weights(solver=rbf.RBF_SOLVER_LBM, q=19, dx=ref["dx"])
    s.init(precision=LBM_PREC[prec], g=(1.0, 0.0, 0.0))
    s.set_kernel_variant(variant)
    s.step(ref["steps"])
    k, _ = s.permeability(M_P)
    F, K = s.drag(M_P)
    assert abs(k - ref["k_over_d2"]) <= bar * ref["k_over_d2"], (prec, k / ref["k_over_d2"] - 1)
    assert abs(K - ref["K"]) <= bar * ref["K"], (prec, K / ref["K"] - 1)
    s.close()


def test_lbm_plain_fp32_bias_at_small_dx_is_bounded_and_refinement_removes_it(rbf, cell):
    """Plain FP32 populations at dx = h_min / 8: the steady k/d^2 is off by the
    accumulated per-step rounding (measured 3.4e-4 with sum-preserving FP32
    weights) but not by more than 1e-3; refined FP32 on the same case is at
    least 100 times closer."""
    ref = _golden("mlbm_small_dx8")
    errs = {}
    for prec in ("fp32", "fp32r"):
        s = rbf.Solver(0)
        s.set_case(cell)
        s.build_stencils(30)
        s.compute_weights(solver=rbf.RBF_SOLVER_LBM, q=19, dx=ref["dx"])
        s.init(precision=LBM_PREC[prec], g=(1.0, 0.0, 0.0))
        s.set_kernel_variant(6)
        s.step(ref["steps"])
        errs[prec] = abs(s.permeability(M_P)[0] / ref["k_over_d2"] - 1.0)
        s.close()
    assert errs["fp32"] <= 1e-3 and errs["fp32r"] <= 1e-2 * errs["fp32"], errs
