"""The precision report of the large mixed-precision ACM cell, on a cell of its
family that the oracle can take to its steady state.

The configured cell (r = 0.45, PHS r^5 + order-3 monomials, N_L = 40, h 0.003 at
the wall to 0.02, 3.0M nodes) would need ~1e6 steps to its steady state, and its
oracle hours per thousand steps.  The same family at h 0.02..0.03 (52,941 nodes)
reaches it in 28,000 oracle steps: tests/golden/steady_references.json, entry
mns_config4_family (written by tests/golden/make_steady_references.py, FP64
oracle, MNS at v_ref = 2).

Each precision runs rbf_solve from rest to the configuration's criterion, a
relative velocity change per step (residual) below 1e-7.  There k/d^2 (Eq.
k_definition) and K (Eqs. integration_force, K_definition) must agree with the
oracle's steady values and with the FP64 GPU path to 1e-4 relative, the
reduced-precision bar.  FP64 continued to a residual of 1e-13 must agree with the
oracle to 1e-8, and compensated FP32 after 28,000 more steps (~40,000 in all; its
residual no longer falls below ~1.4e-8) to 1e-5.
"""
import json
import os

import pytest

import synth
from gpu_common import gpu_or_skip

pytestmark = pytest.mark.gpu

N_L, PHS_K, MONO_M, M_P, V_REF = 40, 5, 3, 32, 2.0


def _ref():
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "steady_references.json")
    return json.load(open(here))["mns_config4_family"]


@pytest.fixture(scope="module")
def rbf():
    return gpu_or_skip()


@pytest.fixture(scope="module")
def case():
    spec = dict(_ref()["case"])
    assert spec.pop("kind") == "refined"
    c = synth.refined_cell(**spec)
    assert c.n == _ref()["nodes"]
    return c


def _solve(rbf, case, prec, stages):
    """k/d^2, K and the steps taken after each (max_steps, residual criterion) stage
    of rbf_solve from rest in turn; a criterion of 0 runs the stage's steps."""
    s = rbf.Solver(0)
    s.set_case(case)
    s.build_stencils(N_L)
    s.compute_weights(k=PHS_K, m=MONO_M, solver=rbf.RBF_SOLVER_ACM)
    s.init(precision=prec, dt=_ref()["dt"], v_ref=V_REF)
    out = []
    for max_steps, tol in stages:
        r = s.solve(max_steps, tol if tol > 0 else 1e-300, check_every=100, m_p=M_P)
        assert r["converged"] or tol == 0, (prec, tol, r)
        k, _ = s.permeability(M_P)
        _, K = s.drag(M_P)
        out.append((k, K, r["steps"]))
    s.close()
    return out


@pytest.fixture(scope="module")
def fp64(rbf, case):
    return _solve(rbf, case, rbf.RBF_FP64, ((60000, 1e-7), (60000, 1e-13)))


def test_fp64_against_oracle(fp64):
    ref = _ref()
    (k7, K7, _), (k, K, _) = fp64
    assert abs(k7 - ref["k_over_d2"]) <= 1e-4 * ref["k_over_d2"] and abs(K7 - ref["K"]) <= 1e-4 * ref["K"]
    assert abs(k - ref["k_over_d2"]) <= 1e-8 * ref["k_over_d2"], k / ref["k_over_d2"] - 1
    assert abs(K - ref["K"]) <= 1e-8 * ref["K"], K / ref["K"] - 1


@pytest.mark.parametrize("prec", ["fp32c", "fp32"])
def test_reduced_precision_at_residual_1e7(rbf, case, fp64, prec):
    ref = _ref()
    p = {"fp32": rbf.RBF_FP32, "fp32c": rbf.RBF_FP32C}[prec]
    # compensated FP32: then 28,000 more steps (~40,000 in all)
    got = _solve(rbf, case, p, [(60000, 1e-7)] + ([(28000, 0)] if prec == "fp32c" else []))
    k, K, _ = got[0]
    k64, K64, _ = fp64[0]
    assert abs(k - ref["k_over_d2"]) <= 1e-4 * ref["k_over_d2"], (prec, k / ref["k_over_d2"] - 1)
    assert abs(K - ref["K"]) <= 1e-4 * ref["K"], (prec, K / ref["K"] - 1)
    assert abs(k - k64) <= 1e-4 * abs(k64) and abs(K - K64) <= 1e-4 * abs(K64), (prec, k / k64 - 1, K / K64 - 1)
    if prec == "fp32c":
        k, K, _ = got[1]
        assert abs(k - ref["k_over_d2"]) <= 1e-5 * ref["k_over_d2"], k / ref["k_over_d2"] - 1
        assert abs(K - ref["K"]) <= 1e-5 * ref["K"], K / ref["K"] - 1
