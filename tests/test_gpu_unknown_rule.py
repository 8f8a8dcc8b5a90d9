"""The MLBM unknown-population rules on the GPU against the oracle.

* rbf_lbm_get_unknown_mask: bit-exact against the oracle's masks for the
  default rule (e_k . n > 0) and the solid check (departure point inside the
  solid), D3Q15 and D3Q19, on an overlapping-sphere cell (r = 0.56) where the
  two rules differ at hundreds of wall nodes.
* Populations after a fixed step count with the solid check, the paper's
  D3Q15 / TRT constants (Lambda = 1, tau+ = 1), switched on after rbf_init:
  FP64 within 1e-9 of the oracle run with the same masks.
* Argument errors: an unknown rule, the solid check without a sphere.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import gpu_or_skip, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbf():
    return gpu_or_skip()


@pytest.fixture(scope="module")
def cell():
    return synth.gaussian_cell(r=0.56, h_min=0.04, seed=3)


def _lbm(rbf, case, q, dx, n_l=25):
    s = rbf.Solver(0)
    s.set_case(case)
    s.build_stencils(n_l)
    s.compute_weights(solver=rbf.RBF_SOLVER_LBM, q=q, dx=dx)
    return s


@pytest.mark.parametrize("q", [15, 19])
def test_masks_bit_exact(rbf, cell, q):
    dx = 0.5 * cell["h_min"]
    s = _lbm(rbf, cell, q, dx)
    normal = oracle.lbm_unknown_normal(cell, q)
    solid = oracle.lbm_unknown_solid(cell, q, dx)
    assert (normal != solid).sum() > 100
    assert np.array_equal(s.lbm_get_unknown_mask(), normal)
    s.lbm_set_unknown_rule(1)
    assert np.array_equal(s.lbm_get_unknown_mask(), solid)
    # the rule persists through a new weight computation at another dx
    s.compute_weights(solver=rbf.RBF_SOLVER_LBM, q=q, dx=0.6 * dx)
    assert np.array_equal(s.lbm_get_unknown_mask(), oracle.lbm_unknown_solid(cell, q, 0.6 * dx))
    s.lbm_set_unknown_rule(0)
    assert np.array_equal(s.lbm_get_unknown_mask(), normal)


@pytest.mark.parametrize("variant", [1, 6])
def test_solid_check_populations_paper_constants(rbf, cell, variant):
    q, tau_p, magic = 15, 1.0, 1.0
    dx = 0.5 * cell["h_min"]
    g = (2e4, 5e3, 0.0)
    s = _lbm(rbf, cell, q, dx)
    s.init(precision=rbf.RBF_FP64, nu=1.0, g=g, tau_plus=tau_p, magic=magic)
    s.set_kernel_variant(variant)
    s.lbm_set_unknown_rule(1)
    n = 40
    s.step(n)
    u = oracle.lbm_units(1.0, tau_p, dx, g)
    idx = oracle.knn(cell["xyz"], cell["xyz"], 25)
    wk = oracle.lbm_weights(cell["xyz"], idx, q, dx)
    tm = oracle.tau_minus(tau_p, magic)
    assert tm == 2.5  # (tau+ - 1/2)(tau- - 1/2) = 1
    f0 = oracle.lbm_equilibrium(q, np.ones(cell.n), np.zeros((cell.n, 3)))
    mask = oracle.lbm_unknown_solid(cell, q, dx)
    fn = oracle.lbm_run(f0, q, cell, idx, wk, tau_p, tm, u["g_lb"], n, unknown=mask)
    want = oracle.lbm_collide(fn, q, tau_p, tm, u["g_lb"])
    _, om, _ = oracle.velocity_set(q)
    got = s.lbm_get_populations()
    assert rel_inf(got - om[:, None], want - om[:, None]) <= 1e-9
    # the default rule gives a different trajectory on this cell
    fd = oracle.lbm_run(f0, q, cell, idx, wk, tau_p, tm, u["g_lb"], n)
    assert rel_inf(fd - om[:, None], fn - om[:, None]) > 1e-6


def test_rule_arguments(rbf, cell):
    s = rbf.Solver(0)
    s.set_nodes(cell["xyz"], cell["type"], cell["normal"])
    s.build_stencils(25)
    s.compute_weights(solver=rbf.RBF_SOLVER_LBM, q=15, dx=0.02)
    with pytest.raises(rbf.RbfError):
        s.lbm_set_unknown_rule(1)       # no sphere
    with pytest.raises(rbf.RbfError):
        s.lbm_set_unknown_rule(2)
    s.lbm_set_unknown_rule(0)
