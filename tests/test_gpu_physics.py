"""Physics checks of the MLBM on a dilute array, through the C-ABI (GPU).

Hasimoto's dilute expansion for the Stokes drag in a simple-cubic array of
spheres at solid fraction c gives K = 1 / (1 - 1.7601 c^(1/3) + c - 1.5593 c^2
+ ...); the omitted terms are below 1e-5 at c = 0.004 (r = 0.1).  At steady
state the force on the grain balances the body force on the fluid,
F_x = rho |g| phi d^3.  Both hold up to the discretisation and surface
quadrature error, a few per cent on this coarse cell (h_min = 0.02, ~120 wall
nodes); a wrong sign, unit conversion, area or porosity factor would miss them
by far more.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import gpu_or_skip

pytestmark = pytest.mark.gpu


def hasimoto_K(c):
    return 1.0 / (1.0 - 1.7601 * c ** (1.0 / 3.0) + c - 1.5593 * c * c)


def test_dilute_array_drag_and_force_balance():
    rbf = gpu_or_skip()
    from paper_2404_14195_gb300 import crossval
    r = 0.1
    case = synth.gaussian_cell(r=r, h_min=0.02, seed=2)
    s = rbf.Solver(0)
    s.set_case(case)
    s.build_stencils(25)
    s.compute_weights(solver=rbf.RBF_SOLVER_LBM, q=15, dx=0.01)
    s.init(precision=rbf.RBF_FP64, nu=1.0, g=(1.0, 0.0, 0.0), tau_plus=1.0, magic=1.0)
    res = crossval.run_to_steady(s, tol=1e-2, window_steps=10_000, max_steps=1_000_000)
    assert res["converged"]
    F, K = s.drag(32)
    phi = oracle.porosity(r)
    K_h = hasimoto_K(1.0 - phi)
    assert abs(K - K_h) / K_h < 0.08, (K, K_h)
    assert abs(F[0] - phi) / phi < 0.08, (F, phi)
    assert abs(F[1]) < 0.02 * phi and abs(F[2]) < 0.02 * phi
    # the permeability is the same force balance seen through the probes:
    # K = F_x / (6 pi r phi q mu) with q = k nu / |g|
    k, q = s.permeability(32)
    assert K == pytest.approx(F[0] / (6.0 * np.pi * r * phi * q), rel=1e-12)
    s.close()
