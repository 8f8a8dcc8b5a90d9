"""rbf_permeability_static: the permeability reduction for callers that cannot
allocate device memory when they call it (their device memory belongs to
another allocator, or cudaMalloc's device-wide synchronisation is not allowed
in their loop).  It must give the same result as rbf_permeability on the same
state, on consecutive calls that reuse its static scratch.

This file is collected last on purpose (test_zz_*): a failure here leaves every
other test already run.  It also passes when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synth
from gpu_common import gpu_or_skip

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("solver", ["acm", "acm_fp32c", "lbm"])
def test_static_permeability_matches_allocating_entry_point(solver):
    rbf = gpu_or_skip()
    case = synth.jittered_cell(r=0.3, n_axis=12, seed=21)
    s = rbf.Solver(0)
    s.set_case(case)
    s.build_stencils(25)
    m_p = 20
    if solver.startswith("acm"):
        rep = s.compute_weights(solver=rbf.RBF_SOLVER_ACM)
        prec = rbf.RBF_FP32C if solver == "acm_fp32c" else rbf.RBF_FP64
        s.init(precision=prec, dt=0.1 * rep["h_min"] ** 2 / 2.0, v_ref=0.01)
        s.step(120)
    else:
        s.compute_weights(solver=rbf.RBF_SOLVER_LBM, q=19, dx=0.5 / 12)
        s.init(precision=rbf.RBF_FP32, g=(3e4, 0.0, 0.0))
        s.step(60)
    # before the probe set exists the static variant refuses (building it allocates)
    with pytest.raises(rbf.RbfError):
        s.permeability_static(m_p)
    k_ref, q_ref = s.permeability(m_p)  # existing entry point (allocating)
    assert k_ref != 0.0
    for _ in range(2):  # two calls in a row share the static scratch
        k, q = s.permeability_static(m_p)
        assert abs(k - k_ref) <= 1e-12 * abs(k_ref)
        assert abs(q - q_ref) <= 1e-12 * abs(q_ref)
    # the state moves on: both entry points follow it
    s.step(10)
    k_ref2, _ = s.permeability(m_p)
    k2, _ = s.permeability_static(m_p)
    assert k_ref2 != k_ref
    assert abs(k2 - k_ref2) <= 1e-12 * abs(k_ref2)
    # through the raw C ABI as well
    L = rbf.lib()
    kk, qq = ctypes.c_double(), ctypes.c_double()
    assert L.rbf_permeability_static(s._h, m_p, ctypes.byref(kk), ctypes.byref(qq)) == rbf.RBF_OK
    assert abs(kk.value - k_ref2) <= 1e-12 * abs(k_ref2)
    # a probe grid that was never built is rejected with a clear error
    assert L.rbf_permeability_static(s._h, m_p + 1, ctypes.byref(kk), ctypes.byref(qq)) == rbf.RBF_EINVAL
    assert b"rbf_permeability" in L.rbf_last_error(s._h)
    s.close()
