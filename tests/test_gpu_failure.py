"""Failure detection of the solvers on the GPU, with no GPU fault: every failure
is made on the host, through the public calls.

* The persistent ACM driver's grid barrier gives up after a wall-clock limit.
  With the limit set to one nanosecond the first block that has to wait for
  the others gives up, raises the launch's error flag, every block leaves its
  step loop at its next barrier and rbf_solve returns RBF_ETIMEOUT.  The
  barrier counters are per launch, so the context stays usable: with the
  default limit restored and the fields re-initialised, a solve matches the
  oracle again.
* Non-finite values written into the fields through rbf_set_fields (ACM) or
  rbf_lbm_set_populations (MLBM) make rbf_solve return RBF_EDIVERGED at its
  next check, and finite fields written afterwards solve normally.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import gpu_or_skip, oracle_acm_setup, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbf():
    return gpu_or_skip()


@pytest.fixture(scope="module")
def cell():
    # 6,857 nodes: 27 blocks of 256 threads in the persistent grid, so blocks wait
    # on each other at every barrier
    return synth.jittered_cell()


def _acm(rbf, case, prec, **kw):
    s = rbf.Solver(0)
    s.set_case(case)
    s.build_stencils(25)
    s.compute_weights(solver=rbf.RBF_SOLVER_ACM)
    s.init(precision=prec, **kw)
    return s


def test_wait_limit_argument_checked(rbf, cell):
    s = _acm(rbf, cell, rbf.RBF_FP64)
    for bad in (0.0, -1.0, 1e-12, 61.0, float("nan")):
        with pytest.raises(rbf.RbfError) as ei:
            s.set_wait_limit(bad)
        assert ei.value.code == rbf.RBF_EINVAL
    s.close()


@pytest.mark.parametrize("code", [256, 4128])  # one node per lane; four lanes per node
def test_grid_barrier_timeout_then_recovery(rbf, cell, code):
    o = oracle_acm_setup(cell, 25)
    dt = oracle.acm_dt(o["h_min"], 1.0)
    s = _acm(rbf, cell, rbf.RBF_FP64, dt=dt, v_ref=2.0)
    s.set_persistent_block(code)
    s.set_wait_limit(1e-9)
    with pytest.raises(rbf.RbfError) as ei:
        s.solve(400, 1e-300, check_every=100)
    assert ei.value.code == rbf.RBF_ETIMEOUT
    assert "barrier" in str(ei.value)
    # default limit, fresh fields: the same context solves and matches the oracle
    s.set_wait_limit(2.0)
    s.init(precision=rbf.RBF_FP64, dt=dt, v_ref=2.0)
    r = s.solve(200, 1e-300, check_every=100)
    assert r["steps"] == 200
    want, _ = oracle.acm_run(cell, o["idx"], o["w4"], o["idxb"], o["wgb"], np.zeros((cell.n, 4)), 200,
                             dt=dt, v_ref=2.0)
    got = s.get_fields()
    for c in range(4):
        assert rel_inf(got[:, c], want[:, c]) <= 1e-9, c
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32c"])
def test_nonfinite_acm_fields_report_divergence(rbf, cell, prec):
    p = {"fp64": rbf.RBF_FP64, "fp32": rbf.RBF_FP32, "fp32c": rbf.RBF_FP32C}[prec]
    s = _acm(rbf, cell, p, v_ref=2.0)
    s.solve(300, 1e-300, check_every=100)
    f = s.get_fields()
    fluid = np.nonzero(cell["type"] == 0)[0]
    bad = f.copy()
    bad[fluid[len(fluid) // 2], 0] = np.nan
    s.set_fields(bad)
    with pytest.raises(rbf.RbfError) as ei:
        s.solve(1000, 1e-300, check_every=50)
    assert ei.value.code == rbf.RBF_EDIVERGED
    # finite fields again: the context solves normally
    s.set_fields(f)
    r = s.solve(100, 1e-300, check_every=50)
    assert r["steps"] == 100 and np.isfinite(s.get_fields()).all()
    bad[fluid[3], 1] = np.inf
    bad[fluid[len(fluid) // 2], 0] = 0.0
    s.set_fields(bad)
    with pytest.raises(rbf.RbfError) as ei:
        s.solve(1000, 1e-300, check_every=50)
    assert ei.value.code == rbf.RBF_EDIVERGED
    s.close()


def test_nonfinite_lbm_populations_report_divergence(rbf, cell):
    s = rbf.Solver(0)
    s.set_case(cell)
    s.build_stencils(25)
    s.compute_weights(solver=rbf.RBF_SOLVER_LBM, q=19, dx=0.0125)
    s.init(precision=rbf.RBF_FP32, g=(1.0, 0.0, 0.0))
    s.step(50)
    f = s.lbm_get_populations()
    bad = f.copy()
    bad[5, cell.n // 2] = np.nan
    s.lbm_set_populations(bad)
    with pytest.raises(rbf.RbfError) as ei:
        s.solve(2000, 1e-300, check_every=100)
    assert ei.value.code == rbf.RBF_EDIVERGED
    s.lbm_set_populations(f)
    r = s.solve(200, 1e-300, check_every=100)
    assert r["steps"] == 200 and np.isfinite(r["k_over_d2"])
    s.close()
