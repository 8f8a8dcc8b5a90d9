"""Compensated FP32 ACM state (RBF_FP32C) against the FP64 oracle.

* From rest, a fixed step count through the graph-captured multi-launch steps and
  through the persistent driver: fields within 1e-4 of the oracle (the FP32 bar).
* rbf_set_fields / rbf_get_fields keep a value to the pair's ~2^-48.
* Sub-ulp increments: from a state of magnitude ~1 with a time step so small that
  each step changes most fields by far less than half a float ulp, plain FP32
  does not move (every update rounds back to the old value) while the pairs
  accumulate the oracle's displacement.
* A warm start into an RBF_FP32C context clears the low words.
"""
import numpy as np
import pytest

import oracle
from gpu_common import gpu_or_skip, oracle_acm_setup, rel_inf, small_cell

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbf():
    return gpu_or_skip()


@pytest.fixture(scope="module")
def cell():
    return small_cell()


@pytest.fixture(scope="module")
def orc(cell):
    return oracle_acm_setup(cell, 25)


def _solver(rbf, case, prec, **kw):
    s = rbf.Solver(0)
    s.set_case(case)
    s.build_stencils(25)
    s.compute_weights(solver=rbf.RBF_SOLVER_ACM)
    s.init(precision=prec, **kw)
    return s


def test_fp32c_fixed_steps_multilaunch_and_persistent(rbf, cell, orc):
    dt = oracle.acm_dt(orc["h_min"], 1.0)
    want, _ = oracle.acm_run(cell, orc["idx"], orc["w4"], orc["idxb"], orc["wgb"], np.zeros((cell.n, 4)), 200,
                             dt=dt, v_ref=0.01)
    a = _solver(rbf, cell, rbf.RBF_FP32C, dt=dt, v_ref=0.01)
    a.step(200)
    b = _solver(rbf, cell, rbf.RBF_FP32C, dt=dt, v_ref=0.01)
    r = b.solve(200, 1e-300, check_every=50)
    assert r["steps"] == 200
    c = _solver(rbf, cell, rbf.RBF_FP32C, dt=dt, v_ref=0.01)
    c.set_persistent_block(4128)  # four lanes per node
    assert c.solve(200, 1e-300, check_every=50)["steps"] == 200
    d = _solver(rbf, cell, rbf.RBF_FP32C, dt=dt, v_ref=0.01)
    d.set_kernel_variant(2128)  # multi-launch sweeps, two lanes per node
    d.step(200)
    for s in (a, b, c, d):
        got = s.get_fields()
        for c in range(4):
            assert rel_inf(got[:, c], want[:, c]) <= 1e-4, c


def test_fp32c_field_round_trip(rbf, cell):
    s = _solver(rbf, cell, rbf.RBF_FP32C, v_ref=0.01)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((cell.n, 4))
    x[cell["type"] == 1, :3] = 0.0
    s.set_fields(x)
    y = s.get_fields()
    assert np.all(np.abs(y - x) <= 2.0 ** -46 * np.abs(x))
    # plain FP32 keeps only ~2^-24
    s32 = _solver(rbf, cell, rbf.RBF_FP32, v_ref=0.01)
    s32.set_fields(x)
    assert np.abs(s32.get_fields() - x).max() > 2.0 ** -30 * np.abs(x).max()


def test_fp32c_accumulates_sub_ulp_increments(rbf, cell, orc):
    dt0 = oracle.acm_dt(orc["h_min"], 1.0)
    base, _ = oracle.acm_run(cell, orc["idx"], orc["w4"], orc["idxb"], orc["wgb"], np.zeros((cell.n, 4)), 300,
                             dt=dt0, v_ref=0.01)
    fluid = cell["type"] == 0
    start = base / np.abs(base[:, :3]).max()  # |v| up to 1: half an ulp ~ 3e-8 near the maximum
    # size the step from the oracle's one-step change: median relative change 1e-9
    probe_dt = 1e-12
    one, _ = oracle.acm_run(cell, orc["idx"], orc["w4"], orc["idxb"], orc["wgb"], start, 1, dt=probe_dt,
                            v_ref=0.01)
    big = fluid & (np.abs(start[:, 0]) > 0.1)
    ratio = np.median(np.abs(one[big, 0] - start[big, 0]) / np.abs(start[big, 0]))
    assert ratio > 0
    dt = probe_dt * 1e-9 / ratio
    K = 1000
    want, _ = oracle.acm_run(cell, orc["idx"], orc["w4"], orc["idxb"], orc["wgb"], start, K, dt=dt, v_ref=0.01)
    D = want[:, 0] - start[:, 0]
    sel = big & (np.abs(D) > 1e-3 * np.abs(D[big]).max())
    assert sel.sum() > 100

    def median_rel(prec):
        s = _solver(rbf, cell, prec, dt=dt, v_ref=0.01)
        s.set_fields(start)
        s0 = s.get_fields()[:, 0]  # the start as the precision holds it
        s.step(K)
        d = s.get_fields()[:, 0] - s0
        return np.median(np.abs(d[sel] - D[sel]) / np.abs(D[sel]))

    e32 = median_rel(rbf.RBF_FP32)
    e32c = median_rel(rbf.RBF_FP32C)
    assert e32 > 0.5, e32      # plain FP32 stalls
    assert e32c < 1e-2, e32c   # the pairs follow the oracle


def test_warm_start_clears_low_words(rbf, cell):
    from oracle import mlp as om
    m = rbf.Mlp(0)
    m.set_params(np.asarray(om.init_params(2), np.float32))
    rng = np.random.default_rng(8)
    junk = 1e-3 * rng.standard_normal((cell.n, 4))
    junk[cell["type"] == 1, :3] = 0.0
    got = []
    for prec in (rbf.RBF_FP32, rbf.RBF_FP32C):
        s = _solver(rbf, cell, prec, v_ref=0.01)
        s.set_fields(1.0 + junk)
        m.warm_start(s, (1.0, 2.0, 3.0, 4.0))
        got.append(s.get_fields())
    assert np.array_equal(got[0], got[1])
    pred = m.predict(cell["xyz"], np.full(cell.n, cell["radius"]),
                     (np.sqrt(((cell["xyz"] - cell["centre"] - np.rint(cell["xyz"] - cell["centre"])) ** 2).sum(1))
                      - cell["radius"]).astype(np.float32))
    fl = cell["type"] == 0
    for c in range(4):
        rows = fl if c < 3 else slice(None)
        want = (c + 1.0) * pred[rows, c].astype(np.float64)
        assert np.abs(got[0][rows, c] - want).max() <= 1e-4 * np.abs(want).max(), c
    assert np.all(got[0][~fl, :3] == 0.0)
