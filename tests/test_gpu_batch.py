"""Persistent ACM driver and batched cells against the oracle.

* rbf_solve (one persistent cooperative launch) run for a fixed step count (an
  unreachable tolerance) equals the oracle's MNS steps to 1e-9;
* a batch of cells with different radii and stencil sizes: every cell's weights
  (solved in one launch for all cells) match the oracle to 1e-10 and every
  cell's fields after a fixed step count to 1e-9;
* a convergence run stops each cell at its own step and the cells' results equal
  single-cell solves.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import gpu_or_skip, oracle_acm_setup, rel_inf, rowwise_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbf():
    return gpu_or_skip()


def _cells():
    return [(synth.jittered_cell(r=0.30, n_axis=12, seed=31), 20),
            (synth.jittered_cell(r=0.38, n_axis=13, seed=32), 25),
            (synth.jittered_cell(r=0.22, n_axis=11, seed=33), 30)]


def test_persistent_single_cell_fixed_steps(rbf):
    case = synth.jittered_cell(r=0.35, n_axis=14, seed=5)
    orc = oracle_acm_setup(case, 25)
    s = rbf.Solver(0)
    s.set_case(case)
    s.build_stencils(25)
    s.compute_weights(solver=rbf.RBF_SOLVER_ACM)
    dt = oracle.acm_dt(orc["h_min"], 1.0)
    s.init(precision=rbf.RBF_FP64, dt=dt, v_ref=0.01)
    res = s.solve(150, 1e-300, check_every=50)
    assert res["steps"] == 150 and not res["converged"]
    want, r_o = oracle.acm_run(case, orc["idx"], orc["w4"], orc["idxb"], orc["wgb"], np.zeros((case.n, 4)), 150,
                               dt=dt, v_ref=0.01)
    got = s.get_fields()
    for c in range(4):
        assert rel_inf(got[:, c], want[:, c]) <= 1e-9, c
    assert abs(res["residual"] - r_o[-1]) <= 1e-6 * r_o[-1]
    # the multi-launch path continues seamlessly from the persistent one
    s.step(20)
    want2, _ = oracle.acm_run(case, orc["idx"], orc["w4"], orc["idxb"], orc["wgb"], want, 20, dt=dt, v_ref=0.01)
    got2 = s.get_fields()
    for c in range(4):
        assert rel_inf(got2[:, c], want2[:, c]) <= 1e-9, c


def test_batch_weights_and_fixed_steps(rbf):
    b = rbf.Batch(0)
    cells = _cells()
    for case, n_l in cells:
        b.add_cell(case, n_l)
    rep = b.build(3, 2)
    assert rep["n_singular"] == 0
    b.init(precision=rbf.RBF_FP64, v_ref=0.01)
    res = b.solve(90, 1e-300, check_every=30)
    assert [r["steps"] for r in res] == [90, 90, 90]
    for i, (case, n_l) in enumerate(cells):
        orc = oracle_acm_setup(case, n_l)
        cs = b.cell(i)
        assert np.array_equal(cs.get_stencils(), orc["idx"])
        for op in range(4):
            assert rowwise_rel(cs.get_weights(op), orc["w4"][:, op, :]) <= 1e-10, (i, op)
        dt = oracle.acm_dt(orc["h_min"], 1.0)  # each cell's own dt
        want, _ = oracle.acm_run(case, orc["idx"], orc["w4"], orc["idxb"], orc["wgb"], np.zeros((case.n, 4)), 90,
                                 dt=dt, v_ref=0.01)
        got = cs.get_fields()
        for c in range(4):
            assert rel_inf(got[:, c], want[:, c]) <= 1e-9, (i, c)


def test_batch_converges_per_cell(rbf):
    b = rbf.Batch(0)
    cells = _cells()
    for case, n_l in cells:
        b.add_cell(case, n_l)
    b.build(3, 2)
    b.init(precision=rbf.RBF_FP32, v_ref=0.01)
    res = b.solve(400000, 2e-6, check_every=200, m_p=16)
    assert all(r["status"] == 0 for r in res), res
    assert len({r["steps"] for r in res}) > 1  # cells stop at their own steps
    for i, (case, n_l) in enumerate(cells):
        s = rbf.Solver(0)
        s.set_case(case)
        s.build_stencils(n_l)
        s.compute_weights(solver=rbf.RBF_SOLVER_ACM)
        s.init(precision=rbf.RBF_FP32, v_ref=0.01)
        r1 = s.solve(400000, 2e-6, check_every=200, m_p=16)
        assert r1["converged"] and r1["steps"] == res[i]["steps"]
        assert abs(r1["k_over_d2"] - res[i]["k_over_d2"]) <= 1e-5 * abs(r1["k_over_d2"])


def test_persistent_block_sizes_give_the_same_fields(rbf):
    case = synth.jittered_cell(r=0.35, n_axis=14, seed=5)
    orc = oracle_acm_setup(case, 25)
    dt = oracle.acm_dt(orc["h_min"], 1.0)
    want, _ = oracle.acm_run(case, orc["idx"], orc["w4"], orc["idxb"], orc["wgb"], np.zeros((case.n, 4)), 120,
                             dt=dt, v_ref=0.01)
    s = rbf.Solver(0)
    s.set_case(case)
    s.build_stencils(25)
    s.compute_weights(solver=rbf.RBF_SOLVER_ACM)
    fields = []
    for block in (256, 128, 64, 32, -16, -8):
        s.init(precision=rbf.RBF_FP64, dt=dt, v_ref=0.01)
        s.set_persistent_block(block)
        r = s.solve(120, 1e-300, check_every=40)
        assert r["steps"] == 120
        fields.append(s.get_fields())
    for f in fields[1:]:
        assert np.array_equal(f, fields[0])  # the schedule changes no field arithmetic
    for c in range(4):
        assert rel_inf(fields[0][:, c], want[:, c]) <= 1e-9, c
    # several lanes per node: the stencil sums are split and recombined (rounding only)
    for code in (2128, 4128, 8128, 4256, 8032):
        s.init(precision=rbf.RBF_FP64, dt=dt, v_ref=0.01)
        s.set_persistent_block(code)
        r = s.solve(120, 1e-300, check_every=40)
        assert r["steps"] == 120
        got = s.get_fields()
        for c in range(4):
            assert rel_inf(got[:, c], want[:, c]) <= 1e-9, (code, c)
    # the tuner restores the state and keeps one of the candidates
    before = s.get_fields()
    times, chosen = s.autotune_persistent(50)
    assert {256, 128, 64, 32, 2128, 4128, 8128, 4256} <= set(times) <= {256, 128, 64, 32, 2128, 4128, 8128, 4256,
                                                                           -16, -8} and chosen in times
    assert np.array_equal(s.get_fields(), before)
    s.step(10)
    want2, _ = oracle.acm_run(case, orc["idx"], orc["w4"], orc["idxb"], orc["wgb"], want, 10, dt=dt, v_ref=0.01)
    got2 = s.get_fields()
    for c in range(4):
        assert rel_inf(got2[:, c], want2[:, c]) <= 1e-9, c


def test_batch_more_cells_than_threads_per_block(rbf):
    """40 small cells with 32-thread blocks: block 0's per-cell bookkeeping loops
    over more cells than it has threads."""
    rng = np.random.default_rng(12)
    cells = [(synth.jittered_cell(r=float(r), n_axis=7, seed=700 + i), 20) for i, r in enumerate(rng.uniform(0.2, 0.4, 40))]
    b = rbf.Batch(0)
    for case, n_l in cells:
        b.add_cell(case, n_l)
    assert b.build(3, 2)["n_singular"] == 0
    b.init(precision=rbf.RBF_FP64, v_ref=0.01)
    b.set_persistent_block(32)
    res = b.solve(60, 1e-300, check_every=20)
    assert [r["steps"] for r in res] == [60] * 40
    for i in (0, 17, 33, 39):
        case, n_l = cells[i]
        orc = oracle_acm_setup(case, n_l)
        dt = oracle.acm_dt(orc["h_min"], 1.0)
        want, r_o = oracle.acm_run(case, orc["idx"], orc["w4"], orc["idxb"], orc["wgb"], np.zeros((case.n, 4)), 60,
                                   dt=dt, v_ref=0.01)
        got = b.cell(i).get_fields()
        for c in range(4):
            assert rel_inf(got[:, c], want[:, c]) <= 1e-9, (i, c)
        assert abs(res[i]["residual"] - r_o[-1]) <= 1e-6 * r_o[-1], i
