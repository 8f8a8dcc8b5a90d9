"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same
seeded inputs (small cells spanning many warps/slices with a ragged tail).

Tolerances (norm-wise): weights 1e-10 per node and operator; FP64 fields 1e-9
after a fixed step count; FP32 fields 1e-4; stencils bit-exact.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import gpu_or_skip, oracle_acm_setup, rel_inf, rowwise_rel, small_cell

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbf():
    return gpu_or_skip()


@pytest.fixture(scope="module")
def cell():
    c = small_cell()
    assert c.n % 32 != 0  # ragged last slice
    return c


@pytest.fixture(scope="module")
def orc_acm(cell):
    return oracle_acm_setup(cell, 25)


def make_solver(rbf, case, n_l, solver, **kw):
    s = rbf.Solver(0)
    s.set_case(case)
    s.build_stencils(n_l)
    rep = s.compute_weights(solver=solver, **kw)
    return s, rep


def test_stencils_bit_exact(rbf, cell):
    s, _ = make_solver(rbf, cell, 25, rbf.RBF_SOLVER_ACM)
    want = oracle.knn(cell["xyz"], cell["xyz"], 25)
    got = s.get_stencils()
    assert np.array_equal(got, want)
    # refined cloud (uneven density, free ordering of the input)
    rc = synth.permute(synth.refined_cell(r=0.3, h_min=0.02, h_max=0.06, ramp=0.2, seed=9), 3)
    s2, _ = make_solver(rbf, rc, 30, rbf.RBF_SOLVER_ACM)
    assert np.array_equal(s2.get_stencils(), oracle.knn(rc["xyz"], rc["xyz"], 30))


def test_acm_weights(rbf, cell, orc_acm):
    s, rep = make_solver(rbf, cell, 25, rbf.RBF_SOLVER_ACM)
    assert rep["n_singular"] == 0
    assert abs(rep["h_min"] - orc_acm["h_min"]) <= 1e-15
    for op in range(4):
        got = s.get_weights(op)
        assert rowwise_rel(got, orc_acm["w4"][:, op, :]) <= 1e-10, op


@pytest.mark.parametrize("k,m,n_l", [(5, 3, 40), (3, 1, 12)])
def test_acm_weights_other_orders(rbf, cell, k, m, n_l):
    s, _ = make_solver(rbf, cell, n_l, rbf.RBF_SOLVER_ACM, k=k, m=m)
    idx = oracle.knn(cell["xyz"], cell["xyz"], n_l)
    w = oracle.acm_weights(cell["xyz"], idx, k, m)
    for op in range(4):
        assert rowwise_rel(s.get_weights(op), w[:, op, :]) <= 1e-10, op


@pytest.mark.parametrize("q", [19, 15])
def test_lbm_weights(rbf, cell, q):
    dx = 0.5 * (1.0 / 14)
    s, _ = make_solver(rbf, cell, 25, rbf.RBF_SOLVER_LBM, q=q, dx=dx)
    idx = oracle.knn(cell["xyz"], cell["xyz"], 25)
    wk = oracle.lbm_weights(cell["xyz"], idx, q, dx)
    for k in range(1, q):
        assert rowwise_rel(s.get_weights(rbf.RBF_OP_LBM0 + k), wk[:, k, :]) <= 1e-10, k


# ACM sweep schedules: threads per block + 1000 x lanes per node
@pytest.mark.parametrize("code", [256, 64, 2128, 2256, 4128, 4064])
def test_acm_fp64_fields(rbf, cell, orc_acm, code):
    s, rep = make_solver(rbf, cell, 25, rbf.RBF_SOLVER_ACM)
    s.set_kernel_variant(code)
    dt = oracle.acm_dt(orc_acm["h_min"], 1.0)
    s.init(precision=rbf.RBF_FP64, nu=1.0, g=(1.0, 0.0, 0.0), dt=dt, v_ref=0.01)
    nsteps = 200
    s.step(nsteps)
    got = s.get_fields()
    want, _ = oracle.acm_run(cell, orc_acm["idx"], orc_acm["w4"], orc_acm["idxb"], orc_acm["wgb"],
                             np.zeros((cell.n, 4)), nsteps, dt=dt, v_ref=0.01)
    for c in range(4):
        assert rel_inf(got[:, c], want[:, c]) <= 1e-9, c
    # continuing in a second call (graph replay + eager remainder) stays on the oracle
    s.step(37)
    want2, _ = oracle.acm_run(cell, orc_acm["idx"], orc_acm["w4"], orc_acm["idxb"], orc_acm["wgb"],
                              want, 37, dt=dt, v_ref=0.01)
    got2 = s.get_fields()
    for c in range(4):
        assert rel_inf(got2[:, c], want2[:, c]) <= 1e-9, c


def test_acm_set_fields_restart(rbf, cell, orc_acm):
    s, _ = make_solver(rbf, cell, 25, rbf.RBF_SOLVER_ACM)
    dt = oracle.acm_dt(orc_acm["h_min"], 1.0)
    s.init(precision=rbf.RBF_FP64, dt=dt, v_ref=0.01)
    rng = np.random.default_rng(4)
    start = 0.01 * rng.standard_normal((cell.n, 4))
    start[cell["type"] == 1, :3] = 0.0
    s.set_fields(start)
    s.step(30)
    want, _ = oracle.acm_run(cell, orc_acm["idx"], orc_acm["w4"], orc_acm["idxb"], orc_acm["wgb"], start, 30,
                             dt=dt, v_ref=0.01)
    got = s.get_fields()
    for c in range(4):
        assert rel_inf(got[:, c], want[:, c]) <= 1e-9, c


@pytest.mark.parametrize("code", [256, 2256, 4128])
def test_acm_fp32_fields(rbf, cell, orc_acm, code):
    s, _ = make_solver(rbf, cell, 25, rbf.RBF_SOLVER_ACM)
    s.set_kernel_variant(code)
    dt = oracle.acm_dt(orc_acm["h_min"], 1.0)
    s.init(precision=rbf.RBF_FP32, dt=dt, v_ref=0.01)
    s.step(200)
    got = s.get_fields()
    want, _ = oracle.acm_run(cell, orc_acm["idx"], orc_acm["w4"], orc_acm["idxb"], orc_acm["wgb"],
                             np.zeros((cell.n, 4)), 200, dt=dt, v_ref=0.01)
    for c in range(4):
        assert rel_inf(got[:, c], want[:, c]) <= 1e-4, c



@pytest.mark.parametrize("code", [0, 32, 512, 1256, 3128, 8128, -256])
def test_acm_schedule_code_rejected(rbf, cell, code):
    s, _ = make_solver(rbf, cell, 25, rbf.RBF_SOLVER_ACM)
    with pytest.raises(rbf.RbfError) as ei:
        s.set_kernel_variant(code)
    assert ei.value.code == rbf.RBF_EINVAL

def _lbm_case(rbf, cell, q, prec, g_phys, n_l=25):
    dx = 0.5 * (1.0 / 14)
    s, _ = make_solver(rbf, cell, n_l, rbf.RBF_SOLVER_LBM, q=q, dx=dx)
    s.init(precision=prec, nu=1.0, g=g_phys, tau_plus=0.8, magic=3.0 / 16.0)
    u = oracle.lbm_units(1.0, 0.8, dx, g_phys)
    idx = oracle.knn(cell["xyz"], cell["xyz"], n_l)
    wk = oracle.lbm_weights(cell["xyz"], idx, q, dx)
    return s, u, idx, wk, dx


@pytest.mark.parametrize("q,variant", [(19, 1), (15, 1), (19, 0), (15, 0), (19, 2), (19, 3), (19, 4), (15, 5),
                                       (19, 6), (15, 6), (19, 7), (15, 7), (19, 8), (15, 9),
                                       (19, 10), (15, 10)])
def test_lbm_fp64_populations(rbf, cell, q, variant):
    # g large enough that f - omega is far above rounding (parity of the arithmetic)
    g = (2e4, 5e3, 0.0)
    s, u, idx, wk, dx = _lbm_case(rbf, cell, q, rbf.RBF_FP64, g)
    s.set_kernel_variant(variant)
    tm = oracle.tau_minus(0.8, 3.0 / 16.0)
    f0 = oracle.lbm_equilibrium(q, np.ones(cell.n), np.zeros((cell.n, 3)))
    n = 60
    s.step(n)
    fn = oracle.lbm_run(f0, q, cell, idx, wk, 0.8, tm, u["g_lb"], n)
    want = oracle.lbm_collide(fn, q, 0.8, tm, u["g_lb"])  # the library's state is post-collision
    got = s.lbm_get_populations()
    _, om, _ = oracle.velocity_set(q)
    assert rel_inf(got - om[:, None], want - om[:, None]) <= 1e-9
    # macroscopic fields (physical units) from the pre-collision state
    mac = oracle.lbm_macro(fn, q)
    fields = s.get_fields()
    assert rel_inf(fields[:, :3], mac[:, :3] * u["vel"]) <= 1e-9
    p_want = oracle.lbm_fields(fn, q, u)[:, 3]
    assert rel_inf(fields[:, 3], p_want) <= 1e-8


@pytest.mark.parametrize("variant", [1, 0, 6, 7, 8, 9, 10])
def test_lbm_fp32_populations(rbf, cell, variant):
    q = 19
    g = (2e4, 5e3, 0.0)
    s, u, idx, wk, dx = _lbm_case(rbf, cell, q, rbf.RBF_FP32, g)
    s.set_kernel_variant(variant)
    tm = oracle.tau_minus(0.8, 3.0 / 16.0)
    f0 = oracle.lbm_equilibrium(q, np.ones(cell.n), np.zeros((cell.n, 3)))
    n = 60
    s.step(n)
    fn = oracle.lbm_run(f0, q, cell, idx, wk, 0.8, tm, u["g_lb"], n)
    want = oracle.lbm_collide(fn, q, 0.8, tm, u["g_lb"])
    _, om, _ = oracle.velocity_set(q)
    got = s.lbm_get_populations()
    assert rel_inf(got - om[:, None], want - om[:, None]) <= 1e-4


@pytest.mark.parametrize("variant", [1, 0, 6, 7, 10])
def test_lbm_fp32r_populations(rbf, cell, variant):
    """Refined FP32 (FP64 base + FP32 correction, one FP64 refresh every 64
    steps): after 200 steps (four refreshes) the populations follow the oracle
    within the FP32 bar.  The body force is the paper's scale (g = 1): the
    correction step is the FP32 step linearised about the rest state, accurate
    while the lattice velocities stay small."""
    q = 19
    g = (1.0, 0.0, 0.0)
    s, u, idx, wk, dx = _lbm_case(rbf, cell, q, rbf.RBF_FP32R, g)
    s.set_kernel_variant(variant)
    tm = oracle.tau_minus(0.8, 3.0 / 16.0)
    f0 = oracle.lbm_equilibrium(q, np.ones(cell.n), np.zeros((cell.n, 3)))
    n = 200
    s.step(n)
    fn = oracle.lbm_run(f0, q, cell, idx, wk, 0.8, tm, u["g_lb"], n)
    want = oracle.lbm_collide(fn, q, 0.8, tm, u["g_lb"])
    _, om, _ = oracle.velocity_set(q)
    got = s.lbm_get_populations()
    assert rel_inf(got - om[:, None], want - om[:, None]) <= 1e-4
    fields = s.get_fields()
    assert rel_inf(fields[:, :3], oracle.lbm_fields(fn, q, u)[:, :3]) <= 1e-4


def test_lbm_fp32r_state_round_trip_and_layout_switch(rbf, cell):
    """rbf_lbm_set_populations writes the FP64 base of a refined FP32 state (the
    values come back to FP64 rounding), and a layout switch keeps the state."""
    q, g = 19, (1.0, 0.0, 0.0)
    s, u, idx, wk, dx = _lbm_case(rbf, cell, q, rbf.RBF_FP32R, g)
    s.set_kernel_variant(1)
    s.step(70)
    f = s.lbm_get_populations()
    rng = np.random.default_rng(1)
    x = f + 1e-9 * rng.standard_normal(f.shape)
    s.lbm_set_populations(x)
    assert np.abs(s.lbm_get_populations() - x).max() <= 1e-15
    s.set_kernel_variant(6)  # pairs -> node records
    assert np.abs(s.lbm_get_populations() - x).max() <= 1e-15
    s.step(10)
    assert np.isfinite(s.lbm_get_populations()).all()


@pytest.mark.parametrize("first,second", [(1, 6), (7, 0)])
def test_lbm_layout_switch_mid_run(rbf, cell, first, second):
    """Switching between schedules of the pairs and node-record layouts rewrites
    the state; the run continues on the oracle's trajectory."""
    q, g = 19, (2e4, 5e3, 0.0)
    s, u, idx, wk, dx = _lbm_case(rbf, cell, q, rbf.RBF_FP64, g)
    s.set_kernel_variant(first)
    s.step(25)
    mid = s.lbm_get_populations()
    s.set_kernel_variant(second)
    assert np.array_equal(s.lbm_get_populations(), mid)
    s.step(35)
    tm = oracle.tau_minus(0.8, 3.0 / 16.0)
    f0 = oracle.lbm_equilibrium(q, np.ones(cell.n), np.zeros((cell.n, 3)))
    fn = oracle.lbm_run(f0, q, cell, idx, wk, 0.8, tm, u["g_lb"], 60)
    want = oracle.lbm_collide(fn, q, 0.8, tm, u["g_lb"])
    _, om, _ = oracle.velocity_set(q)
    assert rel_inf(s.lbm_get_populations() - om[:, None], want - om[:, None]) <= 1e-9


def test_permeability_and_drag_fp64(rbf, cell, orc_acm):
    s, _ = make_solver(rbf, cell, 25, rbf.RBF_SOLVER_ACM)
    dt = oracle.acm_dt(orc_acm["h_min"], 1.0)
    s.init(precision=rbf.RBF_FP64, dt=dt, v_ref=0.01)
    s.step(300)
    want, _ = oracle.acm_run(cell, orc_acm["idx"], orc_acm["w4"], orc_acm["idxb"], orc_acm["wgb"],
                             np.zeros((cell.n, 4)), 300, dt=dt, v_ref=0.01)
    m_p = 24
    pr = oracle.probe_setup(cell["xyz"], cell["centre"], cell["radius"], m_p, 25)
    k_want, q_want = oracle.permeability(pr, want[:, 0], 1.0, 1.0)
    k_got, q_got = s.permeability(m_p)
    assert abs(k_got - k_want) <= 1e-9 * abs(k_want)
    F_want = oracle.drag(cell, orc_acm["idx"], orc_acm["w4"][orc_acm["wl"]][:, :3], want, 1.0)
    F_got, K_got = s.drag(m_p)
    assert rel_inf(F_got, F_want) <= 1e-9
    K_want = oracle.drag_coefficient(F_want[0], cell["radius"], q_want, 1.0)
    assert abs(K_got - K_want) <= 1e-9 * abs(K_want)


def test_lbm_drag_fp64(rbf, cell):
    q = 19
    g = (2e4, 0.0, 0.0)
    s, u, idx, wk, dx = _lbm_case(rbf, cell, q, rbf.RBF_FP64, g)
    tm = oracle.tau_minus(0.8, 3.0 / 16.0)
    f0 = oracle.lbm_equilibrium(q, np.ones(cell.n), np.zeros((cell.n, 3)))
    s.step(40)
    fn = oracle.lbm_run(f0, q, cell, idx, wk, 0.8, tm, u["g_lb"], 40)
    uvwp = oracle.lbm_fields(fn, q, u)
    wall = np.nonzero(cell["type"] == 1)[0]
    wg = oracle.rbf_weights(cell["xyz"], cell["xyz"][wall], idx[wall], 3, 2, oracle.ACM_OPS[:3])
    F_want = oracle.drag(cell, idx, wg, uvwp, 1.0)
    F_got, _ = s.drag(16)
    assert rel_inf(F_got, F_want) <= 1e-8
    m_p = 16
    pr = oracle.probe_setup(cell["xyz"], cell["centre"], cell["radius"], m_p, 25)
    k_want, _ = oracle.permeability(pr, uvwp[:, 0], 1.0, float(np.linalg.norm(g)))
    k_got, _ = s.permeability(m_p)
    assert abs(k_got - k_want) <= 1e-8 * abs(k_want)


def test_errors_are_reported(rbf, cell):
    s = rbf.Solver(0)
    with pytest.raises(rbf.RbfError):
        s.step(1)  # nothing set up
    bad = cell["xyz"].copy()
    bad[0, 0] = 1.5
    with pytest.raises(rbf.RbfError):
        s.set_nodes(bad, cell["type"], cell["normal"])
    s.set_case(cell)
    with pytest.raises(rbf.RbfError):
        s.build_stencils(200)
    s.build_stencils(8)
    with pytest.raises(rbf.RbfError):  # N_L < N_p
        s.compute_weights(k=3, m=2)
    # coplanar stencils are singular
    g = np.array([(i, j, 0.0) for i in range(6) for j in range(6)], np.float64) * 0.05 + 0.3
    s2 = rbf.Solver(0)
    s2.set_nodes(g, np.zeros(len(g), np.uint8))
    s2.build_stencils(12)
    with pytest.raises(rbf.RbfError) as ei:
        s2.compute_weights(k=3, m=2)
    assert ei.value.code == rbf.RBF_ESINGULAR


@pytest.mark.parametrize("solver", ["lbm", "acm"])
def test_autotune_keeps_state_and_parity(rbf, cell, orc_acm, solver):
    if solver == "lbm":
        q, g = 19, (2e4, 5e3, 0.0)
        s, u, idx, wk, dx = _lbm_case(rbf, cell, q, rbf.RBF_FP64, g)
        s.step(7)
        before = s.lbm_get_populations()
        times, chosen = s.autotune(10)
        assert len(times) == 11 and chosen in times
        assert np.array_equal(s.lbm_get_populations(), before)
        s.step(23)
        tm = oracle.tau_minus(0.8, 3.0 / 16.0)
        f0 = oracle.lbm_equilibrium(q, np.ones(cell.n), np.zeros((cell.n, 3)))
        fn = oracle.lbm_run(f0, q, cell, idx, wk, 0.8, tm, u["g_lb"], 30)
        want = oracle.lbm_collide(fn, q, 0.8, tm, u["g_lb"])
        _, om, _ = oracle.velocity_set(q)
        assert rel_inf(s.lbm_get_populations() - om[:, None], want - om[:, None]) <= 1e-9
    else:
        s, _ = make_solver(rbf, cell, 25, rbf.RBF_SOLVER_ACM)
        dt = oracle.acm_dt(orc_acm["h_min"], 1.0)
        s.init(precision=rbf.RBF_FP64, dt=dt, v_ref=0.01)
        s.step(5)
        before = s.get_fields()
        times, chosen = s.autotune(10)
        assert set(times) == {256, 128, 64, 2128, 2256, 4128, 4256} and chosen in times
        assert np.array_equal(s.get_fields(), before)
        s.step(25)
        want, _ = oracle.acm_run(cell, orc_acm["idx"], orc_acm["w4"], orc_acm["idxb"], orc_acm["wgb"],
                                 np.zeros((cell.n, 4)), 30, dt=dt, v_ref=0.01)
        got = s.get_fields()
        for c in range(4):
            assert rel_inf(got[:, c], want[:, c]) <= 1e-9, c


@pytest.mark.parametrize("k,m", [(5, 4), (3, 2)])
def test_acm_at_the_largest_stencil(rbf, cell, k, m):
    """The library's maximum sizes: N_L = 64 nearest neighbours and monomials up
    to degree 4 (saddle systems of 64 + 35 = 99 unknowns).  Weights norm-wise per
    node and operator within 1e-10 of the oracle, then 20 FP64 steps of the
    per-sweep kernels and of the persistent driver within 1e-9 of the oracle."""
    n_l = 64
    s, rep = make_solver(rbf, cell, n_l, rbf.RBF_SOLVER_ACM, k=k, m=m)
    assert rep["n_singular"] == 0
    idx = oracle.knn(cell["xyz"], cell["xyz"], n_l)
    assert np.array_equal(s.get_stencils(), idx)
    w4 = oracle.acm_weights(cell["xyz"], idx, k, m)
    for op in range(4):
        assert rowwise_rel(s.get_weights(op), w4[:, op]) <= 1e-10, op
    wl, idxb = oracle.neumann_stencils(cell, n_l)
    wgb = oracle.neumann_weights(cell, idxb, k, m)
    dt = oracle.acm_dt(rep["h_min"], 1.0)
    want, _ = oracle.acm_run(cell, idx, w4, idxb, wgb, np.zeros((cell.n, 4)), 20, dt=dt, v_ref=2.0)
    s.init(precision=rbf.RBF_FP64, dt=dt, v_ref=2.0)
    s.step(20)
    got = s.get_fields()
    s.init(precision=rbf.RBF_FP64, dt=dt, v_ref=2.0)
    assert s.solve(20, 1e-300, check_every=10)["steps"] == 20
    got_p = s.get_fields()
    for c in range(4):
        assert rel_inf(got[:, c], want[:, c]) <= 1e-9, c
        assert rel_inf(got_p[:, c], want[:, c]) <= 1e-9, c


@pytest.mark.parametrize("variant", [1, 6])
def test_lbm_at_the_largest_stencil(rbf, cell, variant):
    """D3Q19 interpolation weights on N_L = 64 stencils (18 right-hand sides per
    node) within 1e-10 of the oracle, and 20 FP64 steps within 1e-9."""
    q, n_l, dx = 19, 64, 0.5 / 14
    g = (2e4, 5e3, 0.0)
    s, _ = make_solver(rbf, cell, n_l, rbf.RBF_SOLVER_LBM, q=q, dx=dx)
    idx = oracle.knn(cell["xyz"], cell["xyz"], n_l)
    wk = oracle.lbm_weights(cell["xyz"], idx, q, dx)
    for kk in (1, 8, 18):
        assert rowwise_rel(s.get_weights(rbf.RBF_OP_LBM0 + kk), wk[:, kk]) <= 1e-10, kk
    s.init(precision=rbf.RBF_FP64, nu=1.0, g=g, tau_plus=0.8, magic=3.0 / 16.0)
    s.set_kernel_variant(variant)
    s.step(20)
    u = oracle.lbm_units(1.0, 0.8, dx, g)
    tm = oracle.tau_minus(0.8, 3.0 / 16.0)
    f0 = oracle.lbm_equilibrium(q, np.ones(cell.n), np.zeros((cell.n, 3)))
    fn = oracle.lbm_run(f0, q, cell, idx, wk, 0.8, tm, u["g_lb"], 20)
    want = oracle.lbm_collide(fn, q, 0.8, tm, u["g_lb"])
    _, om, _ = oracle.velocity_set(q)
    assert rel_inf(s.lbm_get_populations() - om[:, None], want - om[:, None]) <= 1e-9
