"""Full-size checks in the launch configuration the benchmark uses, on samples the
oracle can compute one by one, plus properties that hold at any size.

* config 2 (D3Q19 MLBM, 149,640 nodes, N_L = 30, FP32): stencils of sampled
  nodes bit-exact; their 18 interpolation weight rows to 1e-10; one fused step
  from the GPU's exported state reproduced at the sampled nodes by the oracle's
  streaming + collision (FP32 against FP64: 1e-4 of the populations' deviation
  from the rest state);
* config 4 (ACM, ~3M nodes, PHS r^5, m = 3, N_L = 40, FP32 and FP64): sampled
  stencils and weights (1e-10); every GPU weight row reproduces all monomials of
  degree <= 3; FP32 and FP64 fields agree after a fixed step count.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import gpu_or_skip, rel_inf, rowwise_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbf():
    return gpu_or_skip()


def _sample(case, k, seed):
    rng = np.random.default_rng(seed)
    wall = np.nonzero(case["type"] == 1)[0]
    fluid = np.nonzero(case["type"] == 0)[0]
    return np.sort(np.concatenate([rng.choice(wall, k // 3, replace=False), rng.choice(fluid, k - k // 3, replace=False)]))


def test_config2_lbm_sampled(rbf):
    case = synth.refined_cell(r=0.40, h_min=0.008, h_max=0.04, ramp=0.2, seed=2)
    assert 140000 < case.n < 160000
    q, n_l, dx = 19, 30, 0.004
    s = rbf.Solver(0)
    s.set_case(case)
    s.build_stencils(n_l)
    s.compute_weights(k=3, m=2, solver=rbf.RBF_SOLVER_LBM, q=q, dx=dx)
    s.init(precision=rbf.RBF_FP32, nu=1.0, g=(1.0, 0.0, 0.0), tau_plus=0.8, magic=3.0 / 16.0)
    s.autotune(20)
    rows = _sample(case, 300, 0)
    idx_o = oracle.knn(case["xyz"], case["xyz"][rows], n_l, grid=True)
    idx_g = s.get_stencils()
    assert np.array_equal(idx_g[rows], idx_o)
    wk_o = oracle.rbf_weights(case["xyz"], case["xyz"][rows], idx_o, 3, 2,
                              [(oracle.OP_INTERP, tuple(-dx * e)) for e in oracle.velocity_set(q)[0]])
    for k in range(1, q):
        assert rowwise_rel(s.get_weights(rbf.RBF_OP_LBM0 + k)[rows], wk_o[:, k, :]) <= 1e-10, k
    s.step(300)
    f_n = s.lbm_get_populations()
    s.step(1)
    f_n1 = s.lbm_get_populations()
    u = oracle.lbm_units(1.0, 0.8, dx, (1.0, 0.0, 0.0))
    streamed = oracle.lbm_stream_rows(f_n, q, case, rows, idx_o, wk_o)
    want = oracle.lbm_collide(streamed, q, 0.8, oracle.tau_minus(0.8, 3.0 / 16.0), u["g_lb"])
    _, om, _ = oracle.velocity_set(q)
    dev_got = f_n1[:, rows] - om[:, None]
    dev_want = want - om[:, None]
    assert rel_inf(dev_got, dev_want) <= 1e-4


def test_config4_acm_sampled(rbf):
    case = synth.refined_cell(r=0.45, h_min=0.003, h_max=0.02, ramp=0.32, seed=4)
    assert 2.5e6 < case.n < 3.5e6
    n_l, k, m = 40, 5, 3
    s = rbf.Solver(0)
    s.set_case(case)
    s.build_stencils(n_l)
    rep = s.compute_weights(k=k, m=m, solver=rbf.RBF_SOLVER_ACM)
    assert rep["n_singular"] == 0
    rows = _sample(case, 150, 1)
    idx_o = oracle.knn(case["xyz"], case["xyz"][rows], n_l, grid=True)
    idx_g = s.get_stencils()
    assert np.array_equal(idx_g[rows], idx_o)
    w_o = oracle.rbf_weights(case["xyz"], case["xyz"][rows], idx_o, k, m, oracle.ACM_OPS)
    ex = oracle.monomials(m)
    # polynomial reproduction of every node's weights (a property at any size), checked
    # on a strided subset of all 3M rows plus the sampled rows
    check = np.unique(np.concatenate([rows, np.arange(0, case.n, 997)]))
    d = oracle.min_image(case["xyz"][idx_g[check]] - case["xyz"][check][:, None, :])  # (r, n_l, 3)
    P = np.stack([np.prod(d ** e, axis=2) for e in ex], 2)  # (r, n_l, N_p)
    want_ops = np.zeros((4, len(ex)))
    for l, (a, b, c) in enumerate(ex):  # d/dx, d/dy, d/dz, Laplacian of x^a y^b z^c at 0
        want_ops[0, l] = 1.0 if (a, b, c) == (1, 0, 0) else 0.0
        want_ops[1, l] = 1.0 if (a, b, c) == (0, 1, 0) else 0.0
        want_ops[2, l] = 1.0 if (a, b, c) == (0, 0, 1) else 0.0
        want_ops[3, l] = 2.0 if (a, b, c) in ((2, 0, 0), (0, 2, 0), (0, 0, 2)) else 0.0
    for op in range(4):
        W = s.get_weights(op)
        assert rowwise_rel(W[rows], w_o[:, op, :]) <= 1e-10, op
        Wc = W[check]
        got = np.einsum("rj,rjl->rl", Wc, P)
        scale = np.abs(Wc).sum(1, keepdims=True) * np.abs(P).max(1) + 1.0
        assert np.all(np.abs(got - want_ops[op][None, :]) <= 1e-8 * scale), op
        del W
    # FP32 and FP64 steps from rest agree
    s.init(precision=rbf.RBF_FP64, v_ref=0.01)
    s.step(200)
    f64 = s.get_fields()
    s.init(precision=rbf.RBF_FP32, v_ref=0.01)
    s.step(200)
    f32 = s.get_fields()
    for c in range(3):
        assert rel_inf(f32[:, c], f64[:, c]) <= 1e-4, c
    assert rel_inf(f32[:, 3], f64[:, 3]) <= 1e-3
