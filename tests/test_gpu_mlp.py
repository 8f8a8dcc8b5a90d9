"""GPU parity of the warm-start network (BF16 tensor-core GEMMs) against the FP64
oracle in oracle/mlp.py.

* forward: against the oracle evaluated with the GPU's rounding model (BF16
  weights, inputs and hidden activations, wide accumulation): 2e-3 of the output
  scale;
* gradient: against the FP64 gradient on the same BF16-rounded weights: 3e-2
  norm-wise per layer (BF16 activations and back-propagated errors);
* Adam: the first updates from the same parameters and batches agree with the
  oracle's to 5 % of the step size on parameters with a clear gradient;
* training reduces the loss; the warm start writes the prediction into the solver;
* the fused training kernels and the per-layer GEMM path give the same loss and
  gradient (same rounding points, different summation order).
"""
import numpy as np
import pytest

import oracle
from gpu_common import bf16_forward as _bf16_forward
from gpu_common import gpu_or_skip
from oracle import mlp as om

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbf():
    return gpu_or_skip()


def _data(n, seed=0):
    rng = np.random.default_rng(seed)
    xyz = rng.random((n, 3))
    r = rng.uniform(0.15, 0.6, n)
    sdf = rng.uniform(0.0, 0.4, n)
    X = om.features(xyz, r, sdf)
    # a smooth periodic target field
    T = np.stack([np.sin(2 * np.pi * xyz[:, 0]) * r, np.cos(2 * np.pi * xyz[:, 1]) * sdf,
                  0.3 * np.sin(2 * np.pi * (xyz[:, 0] + xyz[:, 2])), r * sdf], 1)
    return xyz, r, sdf, X, T


def test_forward_matches_bf16_model(rbf):
    m = rbf.Mlp(0)
    theta = om.init_params(5).astype(np.float32).astype(np.float64)
    m.set_params(theta)
    xyz, r, sdf, X, T = _data(1000)
    got = m.predict(xyz, r, sdf)
    want = _bf16_forward(theta, X)
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 2e-3 * scale, np.abs(got - want).max() / scale
    # and a second, deeper check: the FP64 network without rounding is close
    want64 = om.forward(theta, X)[0][:, :4]
    assert np.abs(got - want64).max() <= 3e-2 * np.abs(want64).max()


def test_gradient_matches_oracle(rbf):
    m = rbf.Mlp(0)
    theta = om.init_params(7).astype(np.float32).astype(np.float64)
    m.set_params(theta)
    xyz, r, sdf, X, T = _data(2000, seed=1)
    m.set_data(xyz, r, sdf, T)
    idx = np.arange(256, dtype=np.int64) * 7 % 2000
    g, loss = m.gradient(idx)
    th_b = theta.copy()
    o = 0
    for fo, fi in om.param_sizes():  # oracle on BF16-rounded weights and inputs
        th_b[o:o + fo * fi] = om.bf16_round(theta[o:o + fo * fi])
        o += fo * fi + fo
    loss_o, g_o = om.loss_and_grad(th_b, om.bf16_round(X[idx]), T[idx])
    assert abs(loss - loss_o) <= 2e-2 * loss_o
    o = 0
    for li, (fo, fi) in enumerate(om.param_sizes()):
        for sl in (slice(o, o + fo * fi), slice(o + fo * fi, o + fo * fi + fo)):
            a, b = g[sl], g_o[sl]
            assert np.abs(a - b).max() <= 3e-2 * np.abs(b).max() + 1e-12, (li, np.abs(a - b).max(), np.abs(b).max())
        o += fo * fi + fo


def test_gradient_matches_oracle_many_tiles(rbf):
    """More 128-row tiles than SMs: the forward kernel runs two tile groups per CTA
    and the backward kernel sums the hidden layers' weight gradients over each CTA's
    tiles in tensor memory before reducing them.  Same bars as the small batch."""
    m = rbf.Mlp(0)
    theta = om.init_params(11).astype(np.float32).astype(np.float64)
    m.set_params(theta)
    xyz, r, sdf, X, T = _data(50000, seed=3)
    m.set_data(xyz, r, sdf, T)
    B = 128 * 321  # 321 tiles over at most 152 CTAs: uneven tile counts per group and per CTA
    idx = (np.arange(B, dtype=np.int64) * 7919) % 50000
    g, loss = m.gradient(idx)
    th_b = theta.copy()
    o = 0
    for fo, fi in om.param_sizes():
        th_b[o:o + fo * fi] = om.bf16_round(theta[o:o + fo * fi])
        o += fo * fi + fo
    loss_o, g_o = om.loss_and_grad(th_b, om.bf16_round(X[idx]), T[idx])
    assert abs(loss - loss_o) <= 2e-2 * loss_o
    o = 0
    for li, (fo, fi) in enumerate(om.param_sizes()):
        for sl in (slice(o, o + fo * fi), slice(o + fo * fi, o + fo * fi + fo)):
            a, b = g[sl], g_o[sl]
            assert np.abs(a - b).max() <= 3e-2 * np.abs(b).max() + 1e-12, (li, np.abs(a - b).max(), np.abs(b).max())
        o += fo * fi + fo


def test_adam_steps_match_oracle(rbf):
    m = rbf.Mlp(0)
    theta0 = om.init_params(11).astype(np.float32).astype(np.float64)
    m.set_params(theta0)
    xyz, r, sdf, X, T = _data(4096, seed=2)
    m.set_data(xyz, r, sdf, T)
    B, lr, seed = 512, 1e-3, 99
    hist = m.train(3, B, lr, seed)
    th_gpu = m.get_params().astype(np.float64)
    th = theta0.copy()
    mm = np.zeros_like(th)
    vv = np.zeros_like(th)
    for s in range(3):
        idx = om.batch_indices(seed, s, B, len(xyz))
        th_b = th.copy()
        o = 0
        for fo, fi in om.param_sizes():
            th_b[o:o + fo * fi] = om.bf16_round(th[o:o + fo * fi])
            o += fo * fi + fo
        loss, g = om.loss_and_grad(th_b, om.bf16_round(X[idx]), T[idx])
        if s == 0:
            assert abs(hist[0] - loss) <= 2e-2 * loss
            g0 = g.copy()
        th, mm, vv = om.adam_step(th, g, mm, vv, s + 1, lr)
    d_gpu, d_orc = th_gpu - theta0, th - theta0
    # Adam normalises the step, so a parameter whose gradient is at the BF16 noise
    # level can step +lr or -lr; compare where the first gradient is clearly
    # resolved (above 2 % of its tensor's largest entry)
    clear = np.zeros_like(g0, bool)
    o = 0
    for fo, fi in om.param_sizes():
        for a, b in ((o, o + fo * fi), (o + fo * fi, o + fo * fi + fo)):
            clear[a:b] = np.abs(g0[a:b]) > 0.02 * np.abs(g0[a:b]).max()
        o += fo * fi + fo
    assert clear.sum() > 1000
    assert np.abs(d_gpu[clear] - d_orc[clear]).max() <= 0.05 * 3 * lr
    assert np.median(np.abs(d_gpu - d_orc)) <= 0.01 * lr
    assert np.all(d_gpu[om.n_params() - 16 + 4:] == 0)  # padded output biases stay zero


def test_training_reduces_loss(rbf):
    m = rbf.Mlp(0)
    m.set_params(om.init_params(3).astype(np.float32))
    xyz, r, sdf, X, T = _data(20000, seed=3)
    m.set_data(xyz, r, sdf, T)
    hist = m.train(400, 1024, 2e-3, 5)
    assert np.isfinite(hist).all()
    assert hist[-20:].mean() < 0.2 * hist[:5].mean()
    pred = m.predict(xyz[:500], r[:500], sdf[:500])
    assert np.mean((pred - T[:500]) ** 2) < 0.2 * np.mean(T[:500] ** 2)


def test_fused_and_per_layer_training_paths_agree(rbf):
    theta = om.init_params(13).astype(np.float32)
    xyz, r, sdf, X, T = _data(3000, seed=4)
    idx = (np.arange(512, dtype=np.int64) * 11) % 3000
    out = {}
    for fused in (True, False):
        m = rbf.Mlp(0)
        m.set_fused(fused)
        m.set_params(theta)
        m.set_data(xyz, r, sdf, T)
        out[fused] = m.gradient(idx)
    (g1, l1), (g0, l0) = out[True], out[False]
    assert abs(l1 - l0) <= 1e-5 * l0
    o = 0
    for fo, fi in om.param_sizes():
        for sl in (slice(o, o + fo * fi), slice(o + fo * fi, o + fo * fi + fo)):
            scale = np.abs(g0[sl]).max()
            assert np.abs(g1[sl] - g0[sl]).max() <= 1e-3 * scale + 1e-12, (fo, fi)
        o += fo * fi + fo
    # several training steps of both schedules from the same start stay together
    hist = {}
    for fused in (True, False):
        m = rbf.Mlp(0)
        m.set_fused(fused)
        m.set_params(theta)
        m.set_data(xyz, r, sdf, T)
        hist[fused] = m.train(20, 256, 1e-3, 3)
    assert np.allclose(hist[True], hist[False], rtol=2e-3)
