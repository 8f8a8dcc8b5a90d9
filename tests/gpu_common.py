"""Shared helpers of the GPU parity tests: library build/load, case set-up on
both sides, and the norm-wise comparison the tolerances refer to."""
import numpy as np
import pytest

import oracle
import synth


def gpu_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_14195_gb300 as rbf
    rbf._build.build()
    return rbf


def rel_inf(a, b):
    """||a - b||_inf / ||b||_inf."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def rowwise_rel(a, b):
    """max over rows of ||a_r - b_r||_inf / ||b_r||_inf (norm-wise per node)."""
    num = np.abs(a - b).max(axis=-1)
    den = np.abs(b).max(axis=-1)
    den = np.where(den > 0, den, 1.0)
    return (num / den).max()


def small_cell(r=0.35, n_axis=14, seed=5):
    return synth.jittered_cell(r=r, n_axis=n_axis, seed=seed)


def oracle_acm_setup(case, n_l, k=3, m=2):
    idx = oracle.knn(case["xyz"], case["xyz"], n_l)
    w4 = oracle.acm_weights(case["xyz"], idx, k, m)
    wl, idxb = oracle.neumann_stencils(case, n_l)
    wgb = oracle.neumann_weights(case, idxb, k, m)
    dmin = np.linalg.norm(oracle.min_image(case["xyz"][idx[:, 1]] - case["xyz"]), axis=1).min()
    return dict(idx=idx, w4=w4, wl=wl, idxb=idxb, wgb=wgb, h_min=dmin)


def bf16_forward(theta, X):
    """The warm-start network's output (n, 4) with the GPU kernels' rounding points:
    BF16 inputs, weights and hidden activations, wide accumulation, FP32 bias
    (the FP64 layers of oracle/mlp.py with BF16 rounding inserted)."""
    from oracle import mlp as om
    L = om.unpack(theta)
    h = om.bf16_round(X)
    for li, (W, b) in enumerate(L):
        z = h @ om.bf16_round(W).T + b
        if li < 4:
            h = om.bf16_round(om.gelu(z))
    return z[:, :4]
