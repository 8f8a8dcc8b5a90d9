"""FP64 CPU oracle of the learned warm start: Fourier-feature MLP, its gradients
and Adam.  TEST INFRASTRUCTURE ONLY (tests, smoke, bench baselines).

The network is not in the paper; its specification is the build's warm-start
design: inputs are the sines and cosines of 2 pi n.x for 16 integer wave vectors
n (periodic in the unit cell), the grain radius r and the signed wall distance
phi_sdf(x) (34 features, zero-padded to 64); five linear layers
64 -> 128 -> 128 -> 128 -> 128 -> 4 (outputs padded to 16), GELU in its tanh
form after the first four; outputs (u, v, w, p) divided by |g| d^2 / nu; mean
squared error over the four outputs; Adam (Kingma & Ba, ICLR 2015) on FP32
master weights.  Everything here is FP64 and written out directly (no
autograd); pins in tests/test_oracle_mlp.py: central finite differences of the
loss, the Adam update against its closed form on a scalar, feature
periodicity.
"""
from __future__ import annotations

import numpy as np

N_IN = 64          # padded input width (34 used)
N_H = 128          # hidden width
N_OUT = 4          # (u, v, w, p)
N_OUT_PAD = 16     # padded output width
LAYERS = [(N_IN, N_H), (N_H, N_H), (N_H, N_H), (N_H, N_H), (N_H, N_OUT_PAD)]  # (fan_in, fan_out)

# 16 integer wave vectors: the 13 directions of {-1,0,1}^3 up to sign, plus 2 e_a
WAVES = np.array([(1, 0, 0), (0, 1, 0), (0, 0, 1),
                  (1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1), (0, 1, 1), (0, 1, -1),
                  (1, 1, 1), (1, 1, -1), (1, -1, 1), (1, -1, -1),
                  (2, 0, 0), (0, 2, 0), (0, 0, 2)], np.float64)

GELU_C = np.sqrt(2.0 / np.pi)


def features(xyz, r, sdf):
    """(n, 64): [sin 2pi n.x, cos 2pi n.x] for the 16 wave vectors interleaved
    (column 2j = sin, 2j+1 = cos), column 32 = r, column 33 = sdf, rest 0."""
    xyz = np.asarray(xyz, np.float64)
    ph = 2.0 * np.pi * (xyz @ WAVES.T)  # (n, 16)
    X = np.zeros((len(xyz), N_IN))
    X[:, 0:32:2] = np.sin(ph)
    X[:, 1:32:2] = np.cos(ph)
    X[:, 32] = np.broadcast_to(np.asarray(r, np.float64), (len(xyz),))
    X[:, 33] = np.asarray(sdf, np.float64)
    return X


def gelu(z):
    t = np.tanh(GELU_C * (z + 0.044715 * z ** 3))
    return 0.5 * z * (1.0 + t)


def gelu_prime(z):
    t = np.tanh(GELU_C * (z + 0.044715 * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_C * (1.0 + 3.0 * 0.044715 * z * z)


def param_sizes():
    """Packed parameter vector: for each layer W (fan_out x fan_in, row-major)
    then b (fan_out)."""
    return [(fo, fi) for fi, fo in LAYERS]


def n_params():
    return sum(fo * fi + fo for fo, fi in param_sizes())


def unpack(theta):
    out, o = [], 0
    for fo, fi in param_sizes():
        W = theta[o:o + fo * fi].reshape(fo, fi)
        o += fo * fi
        b = theta[o:o + fo]
        o += fo
        out.append((W, b))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


def init_params(seed: int):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases; padded
    inputs (columns 34..63 of W1) and padded outputs (rows 4..15 of W5) zero."""
    rng = np.random.default_rng(seed)
    layers = []
    for li, (fo, fi) in enumerate(param_sizes()):
        fan = 34 if li == 0 else fi
        W = rng.uniform(-1.0, 1.0, (fo, fi)) / np.sqrt(fan)
        if li == 0:
            W[:, 34:] = 0.0
        if li == 4:
            W[N_OUT:, :] = 0.0
        layers.append((W, np.zeros(fo)))
    return pack(layers)


def forward(theta, X):
    """Returns the output (n, 16) and the cache of pre-activations Z and inputs H."""
    H = [X]
    Z = []
    L = unpack(theta)
    for li, (W, b) in enumerate(L):
        z = H[-1] @ W.T + b
        Z.append(z)
        if li < len(L) - 1:
            H.append(gelu(z))
    return Z[-1], (H, Z)


def loss_and_grad(theta, X, T):
    """MSE over the 4 real outputs, (1 / (n * 4)) sum (y - t)^2, and its gradient
    by back-propagation (written out layer by layer)."""
    n = len(X)
    Y, (H, Z) = forward(theta, X)
    E = Y[:, :N_OUT] - T
    loss = (E * E).sum() / (n * N_OUT)
    dY = np.zeros_like(Y)
    dY[:, :N_OUT] = 2.0 * E / (n * N_OUT)
    L = unpack(theta)
    grads = [None] * len(L)
    d = dY
    for li in range(len(L) - 1, -1, -1):
        W, b = L[li]
        gW = d.T @ H[li]
        gb = d.sum(0)
        if li == 4:
            gW[N_OUT:, :] = 0.0
            gb[N_OUT:] = 0.0
        grads[li] = (gW, gb)
        if li > 0:
            d = (d @ W) * gelu_prime(Z[li - 1])
    g = pack(grads)
    return loss, g


def adam_step(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba): bias-corrected first and second moments."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    theta = theta - lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m, v


def bf16_round(a):
    """Round FP64 values to the nearest bfloat16 (ties to even), returned as FP64."""
    a32 = np.asarray(a, np.float64).astype(np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def splitmix64(x):
    """SplitMix64 output for the 64-bit counters x (Steele, Lea & Flood 2014),
    the counter-based generator both sides use to draw mini-batches."""
    x = (np.asarray(x, np.uint64) + np.uint64(0x9E3779B97F4A7C15))
    with np.errstate(over="ignore"):
        z = x
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def batch_indices(seed: int, step: int, batch: int, n: int):
    """Sample indices of mini-batch `step`: splitmix64(seed * 2^32 + step * batch + i) mod n."""
    c = np.uint64(seed) * np.uint64(1 << 32) + np.uint64(step) * np.uint64(batch) + np.arange(batch, dtype=np.uint64)
    return (splitmix64(c) % np.uint64(n)).astype(np.int64)
