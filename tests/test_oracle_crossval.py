"""Pins of the cross-validation quantities (no GPU).

* Eq. pointwise_error: closed forms that a swapped numerator / denominator, a
  non-Euclidean norm or a missing zero guard would break.
* Eq. stopCrit: exact values on a linear and an exponential k(t).
* The Gaussian spacing of Eq. refinement_function as generated by the node
  fill: nearest-neighbour distances follow h(x) across the cell, and the
  node count falls in the range the paper's discretisation gives.
"""
import numpy as np

import oracle
import synth


def test_pointwise_closed_forms():
    b = np.array([[3.0, 4.0, 0.0], [1.0, 0.0, 0.0], [0.0, 2.0, 0.0], [0.0, 0.0, 0.0], [1.0, -2.0, 2.0]])
    a = np.array([[0.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 4.0, 0.0], [1.0, 0.0, 0.0], [1.0, -2.0, 2.0]])
    delta, dv = oracle.pointwise_difference(a, b)
    # |(3,4,0)| = 5 (Euclidean; the max norm would give 4)
    assert dv[0] == 5.0 and delta[0] == 1.0
    # orthogonal vectors of equal length: |a - b| = sqrt(2) |b|
    assert abs(delta[1] - np.sqrt(2.0)) < 1e-15
    # a = 2 b: delta = 1 with b in the denominator, 0.5 if the roles were swapped
    assert delta[2] == 1.0 and dv[2] == 2.0
    d_swap, _ = oracle.pointwise_difference(b[2:3], a[2:3])
    assert d_swap[0] == 0.5
    # v_b = 0: undefined
    assert np.isnan(delta[3]) and dv[3] == 1.0
    # identical vectors
    assert delta[4] == 0.0 and dv[4] == 0.0


def test_stop_criterion_exact():
    # linear k(t) = a + b t: |Delta| = b / k(t) for any window (to the rounding of
    # the difference of two close values)
    a, b = 0.02, 3e-4
    for t, w in [(1.0, 0.1), (5.0, 2.0)]:
        want = b / (a + b * t)
        assert abs(oracle.stop_criterion(a + b * t, a + b * (t - w), w) - want) < 1e-10 * want
    # relaxation k(t) = k_inf (1 - exp(-t / tau))
    k_inf, tau, w = 0.03, 0.2, 0.05
    k = lambda t: k_inf * (1.0 - np.exp(-t / tau))
    t = 1.3
    want = k_inf * np.exp(-t / tau) * (np.exp(w / tau) - 1.0) / (k(t) * w)
    assert abs(oracle.stop_criterion(k(t), k(t - w), w) - want) < 1e-12 * want


def _nn_over_h(case):
    from scipy.spatial import cKDTree
    x = np.mod(case["xyz"], 1.0)
    d, _ = cKDTree(x, boxsize=1.0).query(x, 2)
    s = oracle.sdf(x, case["centre"], case["radius"])
    t = s / (np.sqrt(3.0) / 2.0 - case["radius"])
    h = case["h_max"] - np.exp(-t * t / (2.0 * 0.295 ** 2)) * (case["h_max"] - case["h_min"])
    return d[:, 1] / h, t


def test_gaussian_refinement_spacing():
    c = synth.gaussian_cell(r=0.062, h_min=0.02, seed=3)
    # Eq. refinement_function with h_max = 2 h_min, eps = 0.295: N ~ 3e4 at h_min = 0.02
    assert 2.0e4 < c.n < 4.0e4
    ratio, t = _nn_over_h(c)
    fl = np.asarray(c["type"]) == 0
    for lo, hi in [(0.0, 0.1), (0.2, 0.4), (0.5, 0.7), (0.8, 1.0)]:
        m = fl & (t >= lo) & (t < hi)
        assert m.sum() > 100
        med = np.median(ratio[m])
        assert 0.8 < med < 1.0, (lo, hi, med)
    # the spacing really varies: far nodes about twice as far apart as near ones
    near = np.median((ratio * (0.04 - np.exp(-t * t / (2 * 0.295 ** 2)) * 0.02))[fl & (t < 0.1)])
    far = np.median((ratio * (0.04 - np.exp(-t * t / (2 * 0.295 ** 2)) * 0.02))[fl & (t > 0.8)])
    assert 1.6 < far / near < 2.4
    # large-sphere cell: wall nodes only outside the other periodic images
    c2 = synth.gaussian_cell(r=0.6526, h_min=0.02, seed=3)
    w = np.asarray(c2["type"]) == 1
    assert np.all(oracle.sdf(c2["xyz"][w], c2["centre"], c2["radius"]) > -1e-9)
    assert np.all(oracle.sdf(c2["xyz"][~w], c2["centre"], c2["radius"]) > 0.0)
