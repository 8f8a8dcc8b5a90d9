"""Pins of the cross-validation quantities (no GPU).

* Eq. pointwise_error: closed forms that a swapped numerator / denominator, a
  non-Euclidean norm or a missing zero guard would break.
* Eq. stopCrit: exact values on a linear and an exponential k(t).
* The Gaussian spacing of Eq. refinement_function as generated by the node
  fill: nearest-neighbour distances follow h(x) across the cell, and the
  node count falls in the range the paper's discretisation gives.
* The oracle's MNS and MLBM, independent discretisations of the same Stokes
  flow, approach each other's steady k/d^2 as the nodes are refined (12 %,
  7 %, 4 % on jittered cells of 1.5k, 3.5k and 6.8k nodes); the flux
  through the five probe planes becomes equal (mass conservation) and the force
  on the grain approaches the body force on the fluid (momentum balance).
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


def _oracle_pair(n_axis, acm_steps, lbm_steps):
    """Both oracle solvers on one jittered cell (r = 0.35), each to a steady state:
    k/d^2 of the MNS and of the MLBM (D3Q15, Lambda = 1, tau+ = 1, dx = h / 2) and
    the relative change of each over its last window."""
    case = synth.jittered_cell(r=0.35, n_axis=n_axis, seed=5)
    n_l = 25
    idx = oracle.knn(case["xyz"], case["xyz"], n_l)
    w4 = oracle.acm_weights(case["xyz"], idx)
    wl, idxb = oracle.neumann_stencils(case, n_l)
    wgb = oracle.neumann_weights(case, idxb)
    dmin = np.linalg.norm(oracle.min_image(case["xyz"][idx[:, 1]] - case["xyz"]), axis=1).min()
    dt = oracle.acm_dt(dmin, 1.0)
    probes = oracle.probe_setup(case["xyz"], case["centre"], case["radius"], 16, n_l)
    # a sound speed (C = beta v_ref = 20) large enough that the pressure relaxes
    # within the run; the steady state does not depend on it
    f = np.zeros((case.n, 4))
    ka = []
    for _ in range(2):
        f, _ = oracle.acm_run(case, idx, w4, idxb, wgb, f, acm_steps // 2, dt=dt, v_ref=2.0)
        ka.append(oracle.permeability(probes, f[:, 0], 1.0, 1.0)[0])
    dx = 0.5 / n_axis
    u = oracle.lbm_units(1.0, 1.0, dx, (1.0, 0.0, 0.0))
    wk = oracle.lbm_weights(case["xyz"], idx, 15, dx)
    fl = oracle.lbm_equilibrium(15, np.ones(case.n), np.zeros((case.n, 3)))
    kl = []
    for _ in range(2):
        fl = oracle.lbm_run(fl, 15, case, idx, wk, 1.0, oracle.tau_minus(1.0, 1.0), u["g_lb"], lbm_steps // 2)
        kl.append(oracle.permeability(probes, oracle.lbm_macro(fl, 15)[:, 0] * u["vel"], 1.0, 1.0)[0])
    def plane_spread(vx):
        # flux through each of the five planes of Eq. k_definition (solid probes 0)
        vals = np.zeros(len(probes["points"]))
        vals[probes["fluid"]] = oracle.apply(probes["idx"], probes["w"], vx)[:, 0]
        per = vals.reshape(5, -1).mean(1)
        return (per.max() - per.min()) / per.mean()

    mac = oracle.lbm_macro(fl, 15)
    spreads = (plane_spread(f[:, 0]), plane_spread(mac[:, 0]))
    # force on the grain over the body force on the fluid, rho |g| phi d^3
    uvwp = oracle.lbm_fields(fl, 15, u)
    phi = oracle.porosity(case["radius"])
    wg = w4[wl][:, :3]
    balance = (oracle.drag(case, idx, wg, f, 1.0)[0] / phi, oracle.drag(case, idx, wg, uvwp, 1.0)[0] / phi)
    return ka[-1], kl[-1], abs(ka[1] - ka[0]) / ka[1], abs(kl[1] - kl[0]) / kl[1], spreads, balance


def test_oracle_solvers_agree_under_refinement():
    """The oracle's two solvers are independent discretisations of the same Stokes
    flow: on the same nodes their steady k/d^2 must approach each other as the
    nodes are refined (the cross-validation of the pointwise comparison section,
    on the CPU).  A dropped term or a wrong unit conversion in either would
    leave a gap that does not shrink."""
    gaps, spreads, balance = [], [], []
    for n_axis, acm_steps, lbm_steps in ((12, 6000, 3000), (16, 10000, 4000), (20, 20000, 6000)):
        ka, kl, da, dl, sp, bal = _oracle_pair(n_axis, acm_steps, lbm_steps)
        assert da < 2e-3 and dl < 2e-3, (n_axis, da, dl)  # both at their steady state
        gaps.append(abs(kl - ka) / ka)
        spreads.append(sp)
        balance.append(bal)
    assert gaps[0] > gaps[1] > gaps[2], gaps
    assert gaps[2] < 0.06, gaps
    # mass conservation: at steady state the same flux crosses every plane; the
    # spread between the planes is discretisation error and shrinks under
    # refinement (MNS 3.3 / 1.9 / 1.3 %, MLBM 1.2 / 0.6 / 0.3 %)
    for s in (0, 1):
        assert spreads[0][s] > spreads[1][s] > spreads[2][s], spreads
    assert spreads[2][0] < 0.02 and spreads[2][1] < 0.01, spreads
    # force balance F_x = rho |g| phi d^3 at steady state, approached under
    # refinement (MNS 0.72 / 0.77 / 0.85, MLBM 0.94 / 0.96 / 0.99): the wall
    # stress quadrature, with the MNS wall gradients the coarser of the two
    for s in (0, 1):
        err = [abs(b[s] - 1.0) for b in balance]
        assert err[0] > err[1] > err[2], balance
    assert abs(balance[2][1] - 1.0) < 0.03 and abs(balance[2][0] - 1.0) < 0.2, balance


def test_acm_steady_state_does_not_depend_on_the_sound_speed():
    """The artificial sound speed C = beta max(max|v|, v_ref) sets how fast the
    MNS pressure relaxes, not where it ends: run long enough, two values of
    v_ref reach the same steady k/d^2, while after a short run the smaller one
    is still far off (the slow transient that the cross-validation avoids with a
    larger v_ref)."""
    case = synth.jittered_cell(r=0.35, n_axis=12, seed=5)
    n_l = 25
    idx = oracle.knn(case["xyz"], case["xyz"], n_l)
    w4 = oracle.acm_weights(case["xyz"], idx)
    _, idxb = oracle.neumann_stencils(case, n_l)
    wgb = oracle.neumann_weights(case, idxb)
    dmin = np.linalg.norm(oracle.min_image(case["xyz"][idx[:, 1]] - case["xyz"]), axis=1).min()
    dt = oracle.acm_dt(dmin, 1.0)
    probes = oracle.probe_setup(case["xyz"], case["centre"], case["radius"], 16, n_l)

    def k_after(v_ref, steps):
        f, _ = oracle.acm_run(case, idx, w4, idxb, wgb, np.zeros((case.n, 4)), steps, dt=dt, v_ref=v_ref)
        return oracle.permeability(probes, f[:, 0], 1.0, 1.0)[0]
    k_fast = k_after(2.0, 8000)
    assert abs(k_after(0.5, 10000) - k_fast) < 1e-3 * k_fast
    assert abs(k_after(0.01, 2000) - k_fast) > 0.3 * k_fast
