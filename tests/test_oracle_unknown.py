"""Pins of the two unknown-population rules of the MLBM bounce-back (no GPU).

* Default rule (Eq. interpolated_bounceback_mlbm where e_k . n > 0): the mask
  form reproduces the C oracle's built-in normal rule bit for bit in a
  streaming step.
* Solid check of the touching-limit study (departure point x - dx e_k inside
  the solid):
  - on a single sphere (r < 1/2) a wall node x = c + r n has |x - dx e - c|^2 =
    r^2 - 2 dx r (e . n) + dx^2 |e|^2, so k is unknown exactly when
    e . n > dx |e|^2 / (2 r): the closed form, away from the threshold;
  - as dx -> 0 it reduces to the default rule wherever e . n is not near zero;
  - on overlapping spheres (r > 1/2) it agrees with a brute-force search over
    the 27 nearest periodic images, and marks populations whose departure
    point lies in a neighbouring sphere that the normal rule keeps.
"""
import numpy as np
import pytest

import oracle
import synth


def _surface_case(r, h, centre=(0.5, 0.5, 0.5)):
    c = np.asarray(centre, np.float64)
    xyz, nrm = synth.sphere_surface(c, r, h)
    typ = np.ones(len(xyz), np.uint8)
    return synth.Case(xyz=xyz, type=typ, normal=nrm, centre=c, radius=float(r), h_min=h, h_max=h, seed=0,
                      kind="surface")


def _bits(mask, q):
    return ((mask[:, None] >> np.arange(q, dtype=np.uint32)[None, :]) & 1).astype(bool)


@pytest.mark.parametrize("q", [15, 19])
def test_normal_mask_matches_builtin_rule(q):
    case = synth.jittered_cell(r=0.3, n_axis=10, seed=4)
    idx = oracle.knn(case["xyz"], case["xyz"], 20)
    dx = 0.05
    wk = oracle.lbm_weights(case["xyz"], idx, q, dx)
    rng = np.random.default_rng(1)
    fpost = 1.0 + 0.1 * rng.standard_normal((q, case.n))
    a = oracle.lbm_stream(fpost, q, case, idx, wk)
    b = oracle.lbm_stream(fpost, q, case, idx, wk, unknown=oracle.lbm_unknown_normal(case, q))
    assert np.array_equal(a, b)
    # and a mask changes the result where it differs from the rule
    m = oracle.lbm_unknown_normal(case, q)
    wall = np.nonzero(case["type"] == 1)[0]
    m2 = m.copy()
    m2[wall[0]] ^= np.uint32(1 << 1)
    c = oracle.lbm_stream(fpost, q, case, idx, wk, unknown=m2)
    assert not np.array_equal(a[:, wall[0]], c[:, wall[0]])
    assert np.array_equal(np.delete(a, wall[0], 1), np.delete(c, wall[0], 1))


@pytest.mark.parametrize("q", [15, 19])
def test_solid_check_closed_form_single_sphere(q):
    r, dx = 0.3, 0.02
    case = _surface_case(r, 0.01)
    e, _, _ = oracle.velocity_set(q)
    got = _bits(oracle.lbm_unknown_solid(case, q, dx), q)
    n = case["normal"]
    en = n @ e.T                              # (nb, q)
    thr = dx * (e * e).sum(1) / (2.0 * r)     # (q,)
    want = en > thr[None, :]
    clear = np.abs(en - thr[None, :]) > 1e-9
    clear[:, 0] = True
    assert not got[:, 0].any()
    assert np.array_equal(got[clear], want[clear])
    # tangential-ish populations (0 < e.n <= thr) are known under the solid check
    # but unknown under the normal rule: the two rules really differ here
    normal = _bits(oracle.lbm_unknown_normal(case, q), q)
    assert (normal & ~got).any()
    assert not (got & ~normal & clear).any()


@pytest.mark.parametrize("q", [15, 19])
def test_solid_check_small_dx_is_normal_rule(q):
    case = _surface_case(0.3, 0.01)
    e, _, _ = oracle.velocity_set(q)
    en = case["normal"] @ e.T
    got = _bits(oracle.lbm_unknown_solid(case, q, 1e-7), q)
    normal = _bits(oracle.lbm_unknown_normal(case, q), q)
    away = np.abs(en) > 1e-4
    assert np.array_equal(got[away], normal[away])


@pytest.mark.parametrize("q", [15, 19])
def test_solid_check_overlapping_spheres_brute_force(q):
    r, dx = 0.56, 0.03
    case = _surface_case(r, 0.02)
    e, _, _ = oracle.velocity_set(q)
    got = _bits(oracle.lbm_unknown_solid(case, q, dx), q)
    shifts = np.array([[i, j, k] for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)], np.float64)
    want = np.zeros_like(got)
    for kk in range(1, q):
        p = case["xyz"] - dx * e[kk]
        d2 = (((p[:, None, :] - case["centre"][None, None, :] - shifts[None, :, :]) ** 2).sum(2)).min(1)
        want[:, kk] = d2 < r * r
    assert np.array_equal(got, want)
    # nodes near the intersection circles: departure points inside the neighbour
    normal = _bits(oracle.lbm_unknown_normal(case, q), q)
    assert (got & ~normal).any()
