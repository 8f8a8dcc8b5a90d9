"""Pins of the oracle's stencils and RBF-FD weights against facts the paper and
the mathematics fix (no GPU).

* kNN: brute-force sort by (distance, index) in numpy; S_i(1) = i.
* Weights (Eqs. operatorApprox, augmentedSystem):
  - reproduction of every monomial of degree <= m (the constraint P^T w = c),
    with the exact operator values taken from sympy's symbolic derivatives;
  - sum rules (derivative weights sum to 0, interpolation weights to 1);
  - the pure-polynomial limit N_L = N_p: on the 7-point star plus three
    diagonal nodes the weights are the textbook 7-point Laplacian and the
    central first differences;
  - exact reproduction of a basis function r^k centred at a stencil node
    (distinguishes the PHS order), interpolated and differentiated;
  - derivative weights equal finite differences of the interpolation weights
    taken with respect to the evaluation point (ties the derivative right-hand
    sides to the interpolation right-hand side);
  - a 50-digit null-space solve (mpmath) of the same saddle problem on tiny
    stencils.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def cell():
    return synth.jittered_cell(r=0.35, n_axis=12, seed=11)


def brute_knn(xyz, q, n_l):
    d = oracle.min_image(xyz[None, :, :] - q[:, None, :])
    d2 = (d * d).sum(-1)
    out = []
    for a in range(len(q)):
        order = np.lexsort((np.arange(len(xyz)), d2[a]))
        out.append(order[:n_l])
    return np.array(out)


def test_knn_matches_brute_force(cell):
    xyz = cell["xyz"]
    idx = oracle.knn(xyz, xyz, 25)
    assert np.array_equal(idx, brute_knn(xyz, xyz, 25))
    assert np.array_equal(idx[:, 0], np.arange(len(xyz)))


def test_grid_knn_equals_brute_force():
    rc = synth.refined_cell(r=0.3, h_min=0.02, h_max=0.06, ramp=0.2, seed=4)
    xyz = rc["xyz"]
    rng = np.random.default_rng(1)
    q = np.concatenate([xyz[::7], rng.random((300, 3))])
    for n_l in (25, 40):
        assert np.array_equal(oracle.knn(xyz, q, n_l, grid=True), oracle.knn(xyz, q, n_l, grid=False))
    lat = synth.lattice(7)
    assert np.array_equal(oracle.knn(lat["xyz"], lat["xyz"], 27, grid=True),
                          oracle.knn(lat["xyz"], lat["xyz"], 27, grid=False))


def test_knn_free_points_and_ties():
    # exact lattice: many equal distances; order must follow the node index
    lat = synth.lattice(6)
    rng = np.random.default_rng(0)
    q = rng.random((40, 3))
    q[:10] = lat["xyz"][:10]  # queries on nodes
    idx = oracle.knn(lat["xyz"], q, 27)
    assert np.array_equal(idx, brute_knn(lat["xyz"], q, 27))


def _mono_values_sympy(m, ops, disp):
    """Exact (L p)(y) for every monomial of degree <= m, via sympy."""
    import sympy as sp
    X, Y, Z = sp.symbols("x y z")
    ex = oracle.monomials(m)
    res = np.zeros((len(ops), len(ex)))
    for e_i, (a, b, c) in enumerate(ex):
        p = X ** int(a) * Y ** int(b) * Z ** int(c)
        for o, (kind, off) in enumerate(ops):
            if kind == oracle.OP_INTERP:
                expr = p
            elif kind in (oracle.OP_DX, oracle.OP_DY, oracle.OP_DZ):
                expr = sp.diff(p, (X, Y, Z)[kind - 1])
            else:
                expr = sp.diff(p, X, 2) + sp.diff(p, Y, 2) + sp.diff(p, Z, 2)
            res[o, e_i] = float(expr.subs({X: off[0], Y: off[1], Z: off[2]}))
    return ex, res


@pytest.mark.parametrize("k,m,n_l", [(3, 2, 25), (5, 3, 40), (3, 1, 12)])
def test_polynomial_reproduction(cell, k, m, n_l):
    xyz = cell["xyz"]
    sel = np.arange(0, len(xyz), 37)
    idx = oracle.knn(xyz, xyz[sel], n_l)
    h = 1.0 / 12
    ops = oracle.ACM_OPS + [(oracle.OP_INTERP, (0.3 * h, -0.2 * h, 0.1 * h)),
                            (oracle.OP_INTERP, (-0.5 * h, 0.0, 0.5 * h))]
    w = oracle.rbf_weights(xyz, xyz[sel], idx, k, m, ops)
    ex, _ = _mono_values_sympy(m, ops, None)
    for s in range(len(sel)):
        d = oracle.min_image(xyz[idx[s]] - xyz[sel[s]])  # displacements from the centre
        P = np.stack([np.prod(d ** e, axis=1) for e in ex], 1)  # (n_l, N_p)
        got = w[s] @ P  # (n_ops, N_p)
        _, want = _mono_values_sympy(m, ops, None) if s == 0 else (None, want)
        scale = np.abs(w[s]).sum(1, keepdims=True) * np.abs(P).max(0, keepdims=True) + 1.0
        assert np.all(np.abs(got - want) <= 1e-11 * scale), (s, np.abs(got - want).max())


def test_sum_rules(cell):
    xyz = cell["xyz"]
    idx = oracle.knn(xyz, xyz, 25)
    w = oracle.acm_weights(xyz, idx)
    scale = np.abs(w).sum(-1)
    assert np.all(np.abs(w.sum(-1)) <= 1e-12 * scale)
    wi = oracle.lbm_weights(xyz, idx, 19, 0.5 / 12)
    assert np.allclose(wi.sum(-1), 1.0, atol=1e-12, rtol=0)


def _star10(h):
    pts = [(0, 0, 0), (h, 0, 0), (-h, 0, 0), (0, h, 0), (0, -h, 0), (0, 0, h), (0, 0, -h),
           (h, h, 0), (h, 0, h), (0, h, h)]
    return np.array(pts, np.float64) + 0.5


def test_pure_polynomial_limit_textbook_stencils():
    # N_L = N_p = 10 (m = 2): the saddle system forces P^T w = c alone, i.e. the
    # unique weights exact on all quadratics - the 7-point Laplacian and central
    # differences, with zero weight on the diagonal nodes.
    h = 0.05
    xyz = _star10(h)
    idx = np.arange(10, dtype=np.int32)[None]
    w = oracle.rbf_weights(xyz, xyz[:1], idx, 3, 2, oracle.ACM_OPS)[0]
    lap = np.array([-6, 1, 1, 1, 1, 1, 1, 0, 0, 0]) / h ** 2
    dx = np.array([0, 1, -1, 0, 0, 0, 0, 0, 0, 0]) / (2 * h)
    dy = np.array([0, 0, 0, 1, -1, 0, 0, 0, 0, 0]) / (2 * h)
    dz = np.array([0, 0, 0, 0, 0, 1, -1, 0, 0, 0]) / (2 * h)
    for got, want in ((w[0], dx), (w[1], dy), (w[2], dz), (w[3], lap)):
        assert np.allclose(got, want, atol=1e-9 * np.abs(want).max(), rtol=0)


@pytest.mark.parametrize("k", [3, 5])
def test_basis_function_reproduction(cell, k):
    # Data u = sum_j lam_j |x - x_j|^k with P^T lam = 0 lie in the space the
    # augmented system reproduces exactly, so every operator is exact on it.
    # Distinguishes the PHS order and ties A and b to the same basis.
    xyz = cell["xyz"]
    sel = np.arange(3, len(xyz), 101)
    n_l = 30
    idx = oracle.knn(xyz, xyz[sel], n_l)
    h = 1.0 / 12
    off = np.array([0.21 * h, -0.33 * h, 0.12 * h])
    ops = [(oracle.OP_INTERP, tuple(off)), (oracle.OP_DX, tuple(off)), (oracle.OP_DY, tuple(off)),
           (oracle.OP_DZ, tuple(off)), (oracle.OP_LAP, tuple(off))]
    w = oracle.rbf_weights(xyz, xyz[sel], idx, k, 2, ops)
    ex = oracle.monomials(2)
    rng = np.random.default_rng(k)
    for s in range(len(sel)):
        d = oracle.min_image(xyz[idx[s]] - xyz[sel[s]])
        P = np.stack([np.prod(d ** e, axis=1) for e in ex], 1)
        q, _ = np.linalg.qr(P, mode="complete")
        lam = q[:, len(ex):] @ rng.standard_normal(n_l - len(ex))  # P^T lam = 0
        R = d[:, None, :] - d[None, :, :]
        u = (np.linalg.norm(R, axis=2) ** k) @ lam
        r = off[None, :] - d
        rn = np.linalg.norm(r, axis=1)
        want = [lam @ rn ** k] + [lam @ (k * rn ** (k - 2) * r[:, a]) for a in range(3)] + \
               [lam @ (k * (k + 1) * rn ** (k - 2))]
        got = w[s] @ u
        scale = np.abs(w[s]).sum(1) * np.abs(u).max()
        assert np.all(np.abs(got - want) <= 1e-11 * scale), (s, got, want)
    # a lone basis function is NOT reproduced (P^T e_j != 0): the test can fail
    d = oracle.min_image(xyz[idx[0]] - xyz[sel[0]])
    u = np.linalg.norm(d - d[7], axis=1) ** k
    assert abs(w[0, 0] @ u - np.linalg.norm(off - d[7]) ** k) > 1e-8


def test_derivatives_are_differences_of_interpolation(cell):
    xyz = cell["xyz"]
    sel = np.arange(5, len(xyz), 89)
    idx = oracle.knn(xyz, xyz[sel], 25)
    h = 1.0 / 12
    y0 = np.array([0.1 * h, 0.2 * h, -0.15 * h])
    eps = 1e-3 * h
    ops = []
    for a in range(3):
        for sgn in (+1, -1):
            ops.append((oracle.OP_INTERP, tuple(y0 + sgn * eps * np.eye(3)[a])))
    ops.append((oracle.OP_INTERP, tuple(y0)))
    ops += [(oracle.OP_DX, tuple(y0)), (oracle.OP_DY, tuple(y0)), (oracle.OP_DZ, tuple(y0)),
            (oracle.OP_LAP, tuple(y0))]
    w = oracle.rbf_weights(xyz, xyz[sel], idx, 3, 2, ops)
    for s in range(len(sel)):
        W = w[s]
        fd = [(W[2 * a] - W[2 * a + 1]) / (2 * eps) for a in range(3)]
        lap = sum((W[2 * a] - 2 * W[6] + W[2 * a + 1]) / eps ** 2 for a in range(3))
        for a in range(3):
            assert np.allclose(fd[a], W[7 + a], atol=1e-5 * np.abs(W[7 + a]).max(), rtol=0)
        assert np.allclose(lap, W[10], atol=1e-3 * np.abs(W[10]).max(), rtol=0)


def _nullspace_weights_mp(d, y, k, m, dps=50):
    """Saddle-point weights by the null-space method in mpmath: w = P^+T c + Z t,
    t solving (Z^T A Z) t = Z^T (b - A w_p).  Unscaled coordinates."""
    import mpmath as mp
    mp.mp.dps = dps
    ex = oracle.monomials(m)
    n = len(d)
    D = [[mp.mpf(float(v)) for v in row] for row in d]
    Y = [mp.mpf(float(v)) for v in y]

    def dist(a, b):
        return mp.sqrt(sum((a[t] - b[t]) ** 2 for t in range(3)))

    A = mp.matrix(n, n)
    for i in range(n):
        for j in range(n):
            A[i, j] = dist(D[i], D[j]) ** k
    P = mp.matrix(n, len(ex))
    for i in range(n):
        for l, e in enumerate(ex):
            P[i, l] = D[i][0] ** int(e[0]) * D[i][1] ** int(e[1]) * D[i][2] ** int(e[2])
    b = mp.matrix(n, 1)
    for i in range(n):
        b[i] = dist(Y, D[i]) ** k
    c = mp.matrix(len(ex), 1)
    for l, e in enumerate(ex):
        c[l] = Y[0] ** int(e[0]) * Y[1] ** int(e[1]) * Y[2] ** int(e[2])
    # QR of P via Gram-Schmidt on the full basis to get Q = [Q1 Z]
    Q, R = mp.qr(P, mode="full")
    np_ = len(ex)
    Q1 = Q[:, :np_]
    Z = Q[:, np_:]
    R1 = R[:np_, :np_]
    wp = Q1 * mp.lu_solve(R1.T, c)
    t = mp.lu_solve(Z.T * A * Z, Z.T * (b - A * wp))
    w = wp + Z * t
    return np.array([float(w[i]) for i in range(n)])


@pytest.mark.parametrize("n_l,m", [(12, 1), (14, 2)])
def test_null_space_high_precision(cell, n_l, m):
    pytest.importorskip("mpmath")
    xyz = cell["xyz"]
    h = 1.0 / 12
    for s in (0, 200, 400):
        idx = oracle.knn(xyz, xyz[s:s + 1], n_l)
        y = np.array([0.3 * h, -0.1 * h, 0.2 * h])
        w = oracle.rbf_weights(xyz, xyz[s:s + 1], idx, 3, m, [(oracle.OP_INTERP, tuple(y))])[0, 0]
        d = oracle.min_image(xyz[idx[0]] - xyz[s])
        ref = _nullspace_weights_mp(d, y, 3, m)
        assert np.abs(w - ref).max() <= 1e-12 * np.abs(ref).max()


def test_singular_stencil_detected():
    # ten coplanar nodes cannot carry the quadratic monomials in z
    g = np.array([(i, j, 0.0) for i in range(4) for j in range(4)], np.float64) * 0.05 + 0.3
    idx = oracle.knn(g, g[:1], 10)
    with pytest.raises(np.linalg.LinAlgError):
        oracle.rbf_weights(g, g[:1], idx, 3, 2, oracle.ACM_OPS)
