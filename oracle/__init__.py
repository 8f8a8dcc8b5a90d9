"""FP64 CPU oracle for the meshless porous-media solvers of arXiv 2404.14195
(Strzelczyk, Rot, Kosec, Matyka, "Cross-validation of meshless Navier-Stokes
solvers in porous media flows").

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only
callers.  Nothing here is imported by the CUDA library and nothing here
imports it; the two sides share only the seeded node clouds of ``synth``.

The numerical kernels are plain C in ``oracle.c`` (FP64, no fused
multiply-add, node loops in OpenMP); this module loads them with ctypes and
composes the post-processing (probes, permeability, drag) in numpy, each
function citing the paper's equation or section it follows.

Pins (what ties each function to the paper rather than to itself) are in
``tests/test_oracle_*.py``; every function below has at least one.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from math import comb

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

OP_INTERP, OP_DX, OP_DY, OP_DZ, OP_LAP = 0, 1, 2, 3, 4


def build() -> str:
    """Compile the oracle's C kernels (gcc, FP64, -ffp-contract=off, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                               "-ffp-contract=off", "-fopenmp", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
            sig = {
                "orc_knn": [I64, P, I64, P, I, P],
                "orc_knn_grid": [I64, P, I64, P, I, P],
                "orc_monomials": [I, P],
                "orc_rbf_weights": [I64, P, I64, P, I, I, P, I, I, I, P, P, I, P],
                "orc_acm_run": [I64, P, P, I, P, P, I64, P, P, P, P, I, I, P, P, P, P, P],
                "orc_lbm_collide": [I64, I, P, P, P, D, D, P, P, P],
                "orc_lbm_stream": [I64, I, P, P, P, P, P, I, P, P, P, P],
                "orc_lbm_stream_rows": [I64, I64, I, P, P, P, P, P, I, P, P, P, P, P],
                "orc_lbm_run": [I64, I, P, P, P, P, P, P, I, P, P, D, D, P, I, P],
                "orc_lbm_macro": [I64, I, P, P, P],
                "orc_apply": [I64, I, P, I, P, P, P],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ---------------------------------------------------------------------------
# geometry: case definition section (periodic unit cell, d = 1)
# ---------------------------------------------------------------------------
def min_image(d):
    """Displacement to the nearest periodic image (cell side d = 1)."""
    d = np.asarray(d, np.float64)
    return d - np.rint(d)


def sdf(x, centre, r):
    """Signed wall distance phi_sdf (case definition section): distance to the
    nearest periodic image of the sphere centre minus r; negative inside the
    solid.  Exact for r < sqrt(2)/2."""
    d = min_image(np.asarray(x, np.float64) - np.asarray(centre, np.float64))
    return np.sqrt((d * d).sum(-1)) - r


def porosity(r: float) -> float:
    """phi = 1 - |sphere ∩ cell|.  For r > 1/2 the sphere pokes out of the six
    faces; each cap of height h = r - 1/2 (volume pi h^2 (3r - h) / 3) is
    occupied by a neighbouring grain's image and is removed once."""
    v = 4.0 / 3.0 * np.pi * r ** 3
    if r > 0.5:
        h = r - 0.5
        v -= 6.0 * np.pi * h * h * (3.0 * r - h) / 3.0
    return 1.0 - v


def wall_area(r: float) -> float:
    """Area A of the solid walls in one cell (Eq. integration_force's A): sphere
    area minus the six caps' areas 2 pi r h for r > 1/2."""
    a = 4.0 * np.pi * r * r
    if r > 0.5:
        a -= 6.0 * 2.0 * np.pi * r * (r - 0.5)
    return a


# ---------------------------------------------------------------------------
# stencils and weights: meshless discretisation and approximation section
# ---------------------------------------------------------------------------
def knn(xyz, queries, n_l: int, grid=None) -> np.ndarray:
    """S = the n_l nearest nodes of each query by periodic distance, ordered by
    (squared distance, node index).  Queries that are nodes get themselves first
    (S_i(1) = i).  Brute force for small problems; a cell-grid search with the
    same result (grid=True) for large ones."""
    xyz, q = _f64(xyz), _f64(queries)
    out = np.empty((len(q), n_l), np.int32)
    fn = _load().orc_knn if (grid is None and len(xyz) * len(q) <= 4e8) or grid is False else _load().orc_knn_grid
    rc = fn(len(xyz), _p(xyz), len(q), _p(q), n_l, _p(out))
    if rc != 0:
        raise ValueError(f"knn failed ({rc})")
    return out


def monomials(m: int) -> np.ndarray:
    """Exponent triples (a, b, c) of x^a y^b z^c, degree <= m, graded
    lexicographic; N_p = C(m + 3, 3) rows (footnote of the augmented system)."""
    ex = np.empty((comb(m + 3, 3), 3), np.int32)
    np_ = _load().orc_monomials(m, _p(ex))
    assert np_ == len(ex)
    return ex


def n_monomials(m: int) -> int:
    return comb(m + 3, 3)


def rbf_weights(xyz, centres, idx, k: int, m: int, ops, centre_is_node: bool = True,
                refine: int = 2) -> np.ndarray:
    """RBF-FD weights (Eqs. operatorApprox, rbfScaling, augmentedSystem).

    ops: list of (kind, offset) with kind in OP_* and offset = y - x_c, the point
    at which the operator is evaluated relative to the stencil centre.
    Returns w (n_centres, n_ops, n_l).  Raises on singular systems.
    """
    if k < 3 or k % 2 == 0:
        raise ValueError("PHS order k must be odd and >= 3")
    xyz, centres, idx = _f64(xyz), _f64(centres), _i32(idx)
    n_l = idx.shape[1]
    kinds = np.ascontiguousarray([o[0] for o in ops], np.int32)
    offs = _f64(np.array([o[1] for o in ops], np.float64).reshape(len(ops), 3))
    w = np.empty((len(centres), len(ops), n_l), np.float64)
    ns = _load().orc_rbf_weights(len(xyz), _p(xyz), len(centres), _p(centres), int(centre_is_node),
                                 n_l, _p(idx), k, m, len(ops), _p(kinds), _p(offs), refine, _p(w))
    if ns < 0:
        raise ValueError("rbf_weights: bad sizes (N_L + N_p too large or N_L < N_p)")
    if ns > 0:
        raise np.linalg.LinAlgError(f"rbf_weights: {ns} singular stencil systems")
    return w


ACM_OPS = [(OP_DX, (0, 0, 0)), (OP_DY, (0, 0, 0)), (OP_DZ, (0, 0, 0)), (OP_LAP, (0, 0, 0))]


def acm_weights(xyz, idx, k: int = 3, m: int = 2) -> np.ndarray:
    """d/dx, d/dy, d/dz and Laplacian weights at every node (n, 4, n_l)."""
    return rbf_weights(xyz, xyz, idx, k, m, ACM_OPS, True)


def neumann_stencils(case, n_l: int):
    """Neumann stencils of the wall nodes: the wall node itself followed by its
    n_l - 1 nearest fluid nodes (ordered by (distance, node index)).  Returns
    (wall node indices, stencils (n_b, n_l))."""
    typ = np.asarray(case["type"])
    wall = np.nonzero(typ == 1)[0]
    fluid = np.nonzero(typ == 0)[0]
    if len(wall) == 0:
        return wall.astype(np.int32), np.zeros((0, n_l), np.int32)
    nb = knn(case["xyz"][fluid], case["xyz"][wall], n_l - 1)
    return wall.astype(np.int32), np.ascontiguousarray(np.concatenate([wall[:, None], fluid[nb]], 1), np.int32)


def neumann_weights(case, idxb, k: int = 3, m: int = 2):
    """d/dx, d/dy, d/dz weights on the wall nodes' Neumann stencils (n_b, 3, n_l)."""
    wall = np.nonzero(np.asarray(case["type"]) == 1)[0]
    if len(wall) == 0:
        return np.zeros((0, 3, idxb.shape[1]))
    return rbf_weights(case["xyz"], case["xyz"][wall], idxb, k, m, ACM_OPS[:3], True)


# ---------------------------------------------------------------------------
# velocity sets (MLBM section).  D3Q15 is the paper's own table; D3Q19 uses the
# textbook weights 1/3, 1/18, 1/36 (Krueger et al. 2016).  Odd k are listed
# and e_k = -e_{k-1} for even k >= 2, as in the paper's table.
# ---------------------------------------------------------------------------
def velocity_set(q: int):
    if q == 15:
        odd = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1), (1, 1, -1), (1, -1, 1), (1, -1, -1)]
        wts = [2.0 / 9.0] + [1.0 / 9.0] * 6 + [1.0 / 72.0] * 8
    elif q == 19:
        odd = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1),
               (0, 1, 1), (0, 1, -1)]
        wts = [1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12
    else:
        raise ValueError("q must be 15 or 19")
    e = [(0, 0, 0)]
    for v in odd:
        e.append(v)
        e.append(tuple(-c for c in v))
    e = np.array(e, np.float64)
    opp = np.array([0] + [k + 1 if k % 2 == 1 else k - 1 for k in range(1, q)], np.int32)
    return e, np.array(wts, np.float64), opp


def lbm_units(nu: float, tau_plus: float, dx: float, g):
    """Unit conversion, Eqs. lbm_viscosity and conversion_factors:
    nu_lb = c_s^2 (tau+ - 1/2); dt = nu_lb dx^2 / nu; g_lb = g dt^2 / dx."""
    nu_lb = (tau_plus - 0.5) / 3.0
    dt = nu_lb * dx * dx / nu
    g_lb = np.asarray(g, np.float64) * dt * dt / dx
    return dict(nu_lb=nu_lb, dt=dt, g_lb=g_lb, vel=dx / dt, press=(dx / dt) ** 2)


def tau_minus(tau_plus: float, magic: float) -> float:
    """TRT magic parameter Lambda = (tau+ - 1/2)(tau- - 1/2), solved for tau-."""
    return 0.5 + magic / (tau_plus - 0.5)


def lbm_weights(xyz, idx, q: int, dx: float, k: int = 3, m: int = 2) -> np.ndarray:
    """Interpolation weights to the departure points x_i - dx e_k of every node
    (n, q, n_l); entry k = 0 (the rest population) is the centre itself."""
    e, _, _ = velocity_set(q)
    ops = [(OP_INTERP, tuple(-dx * e[kk])) for kk in range(q)]
    return rbf_weights(xyz, xyz, idx, k, m, ops, True)


def lbm_equilibrium(q: int, rho, vel):
    """Eq. feq for arrays rho (n,) and vel (n, 3); returns (q, n)."""
    e, om, _ = velocity_set(q)
    rho = np.asarray(rho, np.float64)
    vel = np.asarray(vel, np.float64).reshape(-1, 3)
    ev = vel @ e.T  # (n, q)
    vv = (vel * vel).sum(1)[:, None]
    feq = rho[:, None] * om[None, :] * (1.0 + 3.0 * ev + 4.5 * ev * ev - 1.5 * vv)
    return np.ascontiguousarray(feq.T)


def lbm_collide(f, q: int, tau_p: float, tau_m: float, g_lb):
    f = _f64(f)
    n = f.shape[1]
    e, om, opp = velocity_set(q)
    out = np.empty_like(f)
    _load().orc_lbm_collide(n, q, _p(e), _p(om), _p(opp), tau_p, tau_m, _p(_f64(g_lb)), _p(f), _p(out))
    return out


def _mask_arg(unknown, rows=None):
    if unknown is None:
        return None, None
    m = np.ascontiguousarray(unknown if rows is None else np.asarray(unknown)[rows], np.uint32)
    return m, _p(m)


def lbm_stream(fpost, q: int, case, idx, wk, unknown=None):
    """Streaming step of Eq. LBM_streaming with the bounce-back of Eq.
    interpolated_bounceback_mlbm at wall nodes; unknown: optional (n,) uint32
    masks (bit k: population k unknown, e.g. lbm_unknown_solid), else the
    normal rule e_k . n > 0."""
    fpost = _f64(fpost)
    n = fpost.shape[1]
    e, _, opp = velocity_set(q)
    out = np.empty_like(fpost)
    keep, mp = _mask_arg(unknown)
    _load().orc_lbm_stream(n, q, _p(e), _p(opp), _p(np.ascontiguousarray(case["type"], np.uint8)),
                           _p(_f64(case["normal"])), mp, idx.shape[1], _p(_i32(idx)), _p(_f64(wk)),
                           _p(fpost), _p(out))
    return out


def lbm_stream_rows(fpost, q: int, case, rows, idx_rows, wk_rows, unknown=None):
    """Streaming (with bounce-back) of the selected nodes `rows` only, from the
    whole post-collision field fpost (q, n); returns (q, len(rows))."""
    fpost = _f64(fpost)
    rows = np.ascontiguousarray(rows, np.int64)
    e, _, opp = velocity_set(q)
    out = np.empty((q, len(rows)))
    typ = np.ascontiguousarray(np.asarray(case["type"])[rows], np.uint8)
    nrm = _f64(np.asarray(case["normal"])[rows])
    keep, mp = _mask_arg(unknown, rows)
    _load().orc_lbm_stream_rows(len(rows), fpost.shape[1], q, _p(e), _p(opp), _p(typ), _p(nrm), mp, idx_rows.shape[1],
                                _p(_i32(idx_rows)), _p(rows), _p(_f64(wk_rows)), _p(fpost), _p(out))
    return out


def lbm_run(f, q: int, case, idx, wk, tau_p: float, tau_m: float, g_lb, nsteps: int, unknown=None):
    """nsteps of COLLIDE then STREAM (MLBM algorithm of the appendix); returns the
    pre-collision populations f (q, n).  unknown: as in lbm_stream."""
    f = _f64(f).copy()
    n = f.shape[1]
    e, om, opp = velocity_set(q)
    keep, mp = _mask_arg(unknown)
    rc = _load().orc_lbm_run(n, q, _p(e), _p(om), _p(opp),
                             _p(np.ascontiguousarray(case["type"], np.uint8)), _p(_f64(case["normal"])), mp,
                             idx.shape[1], _p(_i32(idx)), _p(_f64(wk)), tau_p, tau_m, _p(_f64(g_lb)),
                             nsteps, _p(f))
    if rc:
        raise MemoryError("lbm_run")
    return f


def lbm_unknown_normal(case, q: int) -> np.ndarray:
    """Unknown-population masks of the default rule (Eq.
    interpolated_bounceback_mlbm applied where e_k . n > 0 at wall nodes, n out
    of the solid), as (n,) uint32 with bit k for population k."""
    e, _, _ = velocity_set(q)
    typ = np.asarray(case["type"])
    nrm = np.asarray(case["normal"], np.float64)
    mask = np.zeros(len(typ), np.uint32)
    wall = typ == 1
    for k in range(1, q):
        en = (e[k, 0] * nrm[wall, 0] + e[k, 1] * nrm[wall, 1]) + e[k, 2] * nrm[wall, 2]
        mask[wall] |= (en > 0.0).astype(np.uint32) << np.uint32(k)
    return mask


def lbm_unknown_solid(case, q: int, dx: float) -> np.ndarray:
    """Unknown-population masks of the solid check used in the touching-limit
    study (section on permeability for various porosities): at a wall node x,
    population k is unknown when its departure point x + dx e_k' = x - dx e_k
    lies inside the solid, i.e. strictly closer than r to the nearest sphere
    centre of the periodic array.  (n,) uint32, bit k for population k."""
    e, _, _ = velocity_set(q)
    typ = np.asarray(case["type"])
    xyz = np.asarray(case["xyz"], np.float64)
    c = np.asarray(case["centre"], np.float64)
    r = float(case["radius"])
    mask = np.zeros(len(typ), np.uint32)
    wall = typ == 1
    for k in range(1, q):
        p = xyz[wall] - dx * e[k]
        d = min_image(p - c)
        s = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        mask[wall] |= (s < r * r).astype(np.uint32) << np.uint32(k)
    return mask


def lbm_fields(f, q: int, units):
    """Physical (u, v, w, p) (n, 4) of a pre-collision state f (q, n): velocity of
    Eq. macro_var times dx/dt, and p = rho_ref (dx/dt)^2 c_s^2 (rho - <rho>) /
    <rho> with c_s^2 = 1/3, rho_ref = 1 and <rho> the node mean (Eq.
    conversion_factors with the lattice reference density taken as the current
    mean density: the meshless streaming does not conserve mass, so <rho> drifts
    at the steady state while v does not; f and c f give the same fields).
    units: lbm_units(...)."""
    mac = lbm_macro(f, q)
    rho = mac[:, 3]
    mean = rho.mean()
    out = np.empty((mac.shape[0], 4))
    out[:, :3] = mac[:, :3] * units["vel"]
    out[:, 3] = (rho - mean) / mean / 3.0 * units["press"]
    return out


def lbm_macro(f, q: int):
    """(n, 4) = (vx, vy, vz, rho) per Eq. macro_var."""
    f = _f64(f)
    n = f.shape[1]
    e, _, _ = velocity_set(q)
    out = np.empty((n, 4))
    _load().orc_lbm_macro(n, q, _p(e), _p(f), _p(out))
    return out


# ---------------------------------------------------------------------------
# meshless Navier-Stokes (ACM)
# ---------------------------------------------------------------------------
def acm_dt(h_min: float, nu: float, cfl: float = 0.1) -> float:
    """Time step of the MNS section, dt = 0.1 h_min^2 / (2 nu) (cfl = 0.1)."""
    return cfl * h_min * h_min / (2.0 * nu)


def acm_run(case, idx, w4, idxb, wgb, uvwp, nsteps: int, nu: float = 1.0, g=(1.0, 0.0, 0.0),
            dt: float = None, beta: float = 10.0, v_ref: float = 0.01, rho: float = 1.0, n_p: int = 3):
    """nsteps of the MNS algorithm; uvwp (n, 4) in, (uvwp_out, residual per step) out.
    idxb / wgb: the wall nodes' Neumann stencils and gradient weights."""
    n = len(case["xyz"])
    uvwp = _f64(uvwp)
    u, v, w, p = (np.ascontiguousarray(uvwp[:, c]) for c in range(4))
    prm = _f64([nu, g[0], g[1], g[2], dt, beta, v_ref, rho])
    res = np.zeros(max(nsteps, 1))
    wall = np.ascontiguousarray(np.nonzero(np.asarray(case["type"]) == 1)[0], np.int32)
    _load().orc_acm_run(n, _p(np.ascontiguousarray(case["type"], np.uint8)), _p(_f64(case["normal"])),
                        idx.shape[1], _p(_i32(idx)), _p(_f64(w4)), len(wall), _p(wall), _p(_i32(idxb)),
                        _p(_f64(wgb)), _p(prm), n_p, nsteps, _p(u), _p(v), _p(w), _p(p), _p(res))
    return np.stack([u, v, w, p], 1), res[:nsteps]


def apply(idx, w, u):
    """Eq. operatorApprox: sum_j w_j u_{S(j)} for every centre and operator."""
    idx, w, u = _i32(idx), _f64(w), _f64(u)
    nc, n_ops, n_l = w.shape
    out = np.empty((nc, n_ops))
    _load().orc_apply(nc, n_l, _p(idx), n_ops, _p(w), _p(u), _p(out))
    return out


# ---------------------------------------------------------------------------
# post-processing: permeability (Eq. k_definition) and drag (Eqs.
# stress_tensor_force, integration_force, K_definition)
# ---------------------------------------------------------------------------
PLANES_X = (0.0, 0.2, 0.4, 0.6, 0.8)


def probe_points(m_p: int) -> np.ndarray:
    """Midpoint grid of m_p x m_p points on each of the five planes x = 0, .2, .4,
    .6, .8 of Eq. k_definition; (5 m_p^2, 3), plane-major."""
    s = (np.arange(m_p) + 0.5) / m_p
    Y, Z = np.meshgrid(s, s, indexing="ij")
    pts = [np.stack([np.full(Y.size, x0), Y.ravel(), Z.ravel()], 1) for x0 in PLANES_X]
    return np.concatenate(pts)


def probe_setup(xyz, centre, r, m_p: int, n_l: int, k: int = 3, m: int = 2):
    """Fluid probes, their n_l-nearest stencils and interpolation weights (L = 1,
    centred at the probe, delta = distance to the nearest node).  Probes inside
    the solid carry no stencil (their velocity is zero)."""
    pts = probe_points(m_p)
    fluid = np.ones(len(pts), bool) if centre is None else (sdf(pts, centre, r) >= 0.0)
    fp = pts[fluid]
    idx = knn(xyz, fp, n_l)
    w = rbf_weights(xyz, fp, idx, k, m, [(OP_INTERP, (0, 0, 0))], centre_is_node=False)
    return dict(points=pts, fluid=fluid, idx=idx, w=w)


def permeability(probes, vx, nu: float, g_mag: float) -> float:
    """k/d^2 = q nu / (|g| d^2), q = mean x-velocity over the five planes
    (midpoint rule, solid probes contribute zero), Eq. k_definition with d = 1."""
    vals = apply(probes["idx"], probes["w"], vx)[:, 0]
    q = vals.sum() / len(probes["points"])
    return q * nu / g_mag, q


def drag(case, idx, wgrad_wall, uvwp, nu: float, rho: float = 1.0, area: float = None):
    """Hydrodynamic force on the grain, Eqs. stress_tensor_force and
    integration_force: sigma = -p I + rho nu (grad v + grad v^T) at wall nodes,
    F_i = (A / N_b) sum_b sigma_ij n_j.  wgrad_wall (N_b, 3, n_l) are the d/dx,
    d/dy, d/dz weights of the wall nodes (in the order of np.nonzero(type)).
    area: A (defaults to the sphere's wall area in the cell).

    The pressure enters relative to its mean over the wall nodes.  The exact
    surface integral of a constant pressure over the closed grain surface is
    zero, and the pressure of the incompressible problem is fixed only up to a
    constant; the equal-weight sum over scattered wall nodes does not annul a
    constant (sum_b n_b != 0), so without the shift the force would follow the
    pressure's arbitrary level (in the MNS that level drifts at steady state)."""
    wall = np.nonzero(np.asarray(case["type"]) == 1)[0]
    nb = len(wall)
    if nb == 0:
        return np.zeros(3)
    grad = np.stack([apply(idx[wall], wgrad_wall, uvwp[:, c]) for c in range(3)], 1)  # (nb, comp i, d/dx_j)
    p = uvwp[wall, 3] - uvwp[wall, 3].mean()
    n = np.asarray(case["normal"])[wall]
    sig = -p[:, None, None] * np.eye(3)[None] + rho * nu * (grad + grad.transpose(0, 2, 1))
    f = np.einsum("bij,bj->i", sig, n)
    A = wall_area(case["radius"]) if area is None else area
    return A / nb * f


def drag_coefficient(fx: float, r: float, q: float, nu: float, rho: float = 1.0) -> float:
    """K = F_{H,0} / (6 pi r phi q mu), Eq. K_definition, mu = rho nu."""
    return fx / (6.0 * np.pi * r * porosity(r) * q * rho * nu)


def pointwise_difference(v_a, v_b):
    """Eq. pointwise_error of the pointwise comparison section: per node,
    dv = |v_a - v_b| and delta = dv / |v_b|, |.| the Euclidean norm of the
    velocity vector (the paper takes a = MLBM, b = MNS).  delta is NaN where
    v_b = 0.  v_a, v_b: (n, 3).  Returns (delta, dv)."""
    a = np.asarray(v_a, np.float64)
    b = np.asarray(v_b, np.float64)
    dv = np.sqrt(((a - b) ** 2).sum(1))
    nb = np.sqrt((b * b).sum(1))
    with np.errstate(divide="ignore", invalid="ignore"):
        delta = np.where(nb > 0.0, dv / np.where(nb > 0.0, nb, 1.0), np.nan)
    return delta, dv


def stop_criterion(k_now: float, k_prev: float, window: float) -> float:
    """|Delta|_{k/d^2} of Eq. stopCrit: the change of k/d^2 over the last window
    of physical length `window` (the paper's Delta t = 10^4 delta t), relative
    to the current value and per unit time.  The paper stops once it is below
    10^-2."""
    return abs(k_now - k_prev) / (abs(k_now) * window)
