"""Seeded synthetic inputs shared by the CUDA library and the CPU oracle.

This module generates node clouds and nothing else: it holds none of the
RBF-FD method's arithmetic (no stencils, weights, time steps or reductions).
Both sides of every parity test receive the arrays built here.

Cases are periodic unit cells (d = 1) holding one sphere at the centre — the
simple-cubic sphere array of the paper's case definition section.  Wall
nodes lie exactly on the sphere surface with unit normals pointing out of the
solid into the fluid; fluid nodes fill the rest of the cell.

Recipes (the shapes of the paper's workloads):

* ``jittered_cell``   — regular grid (i+1/2)h jittered by U[-0.2h, 0.2h]^3,
  nodes closer than 0.5h to the wall dropped, plus a Fibonacci surface set of
  round(4 pi r^2 / h^2) nodes.  h = 1/20, r = 0.35 gives about 7k nodes.
* ``refined_cell``    — variable-density advancing-front fill with spacing
  h(d) = h_min + (h_max - h_min) * min(1, d / ramp), d the wall distance,
  seeded by surface nodes at spacing h_min.  h_min = 0.008, h_max = 0.04,
  ramp = 0.2, r = 0.4 gives about 150k nodes.
* ``channel``         — plane Poiseuille channel (walls at y = 0 and y = H,
  periodic in x and z) for the analytic-flow checks.
* ``lattice``         — an exact periodic cubic lattice, on which the meshless
  streaming step reduces to the lattice shift.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nodegen.c")
_LIB = os.path.join(_HERE, "_build", "libnodegen.so")
_lock = threading.Lock()
_lib = None

WALL = 1
FLUID = 0


def build() -> str:
    """Compile the node generator (plain C, a second or so)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.sg_jittered_grid.restype = ctypes.c_int64
            lib.sg_jittered_grid.argtypes = [ctypes.c_int, ctypes.c_double, P, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_uint64, P, ctypes.c_int64]
            lib.sg_sphere_surface.restype = ctypes.c_int64
            lib.sg_sphere_surface.argtypes = [P, ctypes.c_double, ctypes.c_double, P, P, ctypes.c_int64]
            lib.sg_advancing_front.restype = ctypes.c_int64
            lib.sg_advancing_front.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, P, P,
                                               ctypes.c_int64]
            lib.sg_advancing_front_gauss.restype = ctypes.c_int64
            lib.sg_advancing_front_gauss.argtypes = lib.sg_advancing_front.argtypes
            lib.sg_rng_stream.restype = ctypes.c_uint64
            lib.sg_rng_stream.argtypes = [ctypes.c_uint64, ctypes.c_int64, P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def rng_stream(seed: int, n: int) -> np.ndarray:
    """First n outputs of xoshiro256** seeded through SplitMix64 (for tests)."""
    out = np.empty(n, np.uint64)
    _load().sg_rng_stream(seed, n, _ptr(out))
    return out


class Case(dict):
    """A node cloud: xyz (N,3) in [0,1), type (N,) uint8 (0 fluid, 1 wall),
    normal (N,3) (unit on wall nodes, zero on fluid nodes), plus the geometry
    (centre, radius) and the spacing parameters used to build it."""

    @property
    def n(self) -> int:
        return int(self["xyz"].shape[0])


def sphere_surface(centre, r: float, h: float):
    c = np.ascontiguousarray(centre, np.float64)
    cap = int(4 * np.pi * r * r / (h * h)) + 16
    xyz = np.empty((cap, 3), np.float64)
    nrm = np.empty((cap, 3), np.float64)
    m = _load().sg_sphere_surface(_ptr(c), r, h, _ptr(xyz), _ptr(nrm), cap)
    if m < 0:
        raise RuntimeError("sphere_surface: capacity exceeded")
    return xyz[:m].copy(), nrm[:m].copy()


def jittered_cell(r: float = 0.35, n_axis: int = 20, jitter: float = 0.2, drop: float = 0.5,
                  seed: int = 1, centre=(0.5, 0.5, 0.5)) -> Case:
    """Jittered-grid cell with a Fibonacci wall set at the same spacing h = 1/n_axis."""
    h = 1.0 / n_axis
    c = np.ascontiguousarray(centre, np.float64)
    cap = n_axis ** 3
    pts = np.empty((cap, 3), np.float64)
    m = _load().sg_jittered_grid(n_axis, jitter, _ptr(c), r, drop, seed, _ptr(pts), cap)
    if m < 0:
        raise RuntimeError("jittered_grid: capacity exceeded")
    wxyz, wn = sphere_surface(c, r, h) if r > 0 else (np.zeros((0, 3)), np.zeros((0, 3)))
    xyz = np.concatenate([wxyz, pts[:m]])
    typ = np.concatenate([np.full(len(wxyz), WALL, np.uint8), np.full(m, FLUID, np.uint8)])
    nrm = np.concatenate([wn, np.zeros((m, 3))])
    return Case(xyz=np.ascontiguousarray(xyz), type=typ, normal=np.ascontiguousarray(nrm),
                centre=c, radius=float(r), h_min=h, h_max=h, seed=seed, kind="jittered")


def refined_cell(r: float = 0.4, h_min: float = 0.008, h_max: float = 0.04, ramp: float = 0.2,
                 seed: int = 2, wall_gap: float = 0.5, excl: float = 0.87, n_cand: int = 24,
                 centre=(0.5, 0.5, 0.5), cap: int | None = None) -> Case:
    """h-refined cell: wall nodes at spacing h_min, advancing-front fluid fill in which
    no two nodes are closer than ``excl`` times the local spacing."""
    c = np.ascontiguousarray(centre, np.float64)
    wxyz, wn = sphere_surface(c, r, h_min)
    if cap is None:
        cap = int(4.0 / h_min ** 3) + len(wxyz) + 1024
    out = np.empty((cap, 3), np.float64)
    m = _load().sg_advancing_front(_ptr(c), r, h_min, h_max, ramp, wall_gap, excl, n_cand, seed,
                                   len(wxyz), _ptr(np.ascontiguousarray(wxyz)), _ptr(out), cap)
    if m < 0:
        raise RuntimeError(f"advancing_front failed ({m})")
    nb = len(wxyz)
    typ = np.zeros(m, np.uint8)
    typ[:nb] = WALL
    nrm = np.zeros((m, 3))
    nrm[:nb] = wn
    return Case(xyz=out[:m].copy(), type=typ, normal=nrm, centre=c, radius=float(r),
                h_min=h_min, h_max=h_max, seed=seed, kind="refined")


def gaussian_cell(r: float = 0.062, h_min: float = 0.01, h_max: float | None = None, eps: float = 0.295,
                  seed: int = 2, wall_gap: float = 0.5, excl: float = 0.87, n_cand: int = 24,
                  centre=(0.5, 0.5, 0.5), cap: int | None = None) -> Case:
    """h-refined cell with the paper's Gaussian spacing (Eq. refinement_function):
    h = h_max - exp(-t^2 / (2 eps^2)) (h_max - h_min), t = wall distance / (sqrt(3)/2 - r);
    defaults h_max = 2 h_min and eps = 0.295 as in the paper's runs."""
    if h_max is None:
        h_max = 2.0 * h_min
    c = np.ascontiguousarray(centre, np.float64)
    wxyz, wn = sphere_surface(c, r, h_min)
    if cap is None:
        cap = int(4.0 / h_min ** 3) + len(wxyz) + 1024
    out = np.empty((cap, 3), np.float64)
    m = _load().sg_advancing_front_gauss(_ptr(c), r, h_min, h_max, eps, wall_gap, excl, n_cand, seed,
                                         len(wxyz), _ptr(np.ascontiguousarray(wxyz)), _ptr(out), cap)
    if m < 0:
        raise RuntimeError(f"advancing_front_gauss failed ({m})")
    nb = len(wxyz)
    typ = np.zeros(m, np.uint8)
    typ[:nb] = WALL
    nrm = np.zeros((m, 3))
    nrm[:nb] = wn
    return Case(xyz=out[:m].copy(), type=typ, normal=nrm, centre=c, radius=float(r),
                h_min=h_min, h_max=h_max, seed=seed, kind="gaussian")


def channel(h: float = 0.05, H: float = 0.5, jitter: float = 0.2, seed: int = 3) -> Case:
    """Plane channel: wall nodes on y = 0 and y = H (normals +y and -y), fluid nodes
    on a jittered grid strictly inside 0 < y < H; periodic in x and z; the slab
    H < y < 1 is solid and holds no nodes."""
    n = int(round(1.0 / h))
    ny = int(round(H / h))
    xs = (np.arange(n) + 0.5) * h
    wall = []
    nrm = []
    for yw, ny_sign in ((0.0, 1.0), (H, -1.0)):
        X, Z = np.meshgrid(xs, xs, indexing="ij")
        wall.append(np.stack([X.ravel(), np.full(X.size, yw), Z.ravel()], 1))
        nrm.append(np.tile([0.0, ny_sign, 0.0], (X.size, 1)))
    wall = np.concatenate(wall)
    nrm = np.concatenate(nrm)
    # fluid rows at y = j*h, j = 1..ny-1, jittered in all three axes
    u = rng_stream(seed, 3 * n * n * (ny - 1)).astype(np.float64)
    u = (u / 2.0 ** 64) * 2.0 - 1.0
    X, Y, Z = np.meshgrid(xs, np.arange(1, ny) * h, xs, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1) + jitter * h * u.reshape(-1, 3)
    pts[:, 0] %= 1.0
    pts[:, 2] %= 1.0
    xyz = np.concatenate([wall, pts])
    typ = np.concatenate([np.full(len(wall), WALL, np.uint8), np.full(len(pts), FLUID, np.uint8)])
    normal = np.concatenate([nrm, np.zeros_like(pts)])
    return Case(xyz=np.ascontiguousarray(xyz), type=typ, normal=np.ascontiguousarray(normal),
                centre=None, radius=0.0, h_min=h, h_max=h, channel_H=H, seed=seed, kind="channel")


def lattice(n_axis: int = 12) -> Case:
    """All-fluid periodic cubic lattice with spacing 1/n_axis."""
    h = 1.0 / n_axis
    g = np.arange(n_axis) * h
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    return Case(xyz=np.ascontiguousarray(xyz), type=np.zeros(len(xyz), np.uint8),
                normal=np.zeros_like(xyz), centre=None, radius=0.0, h_min=h, h_max=h,
                seed=0, kind="lattice")


def permute(case: Case, seed: int) -> Case:
    """The same cloud with its nodes listed in a seeded random order."""
    rng = np.random.default_rng(seed)
    p = rng.permutation(case.n)
    out = Case(case)
    for key in ("xyz", "type", "normal"):
        out[key] = np.ascontiguousarray(case[key][p])
    return out
