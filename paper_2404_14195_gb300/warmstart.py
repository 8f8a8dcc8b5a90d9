"""Learned warm start of the steady ACM solve: training data from steady fields
the solver itself produces, training of the network, and evaluation against a
zero start.  Orchestration only: every solve, the training and the inference run
in the library's kernels (rbf_batch_*, rbf_mlp_*)."""
from __future__ import annotations

import time

import numpy as np

from . import RBF_FP32C, Batch, Mlp, Solver

N_L_DEFAULT = 25
# Reference speed of Eq. MNS_C for the steady solves here: C = beta v_ref = 20
# makes the artificial sound waves relax faster than the viscous modes on cells
# of this family (h ~ 1/12 .. 1/20), so a start's remaining error decays at the
# viscous rate and a better start saves steps; with v_ref = 0.01 the slow
# artificial-compressibility mode sets the time to steady whatever the start.
V_REF_DEFAULT = 2.0


# network shape (rbf_mlp_*): five layers (fan_in, fan_out); 34 real inputs
# zero-padded to 64, 4 real outputs padded to 16
LAYERS = ((64, 128), (128, 128), (128, 128), (128, 128), (128, 16))
N_FEATURES, N_OUTPUTS = 34, 4


def init_params(seed: int) -> np.ndarray:
    """Initial FP32 parameter vector in the packed order of rbf_mlp_set_params
    (per layer W row-major (fan_out x fan_in), then b): W uniform in
    +-1/sqrt(fan_in) (fan_in of the first layer counted as its 34 real inputs),
    b = 0; the padded input columns and output rows start, and stay, at zero."""
    rng = np.random.default_rng(seed)
    parts = []
    for li, (fi, fo) in enumerate(LAYERS):
        fan = N_FEATURES if li == 0 else fi
        W = rng.uniform(-1.0, 1.0, (fo, fi)) / np.sqrt(fan)
        if li == 0:
            W[:, N_FEATURES:] = 0.0
        if li == len(LAYERS) - 1:
            W[N_OUTPUTS:, :] = 0.0
        parts += [W.ravel(), np.zeros(fo)]
    return np.concatenate(parts).astype(np.float32)


def signed_distance(xyz, centre, r):
    d = np.asarray(xyz, np.float64) - np.asarray(centre, np.float64)
    d -= np.rint(d)
    return np.sqrt((d * d).sum(1)) - r


def steady_training_set(cases, n_l=N_L_DEFAULT, tol=1e-6, max_steps=2_000_000, check_every=1000,
                        precision=RBF_FP32C, device=0, v_ref=V_REF_DEFAULT):
    """Solve every case to steady state in one batched persistent launch; returns
    (xyz, radius, sdf, targets (u, v, w, p)) over all nodes, the per-cell results
    and the wall time."""
    t0 = time.perf_counter()
    b = Batch(device)
    for c in cases:
        b.add_cell(c, n_l)
    b.build(3, 2)
    b.init(precision=precision, v_ref=v_ref)
    res = b.solve(max_steps, tol, check_every=check_every)
    X, R, S, T = [], [], [], []
    for i, c in enumerate(cases):
        f = b.cell(i).get_fields()
        X.append(c["xyz"])
        R.append(np.full(c.n, c["radius"], np.float32))
        S.append(signed_distance(c["xyz"], c["centre"], c["radius"]).astype(np.float32))
        T.append(f.astype(np.float32))
    b.close()
    return (np.concatenate(X), np.concatenate(R), np.concatenate(S), np.concatenate(T)), res, time.perf_counter() - t0


def output_scale(targets):
    """Per-output normalisation of the targets (u, v, w, p): their RMS over the
    training set, so that every output weighs alike in the squared-error loss."""
    t = np.asarray(targets, np.float64)
    s = np.sqrt((t * t).mean(0))
    return np.where(s > 0.0, s, 1.0)


def train(data, init_params, steps=3000, batch=1024, lr=2e-3, seed=7, device=0, normalise=True, decay=()):
    """Train the network on (xyz, radius, sdf, targets); with `normalise` each
    output is divided by its RMS for training and the network's out_scale set to
    match, so warm_start writes fields in the solver's units.  `decay`: further
    (steps, lr) phases run after the first (Adam's moments carry over; each phase
    draws its batches with its own seed)."""
    m = Mlp(device)
    m.set_params(np.asarray(init_params, np.float32))
    xyz, rad, sdf, tgt = data
    if normalise:
        m.out_scale = output_scale(tgt)
        tgt = (np.asarray(tgt, np.float64) / m.out_scale).astype(np.float32)
    m.set_data(xyz, rad, sdf, tgt)
    t0 = time.perf_counter()
    hist = [m.train(steps, batch, lr, seed)]
    for k, (st, lr_k) in enumerate(decay):
        hist.append(m.train(st, batch, lr_k, seed + 1 + k))
    return m, np.concatenate(hist), time.perf_counter() - t0


def solve_case(case, mlp=None, n_l=N_L_DEFAULT, precision=RBF_FP32C, tol=1e-6, max_steps=2_000_000,
               check_every=1000, m_p=24, device=0, v_ref=V_REF_DEFAULT):
    """Steady solve of one case from a zero start or from the network's prediction."""
    s = Solver(device)
    s.set_case(case)
    s.build_stencils(n_l)
    s.compute_weights(solver=0)
    s.init(precision=precision, v_ref=v_ref)
    t0 = time.perf_counter()
    if mlp is not None:
        mlp.warm_start(s, 1.0)
    r = s.solve(max_steps, tol, check_every=check_every, m_p=m_p)
    r["seconds"] = time.perf_counter() - t0
    return s, r


def permeability_history(case, mlp=None, chunk=200, max_steps=20000, n_l=N_L_DEFAULT, precision=RBF_FP32C,
                         m_p=24, device=0, v_ref=V_REF_DEFAULT, tune_steps=0, schedule=None):
    """k/d^2 after every `chunk` steps of one case from a zero start or from the
    network's prediction: [(steps, k/d^2, seconds since the start)], step 0 the
    start itself (the network's evaluation and the warm start included in the
    time, the permeability reads excluded).  tune_steps > 0: autotune the
    persistent driver first (untimed, state restored); schedule: a fixed
    persistent schedule code instead.  Returns (history, schedule code used)."""
    s = Solver(device)
    s.set_case(case)
    s.build_stencils(n_l)
    s.compute_weights(solver=0)
    s.init(precision=precision, v_ref=v_ref)
    if schedule is not None:
        s.set_persistent_block(schedule)
    elif tune_steps > 0:
        schedule = s.autotune_persistent(tune_steps)[1]
    t0 = time.perf_counter()
    if mlp is not None:
        mlp.warm_start(s, 1.0)
    t_run = time.perf_counter() - t0
    hist = [(0, s.permeability(m_p)[0], t_run)]
    steps = 0
    while steps < max_steps:
        t1 = time.perf_counter()
        s.solve(chunk, 1e-300, check_every=chunk, m_p=m_p)
        t_run += time.perf_counter() - t1
        steps += chunk
        hist.append((steps, s.permeability(m_p)[0], t_run))
    s.close()
    return hist, schedule


def first_within(hist, k_ref, rel=1e-4):
    """The first (steps, k, seconds) of a permeability history after which k stays
    within rel of k_ref until the end of the history; None if it never settles."""
    ok = [abs(k - k_ref) <= rel * abs(k_ref) for _, k, _ in hist]
    for i in range(len(ok)):
        if all(ok[i:]):
            return hist[i]
    return None
