"""What the trained network gains: held-out cells reach the steady residual in
fewer steps from the network's prediction than from rest, and land on the same
permeability.  Training data are steady fields of other cells, solved by the
library itself in one batched persistent launch; training and inference run on
the tensor-core kernels."""
import numpy as np
import pytest

import synth
from gpu_common import gpu_or_skip
from oracle import mlp as om

pytestmark = pytest.mark.gpu


def test_warm_start_needs_fewer_steps():
    rbf = gpu_or_skip()
    from paper_2404_14195_gb300 import warmstart as ws
    rng = np.random.default_rng(0)
    train_cases = [synth.jittered_cell(r=float(r), n_axis=12, seed=100 + i)
                   for i, r in enumerate(rng.uniform(0.15, 0.45, 8))]
    data, res, t_data = ws.steady_training_set(train_cases, tol=1e-6)
    assert all(r["status"] == 0 for r in res)
    m, hist, t_train = ws.train(data, om.init_params(1), steps=3000, batch=1024)
    assert hist[-50:].mean() < 0.2 * hist[:10].mean()
    zero, warm = 0, 0
    for i, r in enumerate((0.25, 0.37)):
        case = synth.jittered_cell(r=r, n_axis=12, seed=500 + i)
        _, rz = ws.solve_case(case, None)
        _, rw = ws.solve_case(case, m)
        assert rz["converged"] and rw["converged"]
        assert abs(rw["k_over_d2"] - rz["k_over_d2"]) <= 1e-2 * rz["k_over_d2"]
        zero += rz["steps"]
        warm += rw["steps"]
    assert warm < 0.8 * zero, (warm, zero)
