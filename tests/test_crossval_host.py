"""Host logic of the cross-validation driver and the studies (no GPU): the
stopping rule of Eq. stopCrit as `run_to_steady` applies it between windows,
the automatic v_ref, and the seed-spread aggregation.  A fake solver stands in
for a library context; it only reports a prescribed k/d^2 history."""
import math

import numpy as np
import pytest

import oracle
from paper_2404_14195_gb300 import RBF_SOLVER_ACM, RBF_SOLVER_LBM, crossval, studies


class FakeSolver:
    def __init__(self, k_of_t, dt, solver=RBF_SOLVER_LBM):
        self.k_of_t, self.dt, self.solver = k_of_t, dt, solver
        self.steps = 0
        self.calls = []

    def time_step(self):
        return self.dt

    def step(self, n):
        self.calls.append(("step", n))
        self.steps += n

    def solve(self, n, tol, check_every=100, m_p=32):
        self.calls.append(("solve", n, check_every))
        self.steps += n
        return dict(steps=n)

    def permeability(self, m_p=32):
        return self.k_of_t(self.steps * self.dt), 0.0


def test_stops_at_first_window_below_the_rate():
    k_inf, tau, dt, w = 0.03, 0.05, 1e-5, 1000
    s = FakeSolver(lambda t: k_inf * (1.0 - math.exp(-t / tau)), dt)
    r = crossval.run_to_steady(s, tol=1e-2, window_steps=w, max_steps=10 ** 7)
    assert r["converged"]
    hist = r["history"]
    rates = [oracle.stop_criterion(hist[i][1], hist[i - 1][1], w * dt) for i in range(1, len(hist))]
    assert rates[-1] < 1e-2 and all(x >= 1e-2 for x in rates[:-1])
    # the analytic window where the rate crosses 1e-2: exp(-t/tau)(exp(w dt/tau) - 1) / (w dt) = 1e-2 k(t)/k_inf
    t_stop = r["steps"] * dt
    assert abs(k_inf - hist[-1][1]) / k_inf < 1e-2 * tau * 1.2
    assert all(c[0] == "step" for c in s.calls)
    assert r["time"] == pytest.approx(t_stop)


def test_acm_windows_use_the_persistent_solve_and_cap():
    s = FakeSolver(lambda t: 1.0 + t, 1e-4, solver=RBF_SOLVER_ACM)  # rate 1/(1+t) never below 1e-2 early
    r = crossval.run_to_steady(s, tol=1e-3, window_steps=500, max_steps=2200)
    assert not r["converged"] and r["steps"] == 2200
    assert [c[1] for c in s.calls] == [500, 500, 500, 500, 200]
    assert all(c[0] == "solve" and c[2] == c[1] for c in s.calls)


def test_nonfinite_k_stops_as_diverged():
    s = FakeSolver(lambda t: float("nan") if t > 0.025 else 0.01 * (1.0 + t), 1e-5)
    r = crossval.run_to_steady(s, tol=1e-2, window_steps=1000, max_steps=10 ** 6)
    assert not r["converged"] and math.isnan(r["history"][-1][1]) and r["steps"] == 3000


def test_constant_k_needs_two_windows():
    s = FakeSolver(lambda t: 0.5, 1e-5)
    r = crossval.run_to_steady(s, tol=1e-2, window_steps=100, max_steps=10 ** 5)
    assert r["converged"] and r["steps"] == 200 and r["rate"] == 0.0


def test_auto_v_ref_courant_number():
    for h in (0.0037, 0.01):
        v = crossval.auto_v_ref(h, nu=1.0, beta=10.0, cfl=0.1, courant=0.01)
        dt = 0.1 * h * h / 2.0
        assert (10.0 * v) * dt / h == pytest.approx(0.01)


def test_seed_spread_aggregation(monkeypatch):
    vals = {1: 1.0, 2: 1.1, 3: 0.9, 4: float("nan")}

    def fake_run(r, h_min, seed=2, **kw):
        k = vals[seed]
        conv = np.isfinite(k)
        return dict(r=r, seed=seed, mlbm=dict(k=k, K=2 * k, converged=conv),
                    mns=dict(k=k, K=3 * k, converged=True))
    monkeypatch.setattr(studies, "_run", fake_run)
    out = studies.seed_spread([0.3], seeds=(1, 2, 3, 4))[0]
    assert out["mlbm_k_n"] == 3
    assert out["mlbm_k_spread"] == pytest.approx(np.std([1.0, 1.1, 0.9], ddof=1) / 1.0)
    assert out["mlbm_K_spread"] == pytest.approx(out["mlbm_k_spread"])
    assert out["mns_k_n"] == 3  # the NaN run is dropped even though flagged converged


def test_diverged_persistent_solve_ends_the_run():
    from paper_2404_14195_gb300 import RBF_EDIVERGED, RBF_EINVAL, RbfError

    class Diverging(FakeSolver):
        def solve(self, n, tol, check_every=100, m_p=32):
            if self.steps >= 2000:
                raise RbfError(self.code, "non-finite fields")
            return super().solve(n, tol, check_every, m_p)

    s = Diverging(lambda t: 0.01 * (1.0 + t), 1e-5, solver=RBF_SOLVER_ACM)
    s.code = RBF_EDIVERGED
    r = crossval.run_to_steady(s, tol=1e-3, window_steps=1000, max_steps=10 ** 6)
    assert not r["converged"] and r["steps"] == 3000 and math.isnan(r["history"][-1][1])
    s = Diverging(lambda t: 0.01 * (1.0 + t), 1e-5, solver=RBF_SOLVER_ACM)
    s.code = RBF_EINVAL  # any other error is not swallowed
    with pytest.raises(RbfError):
        crossval.run_to_steady(s, tol=1e-3, window_steps=1000, max_steps=10 ** 6)
