"""Host arithmetic of the parameter studies (no GPU): the grid convergence
index of the appendix and the refinement error.

* The apparent order p is recovered exactly from errors that follow A h^p.
* Richardson's property: for X(h) = X_inf + c h^p and the true p, GCI / F_s on
  the finer grid of a pair equals the true relative error |X_fine - X_inf| /
  X_fine, whatever the refinement ratio.
* GCI belongs to the finer grid of each successive pair, in any input order.
"""
import numpy as np
import pytest

from paper_2404_14195_gb300 import studies


def test_apparent_order_exact_power_law():
    h = np.array([0.02, 0.014, 0.01, 0.007, 0.005])
    for p in (1.0, 1.7, 2.5):
        X = 0.3 * (1.0 + 40.0 * h ** p)
        X[-1] = 0.3  # the reference value: e = A h^p exactly for the others
        assert abs(studies.apparent_order(h, X) - p) < 1e-10


@pytest.mark.parametrize("p,h", [(2.0, [0.02, 0.01]), (1.5, [0.02, 0.014, 0.01, 0.007]), (3.0, [0.05, 0.02])])
def test_gci_richardson_property(p, h):
    X_inf, c = 1.25, -7.0
    h = np.array(h)
    X = X_inf + c * h ** p
    _, g = studies.gci(h, X, F_s=1.3, p=p)
    for i in range(1, len(h)):
        fine = X[i]
        assert abs(g[float(h[i])] / 1.3 - abs(fine - X_inf) / abs(fine)) < 1e-12


def test_gci_pairs_go_to_the_finer_grid():
    h = [0.01, 0.02, 0.014]  # any order
    X = [1.0, 1.2, 1.1]
    _, g = studies.gci(h, X, p=2.0)
    assert sorted(g) == [0.01, 0.014]
    # pair (0.02, 0.014): eps = 0.1 / 1.1, r = 0.02 / 0.014
    assert abs(g[0.014] - 1.3 * (0.1 / 1.1) / ((0.02 / 0.014) ** 2 - 1.0)) < 1e-15
    with pytest.raises(ValueError):
        studies.apparent_order([0.02, 0.01], [1.1, 1.0])


def test_refinement_error():
    assert studies.refinement_error(1.1, 1.0) == pytest.approx(0.1)
    assert studies.refinement_error(0.9, 1.0) == pytest.approx(0.1)


def _fake_run_factory(K_of, k_of=None, fail=()):
    def fake_run(r, h_min, seed=2, h_ratio=2.0, eps=0.295, n_l=25, **kw):
        key = (h_min, h_ratio, eps, n_l)
        conv = key not in fail
        K = K_of(*key) if conv else float("nan")
        k = (k_of or K_of)(*key) if conv else float("nan")
        return dict(r=r, h_min=h_min, h_ratio=h_ratio, eps=eps, n_l=n_l,
                    mlbm=dict(k=k, K=K, converged=conv), mns=dict(k=2 * k, K=2 * K, converged=conv))
    return fake_run


def test_refinement_study_errors_against_the_uniform_cell(monkeypatch):
    # K = 10 on the uniform cell (ratio 1), 10 (1 + 0.01 ratio eps) otherwise; (4, 0.1) diverges
    K_of = lambda h, ratio, eps, n_l: 10.0 if ratio == 1.0 else 10.0 * (1.0 + 0.01 * ratio * eps)
    monkeypatch.setattr(studies, "_run", _fake_run_factory(K_of, fail={(0.02, 4.0, 0.1, 25)}))
    out = studies.refinement_parameter_study(0.5, 0.02)
    assert out["reference"]["h_ratio"] == 1.0
    assert len(out["rows"]) == 9
    for x in out["rows"]:
        if (x["h_ratio"], x["eps"]) == (4.0, 0.1):
            assert np.isnan(x["mlbm"]["E"]) and np.isnan(x["mns"]["E"])
        else:
            assert x["mlbm"]["E"] == pytest.approx(0.01 * x["h_ratio"] * x["eps"])
            assert x["mns"]["E"] == pytest.approx(0.01 * x["h_ratio"] * x["eps"])


def test_convergence_study_wires_gci(monkeypatch):
    p = 2.0
    K_of = lambda h, ratio, eps, n_l: 3.0 * (1.0 + 50.0 * h ** p) if h > 0.01 else 3.0
    monkeypatch.setattr(studies, "_run", _fake_run_factory(K_of))
    out = studies.convergence_study(0.3, [0.028, 0.02, 0.014, 0.01])
    assert out["mlbm_K_p"] == pytest.approx(p)
    assert out["mns_k_p"] == pytest.approx(p)
    _, g = studies.gci([0.028, 0.02, 0.014, 0.01], [K_of(h, 2, 0.3, 25) for h in (0.028, 0.02, 0.014, 0.01)])
    assert out["mlbm_K_gci"] == pytest.approx(g)


def test_cli_dispatch_and_json(monkeypatch, capsys, tmp_path):
    """The studies command line hands its arguments to the study and prints one
    JSON object (NaN as null); single process, no GPU."""
    import json
    seen = {}

    def fake_sweep(radii, h_min, solid_check_above=None, _ranks=(), **kw):
        seen.update(radii=radii, h_min=h_min, solid=solid_check_above, kw=kw)
        return [dict(r=r, k=float("nan")) for r in radii]
    monkeypatch.setattr(studies, "porosity_sweep", fake_sweep)
    out = tmp_path / "o.json"
    studies.main(["porosity", "--radii", "0.3,0.6", "--h-min", "0.03", "--solid-check-above", "0.5",
                  "--window", "500", "--out", str(out)])
    d = json.loads(capsys.readouterr().out)
    assert seen["radii"] == (0.3, 0.6) and seen["h_min"] == 0.03 and seen["solid"] == 0.5
    assert seen["kw"]["window_steps"] == 500 and seen["kw"]["device"] == 0
    assert d["study"] == "porosity" and d["ranks"] == 1 and d["result"][0] == {"r": 0.3, "k": None}
    assert json.loads(out.read_text()) == d


def test_crossval_cli_dispatch(monkeypatch, capsys):
    import json
    from paper_2404_14195_gb300 import crossval
    seen = {}

    def fake_cv(case, **kw):
        seen.update(kw, n=case.n, r=case["radius"])
        return dict(mlbm=dict(history=[(1, 0.1)] * 8), mns=dict(history=[(1, 0.1)] * 8),
                    line=dict(x=np.arange(200.0), node=np.arange(200), speed_a=np.ones(200)))
    monkeypatch.setattr(crossval, "cross_validate", fake_cv)
    crossval.main(["--r", "0.6526", "--h-min", "0.04", "--v-ref", "auto", "--unknown-rule", "1", "--q", "19"])
    d = json.loads(capsys.readouterr().out)
    assert seen["v_ref"] == "auto" and seen["unknown_rule"] == 1 and seen["q"] == 19 and seen["r"] == 0.6526
    assert len(d["mlbm"]["history"]) == 5          # the last windows only
    assert len(d["line"]["x"]) <= 67 and "node" not in d["line"]
