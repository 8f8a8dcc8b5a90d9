"""The oracle against the values the paper prints (tests/golden/paper_printed_values.txt):
the D3Q15 direction and weight tables of the MLBM section, the porosity range of the
case definition, and the time-step ranges of the MNS and MLBM footnotes."""
import os
from fractions import Fraction

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_printed_values.txt")


def _rows(name):
    out = []
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].split()
        if line and line[0] == name:
            out.append(line[1:])
    assert out, name
    return out


def test_d3q15_directions_and_weights():
    e, w, opp = oracle.velocity_set(15)
    for k, x, y, z in _rows("d3q15_e"):
        k = int(k)
        assert tuple(e[k]) == (int(x), int(y), int(z)), k
        if k:
            assert tuple(e[k + 1]) == (-int(x), -int(y), -int(z)), k + 1
    assert len(e) == 15
    for lo, hi, val in _rows("d3q15_w"):
        for k in range(int(lo), int(hi) + 1):
            assert abs(w[k] - float(Fraction(val))) < 1e-16, k


def test_porosity_range():
    for r, phi, digits in _rows("porosity"):
        assert round(oracle.porosity(float(r)), int(digits)) == float(phi), r


def test_time_step_ranges():
    for h, dt in _rows("acm_dt"):
        assert abs(oracle.acm_dt(float(h), 1.0) - float(dt)) <= 1e-12 * float(dt), h
    for dx, dt in _rows("lbm_dt"):
        got = oracle.lbm_units(1.0, 1.0, float(dx), (1.0, 0.0, 0.0))["dt"]
        assert f"{got:.2e}" == f"{float(dt):.2e}", (dx, got)
