"""The oracle against the stored expected values under tests/golden/ (each
fixture cites its source: the paper's printed equations, a textbook
constant, a published known-answer table)."""
import os

import pytest

from oracle import dynamics as D
from oracle import reference as R

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                out.append(line)
    return out


def value(name, key):
    vals = [r[1:] for r in rows(name) if r[0] == key]
    assert vals, f"{key} missing from {name}"
    return [float(v) for v in vals[0]]


def test_ucap_printed_polynomial():
    c6, c5, c4, c0 = value("paper_values.txt", "ucap_poly")
    for x in (0.0, 0.1, 0.37, 0.5, 0.8, 0.999):
        assert R.ucap(x)[0] == pytest.approx(c6 * x**6 + c5 * x**5 + c4 * x**4 + c0, rel=1e-13, abs=1e-12)
    assert R.ucap(0.0)[0] == pytest.approx(value("paper_values.txt", "ucap_at_zero")[0], abs=1e-12)


def test_switching_printed_values():
    onset = value("paper_values.txt", "hA_onset")[0]
    assert R.switching(onset)[0] == 0.0
    assert R.switching(onset + 1e-3)[0] > 0.0
    for r in rows("paper_values.txt"):
        if r[0] == "end_state":
            lam, hA, hB = map(float, r[1:])
            got = R.switching(lam)
            assert got[0] == pytest.approx(hA, abs=1e-15) and got[1] == pytest.approx(hB, abs=1e-15)
    assert R.S22(0.5)[0] == pytest.approx(value("paper_values.txt", "S22_half")[0], abs=1e-15)
    assert R.S32(0.5)[0] == pytest.approx(value("paper_values.txt", "S32_half")[0], abs=1e-15)


def test_mirror_map_printed_cases():
    for r in rows("paper_values.txt"):
        if r[0] == "mirror":
            theta, lam, s = map(float, r[1:])
            got_lam, got_s = D.theta_to_lambda(theta)
            assert got_lam == pytest.approx(lam, abs=1e-12) and got_s == s
