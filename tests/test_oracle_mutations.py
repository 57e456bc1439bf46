"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each case monkeypatches one plausible error into the oracle (a dropped
term, a wrong sign, a transposed operand, a shifted index) and checks that
the circle eigen-expansion pin no longer holds.
"""
import numpy as np
import pytest

import oracle.assembly as oa
from oracle import rules
from paper_1703_10016_gb300 import workloads as wl
from tests.test_oracle_assembly import circle_fourier_matrix

R, N, D = 0.5, 32, 3


def _pin_error():
    A = oa.assemble(wl.nurbs_circle(R), N, D, 2)["A"]
    Ar = circle_fourier_matrix(R, N, D)
    return np.linalg.norm(A - Ar) / np.linalg.norm(Ar)


def test_unmutated_oracle_meets_pin():
    assert _pin_error() < 5e-4


def _drop_images(disc):
    return [0.0]


def _k1_sign(orig):
    def f(*a, **k):
        return -orig(*a, **k)
    return f


def _transpose_ws(orig):
    def f(disc, rows=None):
        Ws = orig(disc, rows)
        return Ws.T if rows is None else Ws
    return f


def _shift_regular(orig):
    def f(disc):
        return np.roll(orig(disc), 1, axis=0)
    return f


@pytest.mark.parametrize("mutation", ["images", "k1_sign", "ws_transpose", "regular_shift"])
def test_planted_mistake_is_caught(monkeypatch, mutation):
    if mutation == "images":
        monkeypatch.setattr(rules, "k2_images", _drop_images)
    elif mutation == "k1_sign":
        monkeypatch.setattr(oa, "kernel_K1", _k1_sign(oa.kernel_K1))
    elif mutation == "ws_transpose":
        monkeypatch.setattr(rules, "singular_rules", _transpose_ws(rules.singular_rules))
    elif mutation == "regular_shift":
        monkeypatch.setattr(rules, "regular_rules", _shift_regular(rules.regular_rules))
    assert _pin_error() > 1e-2
