"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each case monkeypatches one plausible error into the oracle (a dropped
term, a wrong sign, a transposed operand, a shifted index) and checks that
the circle eigen-expansion pin no longer holds; for the right-hand side, that
Gauss's identity (constant data give beta = 0, Sect. 5) no longer holds when
the double-layer kernel has a wrong sign, the tangential in place of the
normal derivative, or a wrong power of the distance.
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


# ---- right-hand side (Sect. 5): Gauss's identity for constant data --------

def _const_rhs_ratio():
    """max |beta| / max row weight for u_D = 1 on the star: zero up to the
    inner rule's error for the correct oracle (b1/2 = b2/(2 pi)); n = 128
    aligns the refined elements with the star's 256 geometry elements, where
    that error is about 3e-12."""
    c = wl.star_curve()
    n, d = 128, 3
    eta, tg, _ = oa.rhs_points(c, n, d, 2)
    beta = oa.build_rhs(c, n, d, 2, np.ones((len(eta), 1)), np.ones((len(tg), 1)))
    m = oa.assemble(c, n, d, 2, keep=True)["P"].sum(axis=0)
    return np.max(np.abs(beta[:, 0])) / np.max(m)


def test_unmutated_rhs_meets_gauss_identity():
    assert _const_rhs_ratio() < 1e-10


def _kbar_sign(orig):
    def f(f_s, f_t, f1_t):
        return -orig(f_s, f_t, f1_t)
    return f


def _kbar_tangent(orig):
    # the tangential instead of the normal derivative of log|x - y|
    def f(f_s, f_t, f1_t):
        dx = f_t[0][None, :] - f_s[0][:, None]
        dy = f_t[1][None, :] - f_s[1][:, None]
        return (dx * f1_t[0][None, :] + dy * f1_t[1][None, :]) / (dx * dx + dy * dy)
    return f


def _kbar_no_square(orig):
    # |f(t) - f(s)| in place of its square in the denominator
    def f(f_s, f_t, f1_t):
        dx = f_t[0][None, :] - f_s[0][:, None]
        dy = f_t[1][None, :] - f_s[1][:, None]
        return (dx * f1_t[1][None, :] - dy * f1_t[0][None, :]) / np.sqrt(dx * dx + dy * dy)
    return f


@pytest.mark.parametrize("mutation", ["sign", "tangent", "no_square"])
def test_planted_rhs_mistake_is_caught(monkeypatch, mutation):
    wrap = {"sign": _kbar_sign, "tangent": _kbar_tangent, "no_square": _kbar_no_square}[mutation]
    monkeypatch.setattr(oa, "kernel_Kbar", wrap(oa.kernel_Kbar))
    assert _const_rhs_ratio() > 1e-3
