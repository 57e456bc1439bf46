"""The seeded input generators shared by the tests and the benchmark (CPU only).

They hold none of the method's arithmetic, but the manufactured solutions of
the parity and solve tests rely on them: the Dirichlet data must be harmonic
with the stated gradient, and a seed must always give the same workload.
"""
import math

import numpy as np
import pytest

from oracle import bspline
from paper_1703_10016_gb300 import workloads as wl


@pytest.mark.parametrize("h", [wl.Harmonic("x2-y2"), wl.Harmonic("log"), wl.rhs_source(3, 8)])
def test_harmonic_data_gradient_and_laplacian(h):
    """Central differences of the value match the stated gradient, and the
    five-point Laplacian vanishes (to the differences' truncation error)."""
    rng = np.random.default_rng(0)
    x, y = rng.uniform(-0.6, 0.6, 50), rng.uniform(-0.6, 0.6, 50)
    e = 1e-5
    gx, gy = h.grad(x, y)
    np.testing.assert_allclose((h.value(x + e, y) - h.value(x - e, y)) / (2 * e), gx, rtol=1e-7, atol=1e-8)
    np.testing.assert_allclose((h.value(x, y + e) - h.value(x, y - e)) / (2 * e), gy, rtol=1e-7, atol=1e-8)
    e = 1e-3
    lap = (h.value(x + e, y) + h.value(x - e, y) + h.value(x, y + e) + h.value(x, y - e) - 4 * h.value(x, y)) / (e * e)
    assert np.max(np.abs(lap)) < 1e-4


def test_point_sources_lie_outside_the_curves():
    """The log data's singular points are at radius 2 or more, the curves within 0.5."""
    for k in range(8):
        assert math.hypot(*wl.rhs_source(k, 8).x0) == pytest.approx(2.5)
    assert math.hypot(*wl.Harmonic("log").x0) > 2.0
    for c in (wl.star_curve(), wl.random_star(np.random.default_rng(1))):
        f = bspline.curve_eval(c, np.linspace(0.0, 1.0, 400, endpoint=False), 0)[0]
        assert np.max(np.hypot(f[0], f[1])) < 0.5


def test_random_star_radius_bounds():
    """r0 (1 + sum a_k cos(..)) with 0 <= a_k <= 0.04, five terms: within r0 (1 +- 0.2)
    (up to the interpolant's deviation between its points)."""
    rng = np.random.default_rng(2)
    for _ in range(5):
        c = wl.random_star(rng)
        f = bspline.curve_eval(c, np.linspace(0.0, 1.0, 1000, endpoint=False), 0)[0]
        r = np.hypot(f[0], f[1])
        assert r.min() > 0.4 * 0.79 and r.max() < 0.4 * 1.21


def test_seeded_batch_and_arrivals_are_reproducible():
    a, b = wl.batch_mix(64), wl.batch_mix(64)
    assert [(p.n_elems, p.degree) for p in a] == [(p.n_elems, p.degree) for p in b]
    np.testing.assert_array_equal(a[7].curve.ctrl, b[7].curve.ctrl)
    assert all(64 <= p.n_elems <= 4096 and p.degree in (2, 3, 4) for p in a)
    r1 = wl.serve_arrivals(2000.0, 0.05)
    r2 = wl.serve_arrivals(2000.0, 0.05)
    assert [(t, p.n_elems, p.degree, k) for t, p, k in r1] == [(t, p.n_elems, p.degree, k) for t, p, k in r2]
    ts = [t for t, _, _ in r1]
    assert all(t1 < t2 for t1, t2 in zip(ts, ts[1:])) and ts[-1] <= 0.05
    assert all(128 <= p.n_elems <= 16384 and p.degree in (2, 3, 4) and 1 <= k <= 8 for _, p, k in r1)
    # about rate x duration arrivals (Poisson, 100 expected)
    assert 60 < len(r1) < 140
