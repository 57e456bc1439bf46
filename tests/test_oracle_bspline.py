"""Pins for the oracle's B-spline / NURBS evaluation and discretisation (CPU)."""
from math import comb, factorial

import numpy as np
import pytest

from oracle import bspline
from oracle.discretization import Discretization
from paper_1703_10016_gb300 import workloads as wl


def cardinal(d, x):
    """Cardinal B-spline on [0, d+1] by the truncated-power formula (independent closed form)."""
    x = np.asarray(x, float)
    return sum((-1) ** k * comb(d + 1, k) * np.maximum(x - k, 0.0) ** d for k in range(d + 2)) / factorial(d)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5])
def test_uniform_bsplines_match_truncated_power_formula(d):
    knots = np.arange(-d, 12 + d + 1, dtype=float)
    x = np.linspace(0.0, 12.0, 777)
    B = bspline.basis_all(knots, d, x)[0]
    for i in range(B.shape[0]):
        u = x - knots[i]
        ref = np.where((u > 0) & (u < d + 1), cardinal(d, np.clip(u, 0, d + 1)), 0.0)
        np.testing.assert_allclose(B[i], ref, atol=1e-12)


@pytest.mark.parametrize("d", [2, 3, 4])
def test_partition_of_unity_and_derivative(d):
    rng = np.random.default_rng(0)
    knots = np.concatenate([[0.0] * d, np.sort(rng.uniform(0, 1, 9)), [1.0] * d])
    knots = np.concatenate([[0.0], knots, [1.0]])
    x = np.linspace(0.0, 1.0, 301)
    B = bspline.basis_all(knots, d, x, nder=1)
    np.testing.assert_allclose(B[0].sum(axis=0), 1.0, atol=1e-13)
    np.testing.assert_allclose(B[1].sum(axis=0), 0.0, atol=1e-9)
    # derivative against a central difference
    h = 1e-6
    xm = x[5:-5]
    Bp = bspline.basis_all(knots, d, xm + h)[0]
    Bm = bspline.basis_all(knots, d, xm - h)[0]
    fd = (Bp - Bm) / (2 * h)
    inner = np.all(np.abs(xm[:, None] - knots[None, :]) > 2 * h, axis=1)
    np.testing.assert_allclose(B[1][:, 5:-5][:, inner], fd[:, inner], atol=2e-5)


def test_nurbs_circle_is_exact():
    c = wl.nurbs_circle(0.5)
    s = np.linspace(0, 1, 1001)
    f, f1 = bspline.curve_eval(c, s, 1)
    np.testing.assert_allclose(np.hypot(f[0], f[1]), 0.5, atol=1e-14)
    # counter-clockwise: f x f' > 0
    assert np.all(f[0] * f1[1] - f[1] * f1[0] > 0)
    # closed and C^1 across the seam
    np.testing.assert_allclose(f[:, 0], f[:, -1], atol=1e-15)
    np.testing.assert_allclose(f1[:, 0], f1[:, -1], rtol=1e-13)


def test_star_interpolates_and_is_periodic_c2():
    c = wl.star_curve()
    th = 2 * np.pi * np.arange(256) / 256
    r = 0.4 * (1 + 0.2 * np.cos(5 * th))
    f, f1, f2 = bspline.curve_eval(c, np.arange(256) / 256, 2)
    np.testing.assert_allclose(f[0], r * np.cos(th), atol=1e-14)
    np.testing.assert_allclose(f[1], r * np.sin(th), atol=1e-14)
    e = bspline.curve_eval(c, np.array([0.0, 1.0]), 2)
    for k in range(3):
        np.testing.assert_allclose(e[k][:, 0], e[k][:, 1], rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("closed", [True, False])
@pytest.mark.parametrize("d,nh,nref", [(2, 10, 1), (3, 8, 2), (4, 9, 2), (3, 12, 3)])
def test_nodes_and_index_sets(closed, d, nh, nref):
    disc = Discretization(0.0, 1.0, nh, d, nref, closed)
    # N_quad = 2d + 2 N_ref N_h - 1 (Sect. 4)
    assert disc.Nq == 2 * d + 2 * nref * nh - 1
    assert np.all(np.diff(disc.eta) > 0)
    Bc = disc.collocation()
    # Schoenberg-Whitney: the collocation matrix has full row rank
    sv = np.linalg.svd(Bc, compute_uv=False)
    assert sv.min() > 1e-3
    Bt = disc.test_basis(disc.eta)[0]
    for i in range(disc.n):
        Ni = disc.support_nodes(i)
        # N^(i) is exactly the set of nodes where B_i is non-zero
        nz = np.nonzero(np.abs(Bt[i]) > 1e-12)[0]
        np.testing.assert_array_equal(Ni, nz)
        Ji = disc.overlapping_fine(i)
        # Sect. 4.1: N_E^(i) <= N_quad^(i) and N_E^(i) <= (1 + N_ref)(d + 1);
        # a wrapped closed-curve function meets the non-wrapped exactness
        # space at both ends of I, which adds up to d - 1 more functions
        assert len(Ji) <= len(Ni)
        wrapped = closed and len(disc._test_support(i)) == 2
        assert len(Ji) <= (1 + nref) * (d + 1) + (d - 1 if wrapped else 0)
    # closed test space: partition of unity of the cyclic basis
    if closed:
        np.testing.assert_allclose(Bt.sum(axis=0), 1.0, atol=1e-13)


def test_nodes_written_out_for_one_small_case():
    """Sect. 4's node vector for d = 2, N_ref = 1, N_h = 4 on [0, 1] written out
    by hand: d + 2 = 4 uniform points (end points included) in the first and the
    last refined element, the midpoint of every inner element and the
    breakpoints between inner elements: N_quad = 2d + 2M - 1 = 11."""
    want = np.array([0.0, 1 / 12, 2 / 12, 3 / 12,          # first element [0, 1/4]
                     3 / 8,                                # midpoint of [1/4, 1/2]
                     1 / 2, 5 / 8,                         # breakpoint 1/2, midpoint of [1/2, 3/4]
                     9 / 12, 10 / 12, 11 / 12, 1.0])       # last element [3/4, 1]
    for closed in (True, False):
        disc = Discretization(0.0, 1.0, 4, 2, 1, closed)
        np.testing.assert_allclose(disc.eta, want, rtol=0, atol=1e-15)
    # d = 3, N_ref = 2, N_h = 4 on [-1, 3] (h_f = 1/2, M = 8): 5 points per end element
    disc = Discretization(-1.0, 3.0, 4, 3, 2, True)
    want = np.array([-1.0, -0.875, -0.75, -0.625, -0.5,                  # [-1, -1/2]
                     -0.25, 0.0, 0.25, 0.5, 0.75, 1.0, 1.25, 1.5, 1.75, 2.0, 2.25,   # midpoints, inner breakpoints
                     2.5, 2.625, 2.75, 2.875, 3.0])                       # [5/2, 3]
    assert disc.Nq == 21
    np.testing.assert_allclose(disc.eta, want, rtol=0, atol=1e-15)
