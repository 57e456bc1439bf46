"""Pins for the oracle's representation formula (Sect. 2), CPU only.

Independent references:
* circle of radius r, q = 1 and u_D = 1: the single layer of a constant
  density is 2 pi r ln r inside the circle and the double layer of a
  constant is 2 pi (Gauss's identity), so u(x) = 1 - r ln r;
* Green's third identity: a harmonic u is reproduced from its exact trace
  and exact flux on a star-shaped curve;
* the logarithmic potential of a unit density on the segment [-1, 1] in
  closed form (open arc, indirect method);
* the full method: the solved density of a manufactured harmonic problem
  reproduces u inside the domain, with the error shrinking under refinement
  (pins the coefficient-to-density step q_h = sum_j alpha_j B_j);
* planted mistakes (a flipped double-layer sign, a dropped Jacobian, a
  shifted coefficient) break one of the above.
"""
import numpy as np
import pytest

import oracle.assembly as oa
from oracle import bspline
from paper_1703_10016_gb300 import workloads as wl

INNER = np.array([[0.0, 0.0], [0.1, 0.05], [-0.15, 0.1], [0.2, -0.1]])


def segment():
    """f(t) = (t, 0), t in [-1, 1]: a degree-1 spline with J = 1."""
    return wl.Curve(1, np.array([-1.0, -1.0, 1.0, 1.0]), np.array([[-1.0, 0.0], [1.0, 0.0]]), None, False)


def segment_log_potential(x1, x2):
    """-(1/2 pi) int_{-1}^{1} ln|(x1, x2) - (t, 0)| dt, x2 != 0, from
    int (1/2) ln(u^2 + c^2) du = (u ln(u^2 + c^2) - 2u + 2c atan(u/c)) / 2."""
    c = abs(x2)

    def F(u):
        return 0.5 * (u * np.log(u * u + c * c) - 2.0 * u + 2.0 * c * np.arctan(u / c))
    return -(F(1.0 - x1) - F(-1.0 - x1)) / (2.0 * np.pi)


def test_circle_constant_density_and_data():
    r = 0.5
    c = wl.nurbs_circle(r)
    pts = np.array([[0.0, 0.0], [0.1, 0.2], [-0.25, 0.1], [0.3, -0.2]])
    errs = []
    for n in (16, 32):
        disc = oa.make_discretization(c, n, 3, 2)
        tg, _ = disc.fine_gauss(oa.G_RHS)
        u = oa.eval_potential(c, n, 3, 2, np.ones((1, disc.n)), np.ones((1, len(tg))), pts)
        errs.append(np.max(np.abs(u - (1.0 - r * np.log(r)))))
    assert errs[1] < 1e-10 and errs[0] > errs[1]


@pytest.mark.parametrize("kind", ["x2-y2", "log"])
def test_green_identity_star(kind):
    """u = -(1/2pi) int ln|x-y| q + (1/2pi) int d/dn_y ln|x-y| u for harmonic u
    (n = 128 aligns the refined elements with the star's geometry elements)."""
    st = wl.star_curve()
    h = wl.Harmonic(kind)
    disc = oa.make_discretization(st, 128, 3, 2)
    tg, wg = disc.fine_gauss(oa.G_RHS)
    f, f1, _ = oa.geometry_at(st, tg)
    nrm = oa.outward_normal(f1)
    gx, gy = h.grad(*f)
    q = (gx * nrm[0] + gy * nrm[1])[None]
    u = oa.potential_sum(INNER.T, f, f1, wg, q, h.value(*f)[None])
    np.testing.assert_allclose(u[0], h.value(*INNER.T), rtol=0, atol=1e-12)


def test_open_segment_closed_form():
    pts = np.array([[0.0, 0.5], [0.3, -0.4], [1.5, 0.2], [-0.9, 0.3]])
    exact = np.array([segment_log_potential(*p) for p in pts])
    for n, tol in ((8, 1e-10), (32, 1e-14)):
        disc = oa.make_discretization(segment(), n, 2, 2)
        u = oa.eval_potential(segment(), n, 2, 2, np.ones((1, disc.n)), None, pts)
        np.testing.assert_allclose(u[0], exact, rtol=0, atol=tol)


def _pipeline(n, d=3):
    st = wl.star_curve()
    hl = wl.Harmonic("log")
    eta, tg, _ = oa.rhs_points(st, n, d, 2)
    fe = bspline.curve_eval(st, eta, 0)[0]
    fg = bspline.curve_eval(st, tg, 0)[0]
    beta = oa.build_rhs(st, n, d, 2, hl.value(*fe)[:, None], hl.value(*fg)[:, None])
    alpha = oa.solve(oa.assemble(st, n, d, 2)["A"], beta)
    u = oa.eval_potential(st, n, d, 2, alpha.T, hl.value(*fg)[None], INNER)
    return np.max(np.abs(u[0] - hl.value(*INNER.T)))


def test_solved_density_reproduces_interior_solution():
    e32, e64 = _pipeline(32), _pipeline(64)
    assert e64 < 1e-6 and e32 > 4 * e64


def _flip_double_layer(orig):
    def f(x, f_t, f1_t, w, q, uD=None):
        return orig(x, f_t, f1_t, w, q, None if uD is None else -uD)
    return f


def _drop_jacobian(orig):
    def f(x, f_t, f1_t, w, q, uD=None):
        J = np.hypot(f1_t[0], f1_t[1])
        return orig(x, f_t, f1_t, w, q / J, uD)
    return f


def _shift_density(orig):
    def f(disc, alpha, s):
        return orig(disc, np.roll(np.asarray(alpha, np.float64).reshape(-1, disc.n), 1, axis=1), s)
    return f


@pytest.mark.parametrize("mutation", ["dl_sign", "jacobian", "density_shift"])
def test_planted_potential_mistake_is_caught(monkeypatch, mutation):
    if mutation == "dl_sign":
        monkeypatch.setattr(oa, "potential_sum", _flip_double_layer(oa.potential_sum))
    elif mutation == "jacobian":
        monkeypatch.setattr(oa, "potential_sum", _drop_jacobian(oa.potential_sum))
    else:
        monkeypatch.setattr(oa, "density_at", _shift_density(oa.density_at))
    caught = False
    try:
        test_circle_constant_density_and_data()
    except AssertionError:
        caught = True
    if not caught:
        try:
            test_solved_density_reproduces_interior_solution()
        except AssertionError:
            caught = True
    assert caught
