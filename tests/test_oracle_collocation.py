"""Pins for the oracle's collocation form (CPU only).

Independent references:
* circle of radius r: the single layer of a constant density is -r ln r on
  the circle, so the rows of Ac sum to -r ln r (the B_j sum to one), with
  the quadrature error shrinking under refinement;
* Gauss's identity: u_D = 1 gives beta_c = 1/2 - (1/2 pi) pi = 0;
* manufactured harmonic solutions with known flux (circle and star): the
  collocation solution converges to the flux;
* the collocation nodes are the Greville abscissae where those are nodes;
* planted mistakes (the K2 part dropped, the double-layer sign flipped, the
  collocation nodes moved by one) break one of the above.
"""
import numpy as np
import pytest

import oracle.assembly as oa
import oracle.collocation as oc
from oracle import bspline
from paper_1703_10016_gb300 import workloads as wl


def _row_sum_errors(r=0.5, ns=(16, 32, 64)):
    c = wl.nurbs_circle(r)
    return [np.max(np.abs(oc.collocation_matrix(c, n, 3, 2)[0].sum(axis=1) + r * np.log(r))) for n in ns]


def test_circle_rows_sum_to_constant_density_potential():
    e = _row_sum_errors()
    assert e[2] < 2e-5 and e[0] > 2.5 * e[1] > 6.0 * e[2]


def _gauss_identity_max():
    st = wl.star_curve()
    n, d = 128, 3
    eta, tg, _ = oa.rhs_points(st, n, d, 2)
    b = oc.collocation_rhs(st, n, d, 2, np.ones((len(eta), 1)), np.ones((len(tg), 1)))
    return np.max(np.abs(b))


def test_constant_data_gives_zero_rhs():
    """5e-13 with the 8-point b2 rule (the rule's error at the nodes)."""
    assert _gauss_identity_max() < 1e-11


def _manufactured(curve, n, d, data, nref=2):
    eta, tg, _ = oa.rhs_points(curve, n, d, nref)
    fe = bspline.curve_eval(curve, eta, 0)[0]
    fg = bspline.curve_eval(curve, tg, 0)[0]
    b = oc.collocation_rhs(curve, n, d, nref, data.value(*fe)[:, None], data.value(*fg)[:, None])
    Ac, _ = oc.collocation_matrix(curve, n, d, nref)
    alpha = oc.collocation_solve(Ac, b)[:, 0]

    def flux(s):
        f, f1 = bspline.curve_eval(curve, s, 1)
        nrm = oa.outward_normal(f1)
        gx, gy = data.grad(*f)
        return gx * nrm[0] + gy * nrm[1]
    return oa.errors(oa.make_discretization(curve, n, d, nref), alpha, flux)[0]


def test_manufactured_circle():
    e = [_manufactured(wl.nurbs_circle(0.5), n, 3, wl.Harmonic("x2-y2")) for n in (16, 32, 64)]
    assert e[2] < 1e-4 and e[0] > e[1] > e[2]


def test_manufactured_star():
    e = [_manufactured(wl.star_curve(), n, 3, wl.Harmonic("log")) for n in (32, 64, 128)]
    assert e[2] < 2e-4 and e[0] > e[1] > e[2]


@pytest.mark.parametrize("d,nref", [(2, 1), (3, 2), (4, 3), (5, 2)])
def test_nodes_are_greville_points(d, nref):
    """Away from the first and last refined element the support centre is a node."""
    disc = oa.make_discretization(wl.star_curve(), 40, d, nref)
    m = oc.collocation_nodes(disc)
    centre = np.mod(disc.a + disc.h * (np.arange(disc.Nh) + (1 - d) / 2.0) - disc.a, disc.L) + disc.a
    inner = (centre > disc.a + disc.hf) & (centre < disc.b - disc.hf)
    np.testing.assert_allclose(disc.eta[m[inner]], centre[inner], rtol=0, atol=1e-13)
    assert len(np.unique(m)) == disc.n


def test_open_arc_is_refused():
    with pytest.raises(ValueError):
        oc.collocation_nodes(oa.make_discretization(wl.parabola_arc(), 12, 2, 2))


def _drop_k2(orig):
    def f(disc, rows=None):
        return 0.0 * orig(disc, rows)
    return f


def _flip_kbar(orig):
    def f(*a, **k):
        return -orig(*a, **k)
    return f


def _shift_nodes(orig):
    def f(disc):
        return (orig(disc) + 1) % disc.Nq
    return f


@pytest.mark.parametrize("mutation", ["k2", "kbar_sign", "node_shift"])
def test_planted_collocation_mistake_is_caught(monkeypatch, mutation):
    from oracle import rules
    if mutation == "k2":
        monkeypatch.setattr(rules, "singular_rules", _drop_k2(rules.singular_rules))
    elif mutation == "kbar_sign":
        monkeypatch.setattr(oc, "kernel_Kbar", _flip_kbar(oc.kernel_Kbar))
    else:
        monkeypatch.setattr(oc, "collocation_nodes", _shift_nodes(oc.collocation_nodes))
    caught = []
    for pin in (test_circle_rows_sum_to_constant_density_potential, test_constant_data_gives_zero_rhs,
                test_manufactured_circle):
        try:
            pin()
        except AssertionError:
            caught.append(pin.__name__)
    assert caught


def test_matrix_rows_match_full():
    c = wl.star_curve()
    full, m = oc.collocation_matrix(c, 24, 3, 2)
    rows = np.array([0, 7, 23])
    part, mr = oc.collocation_matrix(c, 24, 3, 2, rows)
    assert np.array_equal(mr, m[rows])
    np.testing.assert_allclose(part, full[rows], rtol=1e-13, atol=1e-16)
