"""Collocation form (the Sect. 7 remark) on the GPU against the oracle, through the C ABI.

Bars: the collocation nodes are identical; the FP64 matrix within 1e-12
relative Frobenius error in both tiers (it is FP64 in both); the solution's
normwise backward error in the oracle's system (the right-hand side measured
by the size of its two cancelling terms u_D/2 and v/(2 pi)) below 2e-12 in
the FP64 tier (matrix plus right-hand side differences) and below 1e-6 in the
MIXED tier (FP32 far-field node potentials); FP64 forward error within the
backward bound times cond(Ac).
"""
import numpy as np
import pytest

import oracle.assembly as oa
import oracle.collocation as oc
from oracle import bspline
from paper_1703_10016_gb300 import workloads as wl
from tests._gpu import Prob, lib, needs_gpu, relF

pytestmark = [pytest.mark.gpu, needs_gpu]


@pytest.fixture(scope="module")
def ctx():
    g = lib()
    c = g.igs_create(0)
    yield c
    g.igs_destroy(c)


def _data(curve, n, d, nref, nrhs):
    eta, tg, _ = oa.rhs_points(curve, n, d, nref)
    fe = bspline.curve_eval(curve, eta, 0)[0]
    fg = bspline.curve_eval(curve, tg, 0)[0]
    un = np.stack([wl.rhs_source(k, nrhs).value(*fe) for k in range(nrhs)])
    ug = np.stack([wl.rhs_source(k, nrhs).value(*fg) for k in range(nrhs)])
    return un, ug


@pytest.mark.parametrize("name,n,d,nref", [("star", 100, 3, 2), ("star", 45, 2, 1), ("circle", 64, 4, 3),
                                           ("star", 30, 5, 2)])
def test_matrix_nodes_and_solution_match_oracle(ctx, name, n, d, nref):
    curve = wl.star_curve() if name == "star" else wl.nurbs_circle(0.5)
    Ac_ref, m_ref = oc.collocation_matrix(curve, n, d, nref)
    un, ug = _data(curve, n, d, nref, 3)
    beta_ref = oc.collocation_rhs(curve, n, d, nref, un.T, ug.T)
    alpha_ref = oc.collocation_solve(Ac_ref, beta_ref).T
    for tier in ("IGS_FP64", "IGS_MIXED"):
        p = Prob(ctx, curve, n, d, nref, getattr(lib(), tier))
        try:
            alpha, Ac, nodes = lib().igs_collocation(p.prob, np.concatenate([un, ug], axis=1), return_matrix=True)
            assert np.array_equal(nodes, m_ref)
            # d = 5: the local systems of Algorithm 1 carry ~1e-10 relative rule error in any FP64 solution
            assert relF(Ac, Ac_ref) < (1e-12 if d <= 4 else 1e-9), tier
            # normwise backward error of the GPU solution in the oracle's system: at most
            # the matrix difference plus the right-hand side difference plus the LU's own
            # O(n eps), i.e. 2e-12 in the FP64 tier (2e-9 for d = 5) and 1e-6 in the MIXED tier.
            # beta_c = u_D/2 - v/(2 pi) cancels (|beta_c| is about |u_D|/9 here), so the
            # right-hand side is measured by the size of its two terms.
            half_u = un[:, m_ref].T / 2.0
            scale_b = np.linalg.norm(half_u) + np.linalg.norm(half_u - beta_ref)
            back = np.linalg.norm(Ac_ref @ alpha.T - beta_ref) / (
                np.linalg.norm(Ac_ref) * np.linalg.norm(alpha) + scale_b)
            if tier == "IGS_FP64":
                assert back < (2e-12 if d <= 4 else 2e-9)
                # forward error: the backward error times the condition number (and the
                # right-hand side's cancellation factor)
                amp = scale_b / np.linalg.norm(beta_ref)
                assert relF(alpha, alpha_ref) < 2e-12 * amp * np.linalg.cond(Ac_ref) * (1 if d <= 4 else 1e3)
            else:
                assert back < 1e-6
        finally:
            p.close()


def test_manufactured_solution_converges(ctx):
    """u = x^2 - y^2 on the circle: the GPU collocation solution has the
    oracle's discretisation error (the flux cos 2 theta)."""
    curve = wl.nurbs_circle(0.5)
    data = wl.Harmonic("x2-y2")
    errs = []
    for n in (16, 32, 64):
        p = Prob(ctx, curve, n, 3, 2, lib().IGS_FP64)
        try:
            xy = lib().igs_rhs_points(p.prob)
            alpha = lib().igs_collocation(p.prob, data.value(xy[:, 0], xy[:, 1])[None, :])[0]

            def flux(s):
                f, f1 = bspline.curve_eval(curve, s, 1)
                nrm = oa.outward_normal(f1)
                gx, gy = data.grad(*f)
                return gx * nrm[0] + gy * nrm[1]
            errs.append(oa.errors(oa.make_discretization(curve, n, 3, 2), alpha, flux)[0])
        finally:
            p.close()
    assert errs[2] < 1e-4 and errs[0] > errs[1] > errs[2]


def test_full_size_sampled_rows_and_residual(ctx):
    """n = 2048 star (the size of the single-matrix workload): sampled rows of
    Ac against the oracle, identical nodes, and the solution satisfies the
    oracle's collocation system."""
    curve = wl.star_curve()
    n, d, nref = 2048, 3, 2
    rows = np.array([0, 1, 1024, 2046, 2047])
    Ac_rows, m_rows = oc.collocation_matrix(curve, n, d, nref, rows)
    un, ug = _data(curve, n, d, nref, 1)
    beta_ref = oc.collocation_rhs(curve, n, d, nref, un.T, ug.T)[:, 0]
    p = Prob(ctx, curve, n, d, nref, lib().IGS_FP64)
    try:
        alpha, Ac, nodes = lib().igs_collocation(p.prob, np.concatenate([un, ug], axis=1), return_matrix=True)
        assert np.array_equal(nodes[rows], m_rows)
        assert relF(Ac[rows], Ac_rows) < 1e-12
        assert np.linalg.norm(Ac @ alpha[0] - beta_ref) <= 1e-10 * np.linalg.norm(beta_ref)
    finally:
        p.close()


def test_arguments(ctx):
    g = lib()
    p = Prob(ctx, wl.parabola_arc(), 12, 2, 2, g.IGS_FP64)
    try:
        with pytest.raises(g.IgsError) as e:
            g.igs_collocation(p.prob, np.ones((1, p.info.n_rhs_pts)))
        assert e.value.code == g.IGS_E_INVALID_ARG
    finally:
        p.close()
    p = Prob(ctx, wl.star_curve(), 16, 3, 2, g.IGS_FP64)
    try:
        with pytest.raises(g.IgsError) as e:
            g.igs_collocation(p.prob, np.ones((9, p.info.n_rhs_pts)))
        assert e.value.code == g.IGS_E_INVALID_ARG
    finally:
        p.close()
