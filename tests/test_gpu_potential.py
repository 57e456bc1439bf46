"""Representation formula (Sect. 2) on the GPU against the oracle, through the C ABI.

FP64 evaluation in every tier: the bar is 1e-12 relative Frobenius error
against oracle.assembly.eval_potential on the same density, data and points.
"""
import numpy as np
import pytest

import oracle.assembly as oa
from oracle import bspline
from paper_1703_10016_gb300 import workloads as wl
from tests._gpu import Prob, lib, needs_gpu, relF

pytestmark = [pytest.mark.gpu, needs_gpu]

TOL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    g = lib()
    c = g.igs_create(0)
    yield c
    g.igs_destroy(c)


def interior_points(rng, count, rmax):
    """Seeded points in the disc of radius rmax (inside the star, whose radius is >= 0.32)."""
    r = rmax * np.sqrt(rng.uniform(0.0, 1.0, count))
    th = rng.uniform(0.0, 2.0 * np.pi, count)
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)


@pytest.mark.parametrize("nrhs,count", [(1, 1), (3, 1000), (8, 333)])
def test_closed_curve_matches_oracle(ctx, nrhs, count):
    """Random density and data (the evaluation alone), star curve, ragged point counts."""
    rng = np.random.default_rng(11 + nrhs)
    c = wl.star_curve()
    n, d, nref = 64, 3, 2
    p = Prob(ctx, c, n, d, nref, lib().IGS_FP64)
    try:
        npts = p.info.n_rhs_pts
        alpha = rng.standard_normal((nrhs, p.info.n))
        uD = rng.standard_normal((nrhs, npts))
        pts = interior_points(rng, count, 0.28)
        u = lib().igs_eval_potential(p.prob, alpha, uD, pts)
        Nq = p.info.n_quad
        ref = oa.eval_potential(c, n, d, nref, alpha, uD[:, Nq:], pts)
        assert u.shape == (nrhs, count)
        assert relF(u, ref) < TOL
    finally:
        p.close()


def test_open_arc_matches_oracle(ctx):
    """Parabola (indirect method: single layer only), points on both sides of the arc."""
    rng = np.random.default_rng(5)
    c = wl.parabola_arc()
    n, d, nref = 24, 2, 2
    p = Prob(ctx, c, n, d, nref, lib().IGS_MIXED)
    try:
        alpha = rng.standard_normal((2, p.info.n))
        pts = np.stack([rng.uniform(-2, 2, 777), rng.uniform(-1.5, 3.0, 777)], axis=1)
        # keep points away from the arc x2 = 1 - x1^2, |x1| <= 1
        keep = (np.abs(pts[:, 0]) > 1.2) | (np.abs(pts[:, 1] - (1 - pts[:, 0] ** 2)) > 0.2)
        pts = np.ascontiguousarray(pts[keep])
        u = lib().igs_eval_potential(p.prob, alpha, None, pts)
        ref = oa.eval_potential(c, n, d, nref, alpha, None, pts)
        assert relF(u, ref) < TOL
    finally:
        p.close()


def test_device_buffers_match_host(ctx):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    c = wl.star_curve()
    p = Prob(ctx, c, 48, 2, 2, lib().IGS_MIXED)
    try:
        alpha = rng.standard_normal((2, p.info.n))
        uD = rng.standard_normal((2, p.info.n_rhs_pts))
        pts = interior_points(rng, 5000, 0.3)
        uh = lib().igs_eval_potential(p.prob, alpha, uD, pts)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        ud = lib().igs_eval_potential(p.prob, dev(alpha), dev(uD), dev(pts))
        torch.cuda.synchronize()
        assert np.array_equal(uh, ud.cpu().numpy())
    finally:
        p.close()


@pytest.mark.parametrize("tier,tol", [("IGS_FP64", 1e-9), ("IGS_MIXED", 1e-5)])
def test_solved_density_reproduces_harmonic_solution(ctx, tier, tol):
    """The whole method on the GPU (n = 512): rules, assembly, right-hand
    side, solve, then the representation formula at interior points gives
    u = log|x - x0| to the discretisation's accuracy (3e-11 with the FP64
    oracle at this size; the MIXED tier's FP32 matrix bounds it near 1e-7)."""
    c = wl.star_curve()
    n, d, nref = 512, 3, 2
    p = Prob(ctx, c, n, d, nref, getattr(lib(), tier))
    try:
        hl = wl.Harmonic("log")
        xy = lib().igs_rhs_points(p.prob)
        uD = np.ascontiguousarray(hl.value(xy[:, 0], xy[:, 1])[None, :])
        p.assemble(np.float64 if tier == "IGS_FP64" else np.float32)
        lib().igs_build_rhs(p.prob, uD)
        alpha, res = lib().igs_solve(p.prob)
        pts = interior_points(np.random.default_rng(9), 2000, 0.25)
        u = lib().igs_eval_potential(p.prob, alpha, uD, pts)
        err = np.max(np.abs(u[0] - hl.value(pts[:, 0], pts[:, 1])))
        assert err < tol
    finally:
        p.close()


def test_full_size_sampled_points(ctx):
    """n = 2048 star (the size of the single-matrix workload): 512 sampled
    interior points against the oracle at the same size."""
    rng = np.random.default_rng(21)
    c = wl.star_curve()
    n, d, nref = 2048, 3, 2
    p = Prob(ctx, c, n, d, nref, lib().IGS_MIXED)
    try:
        alpha = rng.standard_normal((1, p.info.n)) / np.sqrt(n)
        uD = rng.standard_normal((1, p.info.n_rhs_pts))
        pts = interior_points(rng, 512, 0.3)
        u = lib().igs_eval_potential(p.prob, alpha, uD, pts)
        ref = oa.eval_potential(c, n, d, nref, alpha, uD[:, p.info.n_quad:], pts)
        assert relF(u, ref) < TOL
    finally:
        p.close()


def test_argument_errors_and_empty(ctx):
    g = lib()
    c = wl.star_curve()
    p = Prob(ctx, c, 32, 2, 2, g.IGS_FP64)
    try:
        alpha = np.ones((1, p.info.n))
        with pytest.raises(g.IgsError):
            g.igs_eval_potential(p.prob, alpha, None, np.zeros((4, 2)))     # closed curve needs u_D
        u = g.igs_eval_potential(p.prob, alpha, np.ones((1, p.info.n_rhs_pts)), np.zeros((0, 2)))
        assert u.shape == (1, 0)
    finally:
        p.close()
