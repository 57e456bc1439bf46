"""The MIXED tier's double-layer sum (b2 of Sect. 5) by a treecode (GPU).

The treecode groups the Gauss points of the b2 rule in parameter order; its
clusters are accepted by their distance in space.  These cases check it where
that distinction matters and where its cluster geometry must follow the curve:

* a curve with a narrow waist, r = 0.4 (1 + 0.8 cos 2 theta): arcs far apart in
  parameter come within 0.16 of each other, at a size where the tree has nine
  levels (beta within the MIXED bar of the oracle's direct sum);
* a geometry change on a problem whose clusters were built for another curve
  (the rebuilt clusters give the same beta as a fresh problem, bit for bit).
"""
import numpy as np
import pytest

import oracle.assembly as oa
from oracle import bspline
from paper_1703_10016_gb300 import workloads as wl

from tests._gpu import Prob, lib, needs_gpu

pytestmark = [pytest.mark.gpu, needs_gpu]


@pytest.fixture(scope="module")
def ctx():
    g = lib()
    c = g.igs_create(0)
    yield c
    g.igs_destroy(c)


def _rhs_bar(tol, S, K):
    # the bar of the parity tests: tol max |terms| + 4 one-ulp sensitivities
    return tol * np.max(np.abs(S)) + 4.0 * np.max(np.abs(K))


def test_treecode_on_a_waisted_curve(ctx):
    curve = wl.star_curve(amp=0.8, k=2)
    n, d, nref = 512, 3, 2
    data = wl.Harmonic("log")
    eta, tg, _ = oa.rhs_points(curve, n, d, nref)
    un = data.value(*bspline.curve_eval(curve, eta, 0)[0])
    ug = data.value(*bspline.curve_eval(curve, tg, 0)[0])
    beta_ref, S, K = oa.build_rhs(curve, n, d, nref, un[:, None], ug[:, None], magnitude=True)
    p = Prob(ctx, curve, n, d, nref, lib().IGS_MIXED)
    try:
        beta = lib().igs_build_rhs(p.prob, np.concatenate([un, ug])[None, :])[0]
        assert np.all(np.isfinite(beta))
        assert np.max(np.abs(beta - beta_ref[:, 0])) <= _rhs_bar(1e-6, S, K)
    finally:
        p.close()


def test_treecode_follows_a_geometry_change(ctx):
    g = lib()
    rng = np.random.default_rng(21)
    first, second = wl.random_star(rng), wl.star_curve(amp=0.5, k=3)
    n, d, nref = 96, 3, 2
    p = Prob(ctx, first, n, d, nref, g.IGS_MIXED)
    fresh = Prob(ctx, second, n, d, nref, g.IGS_MIXED)
    g2 = g.igs_create_geometry(ctx, second.degree, second.knots, second.ctrl, second.weights, second.closed)
    try:
        xy = g.igs_rhs_points(p.prob)
        g.igs_build_rhs(p.prob, wl.Harmonic("log").value(xy[:, 0], xy[:, 1])[None, :])
        g.igs_set_geometry(p.prob, g2)
        xy2 = g.igs_rhs_points(p.prob)
        U = wl.Harmonic("log").value(xy2[:, 0], xy2[:, 1])[None, :]
        beta = g.igs_build_rhs(p.prob, U)
        xyf = g.igs_rhs_points(fresh.prob)
        np.testing.assert_array_equal(xy2, xyf)
        ref = g.igs_build_rhs(fresh.prob, U)
        np.testing.assert_array_equal(beta, ref)
    finally:
        p.close()
        fresh.close()
        g.igs_destroy_geometry(g2)
