"""Bounded waits between thread blocks (the triangular solves' word waits):
a wait on a word that nothing writes gives up by its budget and the context
stays usable for a full solve afterwards."""
import numpy as np
import pytest

from paper_1703_10016_gb300 import igs
from paper_1703_10016_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_wait_gives_up_and_context_survives():
    ctx = igs.igs_create(0)
    try:
        assert igs.igs_selftest_wait(ctx, 0.005) == 1
        c = wl.star_curve()
        geom = igs.igs_create_geometry(ctx, c.degree, c.knots, c.ctrl, c.weights, c.closed)
        prob = igs.igs_create_problem(geom, 3, 256, 2, igs.IGS_MIXED)
        igs.igs_assemble(prob)
        xy = igs.igs_rhs_points(prob)
        igs.igs_build_rhs(prob, wl.Harmonic("log").value(xy[:, 0], xy[:, 1])[None, :])
        alpha, res = igs.igs_solve(prob)
        assert np.all(np.isfinite(alpha)) and res[0] <= 1e-10
        igs.igs_destroy_problem(prob)
        igs.igs_destroy_geometry(geom)
    finally:
        igs.igs_destroy(ctx)
