"""igs_assemble without a copy returns before its kernels finish (GPU).

Later calls on the problem are ordered after the queued kernels on the
context stream, and igs_problem_timing waits for them: the matrix read back
right after the call equals the one an assembly with a copy returns, bit for
bit, and the assembly time is reported.
"""
import numpy as np
import pytest

from paper_1703_10016_gb300 import workloads as wl

from tests._gpu import Prob, lib, needs_gpu

pytestmark = [pytest.mark.gpu, needs_gpu]


@pytest.fixture(scope="module")
def ctx():
    g = lib()
    c = g.igs_create(0)
    yield c
    g.igs_destroy(c)


@pytest.mark.parametrize("tier", ["MIXED", "FP64"])
def test_queued_assembly_orders_later_calls(ctx, tier):
    g = lib()
    curve = wl.star_curve()
    p = Prob(ctx, curve, 160, 3, 2, getattr(g, "IGS_" + tier))
    q = Prob(ctx, curve, 160, 3, 2, getattr(g, "IGS_" + tier))
    try:
        n = p.info.n
        g.igs_assemble(p.prob)                       # queued, returns at once
        A = np.empty((n, n))
        g.igs_get_matrix(p.prob, A)                  # ordered after the assembly
        B = q.assemble()                             # assembly with a copy
        np.testing.assert_array_equal(A, B)
        t = g.igs_problem_timing(p.prob)
        assert t.assemble_ms > 0 and t.geometry_ms > 0
        xy = g.igs_rhs_points(p.prob)
        g.igs_assemble(p.prob)                       # again, then solve on the same stream
        U = wl.Harmonic("log").value(xy[:, 0], xy[:, 1])[None, :]
        alpha, res = g.igs_solve_data(p.prob, U)
        assert res[0] <= 1e-10 and np.all(np.isfinite(alpha))
    finally:
        p.close()
        q.close()
