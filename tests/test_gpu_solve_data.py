"""igs_solve_data (right-hand side beside the factorisation) against
igs_build_rhs + igs_solve, in both tiers, host and device buffers, for a
first factorisation, a reused factor and a factorisation replayed from the
captured graph.  The refinement's residual norms are sums by atomic
addition, so two solves of the same system need not agree bit for bit: the
solutions are compared to the refinement's accuracy (FP64 tier: 1e-12; MIXED
tier: the 1e-10 residual bar times cond(A) < 1e4 gives 1e-6) and both must
meet the residual bar."""
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


@pytest.mark.parametrize("tier,n,nrhs", [("IGS_MIXED", 300, 3), ("IGS_FP64", 200, 1), ("IGS_MIXED", 4160, 2)])
def test_same_bits_as_separate_calls(ctx, tier, n, nrhs):
    g = lib()
    curve = wl.star_curve()
    runs = []
    for mode in ("separate", "together"):
        p = Prob(ctx, curve, n, 3, 1 if n > 4096 else 2, getattr(g, tier))
        try:
            xy = g.igs_rhs_points(p.prob)
            U = np.stack([wl.rhs_source(k, nrhs).value(xy[:, 0], xy[:, 1]) for k in range(nrhs)])
            out = []
            # first factorisation (issued directly), factor reused, factorisation again (graph)
            for assemble in (True, False, True):
                if assemble:
                    g.igs_assemble(p.prob)
                if mode == "separate":
                    g.igs_build_rhs(p.prob, U, return_beta=False)
                    alpha, res = g.igs_solve(p.prob, nrhs=nrhs)
                else:
                    alpha, res = g.igs_solve_data(p.prob, U)
                out.append((alpha.copy(), res.copy()))
            runs.append(out)
        finally:
            p.close()
    tol = 1e-12 if tier == "IGS_FP64" else 1e-6
    for (a1, r1), (a2, r2) in zip(*runs):
        assert np.linalg.norm(a1 - a2) <= tol * np.linalg.norm(a1)
        assert np.all(r1 <= 1e-10) and np.all(r2 <= 1e-10)


def test_device_buffers(ctx):
    torch = pytest.importorskip("torch")
    g = lib()
    p = Prob(ctx, wl.star_curve(), 256, 3, 2, g.IGS_MIXED)
    try:
        xy = g.igs_rhs_points(p.prob)
        U = wl.Harmonic("log").value(xy[:, 0], xy[:, 1])[None, :]
        g.igs_assemble(p.prob)
        ah, rh = g.igs_solve_data(p.prob, U)
        g.igs_assemble(p.prob)
        ad, rd = g.igs_solve_data(p.prob, torch.from_numpy(np.ascontiguousarray(U)).cuda())
        torch.cuda.synchronize()
        assert np.linalg.norm(ah - ad.cpu().numpy()) <= 1e-6 * np.linalg.norm(ah)
        assert np.all(rh <= 1e-10) and np.all(rd <= 1e-10)
        with pytest.raises(g.IgsError):
            g.igs_solve_data(p.prob, np.ones((9, p.info.n_rhs_pts)))
    finally:
        p.close()
