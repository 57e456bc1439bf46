"""igs_solve_data (right-hand side beside the factorisation) against
igs_build_rhs + igs_solve, in both tiers, host and device buffers, for a
first factorisation, a reused factor and a factorisation replayed from the
captured graph.  Every reduction on the path has a fixed order (the
refinement's residual norms included), so the two routes give the same bits."""
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
    for (a1, r1), (a2, r2) in zip(*runs):
        np.testing.assert_array_equal(a1, a2)
        np.testing.assert_array_equal(r1, r2)
        assert np.all(r1 <= 1e-10)
    # the same problem solved again gives the same bits
    np.testing.assert_array_equal(runs[0][0][0], runs[0][2][0])


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
        np.testing.assert_array_equal(ah, ad.cpu().numpy())
        np.testing.assert_array_equal(rh, rd)
        assert np.all(rh <= 1e-10)
        with pytest.raises(g.IgsError):
            g.igs_solve_data(p.prob, np.ones((9, p.info.n_rhs_pts)))
    finally:
        p.close()
