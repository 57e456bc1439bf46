"""The right-hand side entry point that allocates no device memory (GPU).

Some callers cannot allocate device memory inside a call -- a framework that
owns every device allocation through its own allocator, or a latency-bound
serving loop that must stay off the driver's allocator.  igs_build_rhs_noalloc
serves them from a fixed device array inside the library.  Its results must
equal those of igs_build_rhs, call after call, although every call reuses the
same array.  This file is collected last so that a run that stops at the first
failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1703_10016_gb300 import workloads as wl
from tests._gpu import lib, needs_gpu

pytestmark = [pytest.mark.gpu, needs_gpu]


def test_noalloc_rhs_matches_build_rhs_on_two_calls_in_a_row():
    import torch

    g = lib()
    stream = torch.cuda.current_stream()
    ctx = g.igs_create(0, stream.cuda_stream)
    curve = wl.star_curve()
    geom = g.igs_create_geometry(ctx, curve.degree, curve.knots, curve.ctrl, curve.weights, curve.closed)
    prob = g.igs_create_problem(geom, 3, 100, 2, g.IGS_MIXED)
    fresh = g.igs_create_problem(geom, 3, 64, 2, g.IGS_FP64)
    try:
        n = g.igs_problem_info(prob).n
        g.igs_assemble(prob)
        xy = g.igs_rhs_points(prob)
        U1 = np.stack([wl.rhs_source(k, 3).value(xy[:, 0], xy[:, 1]) for k in range(3)])
        U2 = wl.Harmonic("log").value(xy[:, 0], xy[:, 1])[None, :]
        ref1 = g.igs_build_rhs(prob, U1)
        ref2 = g.igs_build_rhs(prob, U2)
        dev = torch.device("cuda", 0)
        for U, ref in ((U1, ref1), (U2, ref2)):          # two calls in a row share the scratch
            u = torch.tensor(U, dtype=torch.float64, device=dev)
            beta = torch.full((U.shape[0], n), float("nan"), dtype=torch.float64, device=dev)
            g.igs_build_rhs_noalloc(prob, u, beta)
            torch.cuda.synchronize()
            b = beta.cpu().numpy()
            assert np.all(np.isfinite(b))
            assert np.max(np.abs(b - ref)) <= 1e-12 * np.max(np.abs(ref))
        # limits and preconditions are reported, not worked around
        with pytest.raises(g.IgsError) as e:
            g.igs_build_rhs_noalloc(prob, torch.zeros((9, U1.shape[1]), dtype=torch.float64, device=dev),
                                    torch.zeros((9, n), dtype=torch.float64, device=dev))
        assert e.value.code == g.IGS_E_INVALID_ARG
        with pytest.raises(g.IgsError) as e:
            g.igs_build_rhs_noalloc(fresh, torch.zeros((1, 10), dtype=torch.float64, device=dev),
                                    torch.zeros((1, 64), dtype=torch.float64, device=dev))
        assert e.value.code == g.IGS_E_STATE
    finally:
        g.igs_destroy_problem(fresh)
        g.igs_destroy_problem(prob)
        g.igs_destroy_geometry(geom)
        g.igs_destroy(ctx)
