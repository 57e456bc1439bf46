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

SCRATCH_DOUBLES = 1 << 21          # the library's fixed array: 16 MiB of doubles


@pytest.fixture(scope="module")
def ctx():
    import torch
    g = lib()
    c = g.igs_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    g.igs_destroy(c)


def _check_two_calls(g, prob, n, curve_closed):
    import torch
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
        # the same kernels on the same data in the same order: equal to rounding
        assert np.max(np.abs(b - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("tier", ["FP64", "MIXED"])
def test_noalloc_rhs_matches_build_rhs_on_two_calls_in_a_row(ctx, tier):
    g = lib()
    curve = wl.star_curve()
    geom = g.igs_create_geometry(ctx, curve.degree, curve.knots, curve.ctrl, curve.weights, curve.closed)
    prob = g.igs_create_problem(geom, 3, 100, 2, getattr(g, "IGS_" + tier))
    try:
        _check_two_calls(g, prob, g.igs_problem_info(prob).n, True)
    finally:
        g.igs_destroy_problem(prob)
        g.igs_destroy_geometry(geom)


def test_noalloc_rhs_open_arc(ctx):
    """Open arc: beta = b1, no double-layer term and so no scratch at all."""
    g = lib()
    curve = wl.parabola_arc()
    geom = g.igs_create_geometry(ctx, curve.degree, curve.knots, curve.ctrl, curve.weights, curve.closed)
    prob = g.igs_create_problem(geom, 3, 37, 2, g.IGS_MIXED)
    try:
        _check_two_calls(g, prob, g.igs_problem_info(prob).n, False)
    finally:
        g.igs_destroy_problem(prob)
        g.igs_destroy_geometry(geom)


# MIXED: the potentials plus the treecode's moments and FP32 data products,
# 1 + ceil((28 C + N_GQ / 2) / n_quad) slots (C clusters); FP64: 8 Gauss slices
@pytest.mark.parametrize("tier,slots,n", [("MIXED", 11, 3000), ("FP64", 8, 4096)])
def test_noalloc_rhs_limit(ctx, tier, slots, n):
    """Sizes just above the fixed array are refused with INVALID_ARG, one data
    set fewer fits; the preconditions are reported, not worked around."""
    import torch
    g = lib()
    curve = wl.star_curve()
    dev = torch.device("cuda", 0)
    geom = g.igs_create_geometry(ctx, curve.degree, curve.knots, curve.ctrl, curve.weights, curve.closed)
    prob = g.igs_create_problem(geom, 3, n, 4, getattr(g, "IGS_" + tier))
    fresh = g.igs_create_problem(geom, 3, 64, 2, g.IGS_FP64)
    try:
        info = g.igs_problem_info(prob)
        assert info.rhs_slots == slots
        assert slots * info.n_quad * 8 > SCRATCH_DOUBLES >= slots * info.n_quad * 7
        xy = g.igs_rhs_points(prob)                    # rules, node geometry, rhs points
        u = torch.tensor(np.stack([wl.rhs_source(k, 8).value(xy[:, 0], xy[:, 1]) for k in range(8)]),
                         dtype=torch.float64, device=dev)
        beta = torch.zeros((8, info.n), dtype=torch.float64, device=dev)
        with pytest.raises(g.IgsError) as e:
            g.igs_build_rhs_noalloc(prob, u, beta)
        assert e.value.code == g.IGS_E_INVALID_ARG
        b7 = beta[:7].contiguous()
        g.igs_build_rhs_noalloc(prob, u[:7].contiguous(), b7)
        ref = g.igs_build_rhs(prob, u[:7].cpu().numpy())
        torch.cuda.synchronize()
        assert np.max(np.abs(b7.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
        # a wrong shape is refused by the binding before the library is reached
        with pytest.raises(g.IgsError) as e:
            g.igs_build_rhs_noalloc(prob, u[:2], torch.zeros((2, info.n - 1), dtype=torch.float64, device=dev))
        assert e.value.code == g.IGS_E_INVALID_ARG
        with pytest.raises(g.IgsError) as e:
            g.igs_build_rhs_noalloc(fresh, torch.zeros((1, g.igs_problem_info(fresh).n_rhs_pts), dtype=torch.float64,
                                                       device=dev),
                                    torch.zeros((1, 64), dtype=torch.float64, device=dev))
        assert e.value.code == g.IGS_E_STATE
    finally:
        g.igs_destroy_problem(fresh)
        g.igs_destroy_problem(prob)
        g.igs_destroy_geometry(geom)
