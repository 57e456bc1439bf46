"""Batched form (GPU): many MIXED-tier assemblies in one persistent launch.

Each problem's matrix from the batch must be the one the single-problem path
produces for it (the per-tile arithmetic is shared), whatever the tile size,
unit order or CTAs per SM the autotuner picks; two of them are also checked
against the oracle within the MIXED bar.
"""
import numpy as np
import pytest

from oracle import assembly as oa
from paper_1703_10016_gb300 import workloads as wl
from tests._gpu import Prob, lib, needs_gpu

pytestmark = [pytest.mark.gpu, needs_gpu]


def relF(A, B):
    return float(np.linalg.norm(A - B) / np.linalg.norm(B))


def _mix():
    rng = np.random.default_rng(11)
    out = []
    for n, d, nref in ((40, 2, 2), (64, 3, 2), (97, 4, 2), (150, 3, 2), (33, 3, 1), (72, 2, 3), (210, 3, 2)):
        out.append((wl.random_star(rng), n, d, nref))
    out.append((wl.parabola_arc(), 45, 3, 2))
    out.append((wl.nurbs_circle(0.5), 64, 3, 2))
    return out


@pytest.fixture(scope="module")
def ctx():
    g = lib()
    c = g.igs_create(0)
    yield c
    g.igs_destroy(c)


def _matrix(g, prob):
    n = g.igs_problem_info(prob).n
    A = np.empty((n, n), dtype=np.float64)
    g.igs_get_matrix(prob, A)
    return A


def test_batch_matches_single_problem_path_and_oracle(ctx):
    g = lib()
    mix = _mix()
    batch_probs = [Prob(ctx, c, n, d, nref, g.IGS_MIXED) for c, n, d, nref in mix]
    single = [Prob(ctx, c, n, d, nref, g.IGS_MIXED) for c, n, d, nref in mix]
    b = g.igs_batch_create(ctx, [p.prob for p in batch_probs])
    try:
        ref = [p.assemble() for p in single]
        configs = [dict(tile=32, order=g.IGS_ORDER_NATURAL), dict(tile=16, order=g.IGS_ORDER_INTERLEAVED),
                   dict(tile=32, order=g.IGS_ORDER_LARGEST_FIRST, ctas_per_sm=1)]
        for cfg in configs:
            g.igs_batch_set_config(b, **cfg)
            for _ in range(2):                       # the graph is replayed
                ms = g.igs_batch_assemble(b)
                assert ms > 0.0
                for p, R in zip(batch_probs, ref):
                    A = _matrix(g, p.prob)
                    assert np.max(np.abs(A - R)) <= 1e-6 * np.max(np.abs(R)), cfg
        # oracle on two members (closed star, open arc)
        for k in (1, 7):
            c, n, d, nref = mix[k]
            assert relF(_matrix(g, batch_probs[k].prob), oa.assemble(c, n, d, nref)["A"]) <= 1e-6
        # autotuner: picks a configuration and keeps the results
        best = g.igs_batch_tune(b, reps=1)
        assert best["tile"] in (16, 32) and best["ms"] > 0.0 and best["ctas_per_sm"] >= 1
        assert g.igs_batch_get_config(b)["tile"] == best["tile"]
        g.igs_batch_assemble(b)
        for p, R in zip(batch_probs, ref):
            assert np.max(np.abs(_matrix(g, p.prob) - R)) <= 1e-6 * np.max(np.abs(R))
        # a held problem cannot be destroyed
        with pytest.raises(g.IgsError) as e:
            g.igs_destroy_problem(batch_probs[0].prob)
        assert e.value.code == g.IGS_E_STATE
    finally:
        g.igs_batch_destroy(b)
        for p in batch_probs + single:
            g.igs_destroy_problem(p.prob)
            g.igs_destroy_geometry(p.geom)


def test_batch_follows_geometry_change_and_solves(ctx):
    g = lib()
    rng = np.random.default_rng(12)
    curves = [wl.random_star(rng) for _ in range(3)]
    probs = [Prob(ctx, c, 64, 3, 2, g.IGS_MIXED) for c in curves]
    b = g.igs_batch_create(ctx, [p.prob for p in probs])
    extra = []
    try:
        g.igs_batch_assemble(b)
        new = wl.random_star(rng)
        g2 = g.igs_create_geometry(ctx, new.degree, new.knots, new.ctrl, new.weights, new.closed)
        extra.append(g2)
        g.igs_set_geometry(probs[1].prob, g2)
        g.igs_batch_assemble(b)
        ref = Prob(ctx, new, 64, 3, 2, g.IGS_MIXED)
        try:
            R = ref.assemble()
            A = _matrix(g, probs[1].prob)
            assert np.max(np.abs(A - R)) <= 1e-6 * np.max(np.abs(R))
        finally:
            g.igs_destroy_problem(ref.prob)
            g.igs_destroy_geometry(ref.geom)
        # the batch leaves each problem ready to solve
        for p in probs:
            xy = g.igs_rhs_points(p.prob)
            U = wl.Harmonic("log").value(xy[:, 0], xy[:, 1])[None, :]
            g.igs_build_rhs(p.prob, U)
            _, res = g.igs_solve(p.prob)
            assert res[0] <= 1e-10
    finally:
        g.igs_batch_destroy(b)
        for p in probs:
            g.igs_destroy_problem(p.prob)
            g.igs_destroy_geometry(p.geom)
        for g2 in extra:
            g.igs_destroy_geometry(g2)


def test_batch_rejects_fp64_and_foreign_problems(ctx):
    g = lib()
    p = Prob(ctx, wl.star_curve(), 40, 3, 2, g.IGS_FP64)
    try:
        with pytest.raises(g.IgsError) as e:
            g.igs_batch_create(ctx, [p.prob])
        assert e.value.code == g.IGS_E_INVALID_ARG
    finally:
        g.igs_destroy_problem(p.prob)
        g.igs_destroy_geometry(p.geom)
