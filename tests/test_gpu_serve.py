"""Served form (GPU): requests of different curves, sizes, degrees and data
counts run through a server whose slots overlap on the device.  Each result
must be the same as when the request runs alone through the direct API: the
slots share no state, the same kernels run and every reduction has a fixed
order, so the solutions agree bit for bit."""
import numpy as np
import pytest

from paper_1703_10016_gb300 import workloads as wl
from tests._gpu import lib, needs_gpu

pytestmark = [pytest.mark.gpu, needs_gpu]


def _sources(k):
    return [2.5 * np.array([np.cos(2 * np.pi * j / 8), np.sin(2 * np.pi * j / 8)]) for j in range(k)]


def _data(xy, k):
    return np.stack([np.log(np.hypot(xy[:, 0] - s[0], xy[:, 1] - s[1])) for s in _sources(k)])


def _requests(g):
    rng = np.random.default_rng(21)
    reqs = []
    for n, d, nrhs in ((40, 2, 1), (64, 3, 2), (96, 4, 3), (128, 3, 1), (150, 2, 2), (72, 3, 8), (200, 3, 1)):
        reqs.append((wl.random_star(rng), d, n, 2, g.IGS_MIXED, nrhs))
    reqs.append((wl.parabola_arc(), 3, 30, 2, g.IGS_MIXED, 2))
    reqs.append((wl.star_curve(), 3, 64, 2, g.IGS_FP64, 2))
    return reqs


def _solo(g, curve, d, n_elems, nref, prec, nrhs):
    ctx = g.igs_create(0)
    geom = g.igs_create_geometry(ctx, curve.degree, curve.knots, curve.ctrl, curve.weights, curve.closed)
    p = g.igs_create_problem(geom, d, n_elems, nref, prec)
    try:
        g.igs_assemble(p)
        xy = g.igs_rhs_points(p)
        g.igs_build_rhs(p, _data(xy, nrhs))
        alpha, res = g.igs_solve(p, nrhs=nrhs)
        return alpha.reshape(nrhs, -1), res
    finally:
        g.igs_destroy_problem(p)
        g.igs_destroy_geometry(geom)
        g.igs_destroy(ctx)


def test_results_in_the_mix_equal_results_alone():
    g = lib()
    reqs = _requests(g)
    s = g.igs_server_create(0, slots=4, mem_budget=8 * 10**9)
    try:
        tickets = [g.igs_server_submit(s, c, d, n, r, p, k, _data) for c, d, n, r, p, k in reqs]
        g.igs_server_drain(s, 600_000)
        for t, (c, d, n, r, p, k) in zip(tickets, reqs):
            st = g.igs_server_wait(s, t)
            assert st["status"] == g.IGS_REQ_DONE, st
            alpha, res, st = g.igs_server_result(s, t, st["n"], k)
            assert np.all(res <= 1e-10)
            ref, rres = _solo(g, c, d, n, r, p, k)
            assert alpha.shape == ref.shape
            np.testing.assert_array_equal(alpha, ref)
            np.testing.assert_array_equal(res, rres)
            assert st["latency_ms"] >= st["run_ms"] > 0.0
    finally:
        g.igs_server_destroy(s)


def test_memory_admission_and_failures():
    g = lib()
    rng = np.random.default_rng(22)
    # a budget that admits one small request at a time: requests queue, all finish
    s = g.igs_server_create(0, slots=4, mem_budget=4 * 10**6)
    try:
        curves = [wl.random_star(rng) for _ in range(5)]
        tickets = [g.igs_server_submit(s, c, 3, 64, 2, g.IGS_MIXED, 1, _data) for c in curves]
        # too large for the budget: refused at submission
        with pytest.raises(g.IgsError) as e:
            g.igs_server_submit(s, curves[0], 3, 4096, 2, g.IGS_MIXED, 1, _data)
        assert e.value.code == g.IGS_E_ADMISSION_REFUSED
        # a failing data callback fails that request only

        def bad(xy, k):
            raise ValueError("no data")
        tb = g.igs_server_submit(s, curves[1], 3, 64, 2, g.IGS_MIXED, 1, bad)
        g.igs_server_drain(s, 600_000)
        for t in tickets:
            st = g.igs_server_wait(s, t)
            assert st["status"] == g.IGS_REQ_DONE
            assert st["device_bytes"] <= 4 * 10**6
            _, res, _ = g.igs_server_result(s, t, st["n"], 1)
            assert res[0] <= 1e-10
        st = g.igs_server_wait(s, tb)
        assert st["status"] == g.IGS_REQ_FAILED and st["error"] == g.IGS_E_INVALID_ARG
        with pytest.raises(g.IgsError):
            g.igs_server_result(s, tb, 64, 1)
        with pytest.raises(g.IgsError) as e:
            g.igs_server_wait(s, 10**9)
        assert e.value.code == g.IGS_E_INVALID_ARG
    finally:
        g.igs_server_destroy(s)


def test_many_mid_size_requests_on_eight_slots():
    """Heavier overlap (16 requests, n 500..2500, 8 slots): every factorisation
    and solve must still equal its solo result (this load exposed a shared-
    memory race in the Cholesky panel that a lone problem never hit)."""
    g = lib()
    rng = np.random.default_rng(23)
    reqs = []
    for _ in range(16):
        n = int(rng.integers(500, 2500))
        d = int(rng.integers(2, 5))
        reqs.append((wl.random_star(rng), d, n, 2, g.IGS_MIXED, int(rng.integers(1, 5))))
    s = g.igs_server_create(0, slots=8, mem_budget=64 * 10**9)
    try:
        tickets = [g.igs_server_submit(s, c, d, n, r, p, k, _data) for c, d, n, r, p, k in reqs]
        g.igs_server_drain(s, 600_000)
        for t, (c, d, n, r, p, k) in zip(tickets, reqs):
            st = g.igs_server_wait(s, t)
            assert st["status"] == g.IGS_REQ_DONE, st
            alpha, res, st = g.igs_server_result(s, t, st["n"], k)
            assert np.all(res <= 1e-10)
            ref, _ = _solo(g, c, d, n, r, p, k)
            np.testing.assert_array_equal(alpha, ref)
    finally:
        g.igs_server_destroy(s)


def test_large_requests_in_the_mix():
    """Sizes of the served workload's upper range (n up to 4160, both
    factorisation paths: per-panel below n = 4096, blocked by four panels on the
    tensor cores from 4096 up), 4 slots: results equal the solo runs bit for bit."""
    g = lib()
    rng = np.random.default_rng(24)
    reqs = [(wl.random_star(rng), d, n, 2 if n < 4096 else 1, g.IGS_MIXED, k)
            for n, d, k in ((4160, 3, 2), (1024, 4, 1), (3000, 2, 3), (4096, 4, 1), (2048, 3, 8), (700, 3, 2))]
    s = g.igs_server_create(0, slots=4, mem_budget=64 * 10**9)
    try:
        tickets = [g.igs_server_submit(s, c, d, n, r, p, k, _data) for c, d, n, r, p, k in reqs]
        g.igs_server_drain(s, 600_000)
        for t, (c, d, n, r, p, k) in zip(tickets, reqs):
            st = g.igs_server_wait(s, t)
            assert st["status"] == g.IGS_REQ_DONE, st
            alpha, res, st = g.igs_server_result(s, t, st["n"], k)
            assert np.all(res <= 1e-10)
            ref, _ = _solo(g, c, d, n, r, p, k)
            np.testing.assert_array_equal(alpha, ref)
    finally:
        g.igs_server_destroy(s)


def test_resident_problems_are_reused_and_change_no_result():
    """With a cache budget a slot keeps its last problems: the same
    discretisation on another curve reuses the rules (curve swapped in), the
    same curve reuses the matrix and factor too; results equal the solo runs."""
    g = lib()
    rng = np.random.default_rng(33)
    c1, c2 = wl.random_star(rng), wl.random_star(rng)
    s = g.igs_server_create(0, slots=1, mem_budget=4 * 10**9, cache_budget=2 * 10**9)
    try:
        plan = [(c1, 2, g.IGS_REUSE_NONE), (c1, 3, g.IGS_REUSE_FACTOR), (c2, 1, g.IGS_REUSE_RULES),
                (c2, 2, g.IGS_REUSE_FACTOR), (c1, 1, g.IGS_REUSE_RULES)]
        for curve, nrhs, want in plan:
            t = g.igs_server_submit(s, curve, 3, 160, 2, g.IGS_MIXED, nrhs, _data)
            st = g.igs_server_wait(s, t)
            assert st["status"] == g.IGS_REQ_DONE, st
            alpha, res, st = g.igs_server_result(s, t, st["n"], nrhs)
            assert st["reuse"] == want, (st["reuse"], want)
            ref, _ = _solo(g, curve, 3, 160, 2, g.IGS_MIXED, nrhs)
            assert np.all(res <= 1e-10)
            np.testing.assert_array_equal(alpha.reshape(nrhs, -1), ref)
        # another discretisation is built fresh
        t = g.igs_server_submit(s, c1, 3, 96, 2, g.IGS_MIXED, 1, _data)
        st = g.igs_server_wait(s, t)
        _, _, st = g.igs_server_result(s, t, st["n"], 1)
        assert st["reuse"] == g.IGS_REUSE_NONE
    finally:
        g.igs_server_destroy(s)


def test_no_cache_budget_means_no_reuse():
    g = lib()
    c = wl.star_curve()
    s = g.igs_server_create(0, slots=1, mem_budget=4 * 10**9)
    try:
        for _ in range(2):
            t = g.igs_server_submit(s, c, 3, 96, 2, g.IGS_MIXED, 1, _data)
            st = g.igs_server_wait(s, t)
            _, _, st = g.igs_server_result(s, t, st["n"], 1)
            assert st["reuse"] == g.IGS_REUSE_NONE
    finally:
        g.igs_server_destroy(s)
