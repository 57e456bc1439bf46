"""The oracle's one-entry-at-a-time assembly (used for parity at n = 16384)
against the dense oracle, entry by entry, at small sizes (CPU only)."""
import numpy as np
import pytest

import oracle.assembly as oa
from oracle import bspline
from oracle.sampled import EntrySampler, local_basis
from paper_1703_10016_gb300 import workloads as wl


@pytest.mark.parametrize("kind", ["uniform", "clamped", "curve"])
def test_local_basis_matches_full_recurrence(kind):
    rng = np.random.default_rng(1)
    if kind == "uniform":
        d, knots = 4, np.arange(-4, 21, dtype=np.float64) / 16.0
    elif kind == "clamped":
        d, knots = 3, np.concatenate([[0.0] * 3, np.linspace(0.0, 1.0, 11), [1.0] * 3])
    else:
        c = wl.nurbs_circle(0.5)
        d, knots = c.degree, c.knots
    a, b = knots[d], knots[len(knots) - d - 1]
    x = np.concatenate([rng.uniform(a, b, 200), knots[d:len(knots) - d], [b]])
    full = bspline.basis_all(knots, d, x, nder=d)
    first, v = local_basis(knots, d, x, nder=d)
    for q in range(d + 1):
        for r in range(d + 1):
            np.testing.assert_allclose(v[q, :, r], full[q, first + r, np.arange(len(x))], rtol=1e-12, atol=1e-12)
        # every other function is zero at x
        mask = np.ones_like(full[q], dtype=bool)
        for r in range(d + 1):
            mask[first + r, np.arange(len(x))] = False
        assert np.all(full[q][mask] == 0.0)


@pytest.mark.parametrize("name,n,d,nref", [("star", 24, 3, 2), ("star", 20, 4, 3), ("circle", 16, 2, 1),
                                           ("arc", 14, 3, 2), ("star", 12, 5, 2), ("arc", 11, 4, 1)])
def test_entries_match_dense_oracle(name, n, d, nref):
    c = {"star": wl.star_curve(), "circle": wl.nurbs_circle(0.5), "arc": wl.parabola_arc()}[name]
    A = oa.assemble(c, n, d, nref)["A"]
    S = EntrySampler(c, n, d, nref)
    m = A.shape[0]
    pairs = [(0, 0), (0, m - 1), (m - 1, 0), (1, 2), (m // 2, m // 2 + 1), (3, m - 2), (m - 1, m - 1), (2, m // 2)]
    for i, j in pairs:
        assert abs(S.entry(i, j) - A[i, j]) <= 1e-14 * np.max(np.abs(A)), (i, j)


@pytest.mark.parametrize("name,n,d,nref", [("star", 24, 3, 2), ("circle", 16, 4, 2), ("arc", 14, 3, 2),
                                           ("star", 12, 5, 1)])
def test_rows_match_dense_oracle(name, n, d, nref):
    """Whole rows from the sparse row sampler (used for the CPU baseline at
    n = 16384) equal the dense oracle's rows."""
    from oracle.sampled import RowSampler
    c = {"star": wl.star_curve(), "circle": wl.nurbs_circle(0.5), "arc": wl.parabola_arc()}[name]
    A = oa.assemble(c, n, d, nref)["A"]
    R = RowSampler(c, n, d, nref)
    for i in (0, 1, A.shape[0] // 2, A.shape[0] - 1):
        np.testing.assert_allclose(R.row(i), A[i], rtol=0, atol=1e-14 * np.max(np.abs(A)))
