"""Single entries of A at large size (oracle; test infrastructure only).

The dense oracle (`assembly.assemble`, `assembly.assemble_rows`) forms
N_quad x n and N_E x N_quad arrays, which do not fit in memory at n = 16384.
The functions here compute one entry A[i, j] by the same definitions, each
restricted to the pieces the entry touches:

* B-spline values: the Cox-de Boor recurrence of `bspline.basis_all` on the
  2d + 2 knots around the point's knot interval (a B-spline depends only on
  its own knots, so the d + 1 non-zero values are the same numbers);
* the regular rule w^(i) of Algorithm 1 for the two test functions i, j:
  moments mu^(i)_j = int B-bar_j B_i by Gauss with d + 1 points on the refined
  elements of supp(B_i), the local collocation matrix (B)^(i) on J^(i) x N^(i),
  minimum-norm solution;
* the Gram matrix G = (B)(B)^T of Algorithm 2 as a band, accumulated node by
  node, and its banded Cholesky factor;
* the modified moments mu_k(s) of eq. mod_mom_gen at the nodes N^(i): the sum
  over refined elements of the elements' polynomial pieces (right-sided
  Taylor coefficients at the left end) against int_e u^k K2(s, t) dt;
* the singular weights W^s[n][n'] = sum_k B-bar_k(eta_n') (G^{-1} mu(eta_n))_k
  for n in N^(i), n' in N^(j);
* A[i, j] = -(1/2 pi) sum_{n in N^(i)} J_n w^(i)_n
             sum_{n' in N^(j)} ( K1(eta_n, eta_n') J_n' w^(j)_n' + W^s[n][n'] J_n' B_j(eta_n') )
  (eqs. IK1e2 and IK1e2_bis).

Pinned against the dense oracle entry by entry at small sizes
(`tests/test_oracle_sampled.py`).
"""
from __future__ import annotations

from math import factorial

import numpy as np
import scipy.linalg as sla

from . import bspline
from .assembly import geometry_at, kernel_K1, make_discretization
from .discretization import Discretization
from .rules import k2_images, local_log_moments


def local_basis(knots, d: int, x, nder: int = 0):
    """(first, vals): the d + 1 B-splines non-zero at each x are
    B_{first + r}, r = 0..d, with values / derivatives vals[q, p, r].
    The recurrence and the derivative formula of `bspline.basis_all`, run on
    each point's window of 2d + 2 knots (all points at once)."""
    t = np.asarray(knots, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n_basis = len(t) - d - 1
    span = bspline._span(t, d, n_basis, x)
    T = t[span[:, None] + np.arange(-d, d + 2)[None, :]]            # (P, 2d + 2), interval d is x's
    P = len(x)

    def ratio(num, den):
        ok = den > 0
        return np.where(ok, num / np.where(ok, den, 1.0), 0.0)

    levels = [np.zeros((2 * d + 1, P))]
    levels[0][d] = 1.0
    for r in range(1, d + 1):
        prev = levels[-1]
        nb = 2 * d + 1 - r
        Bn = np.zeros((nb, P))
        for i in range(nb):
            Bn[i] = ratio(x - T[:, i], T[:, i + r] - T[:, i]) * prev[i] + \
                ratio(T[:, i + r + 1] - x, T[:, i + r + 1] - T[:, i + 1]) * prev[i + 1]
        levels.append(Bn)
    vals = np.zeros((nder + 1, P, d + 1))
    vals[0] = levels[d].T
    for q in range(1, min(nder, d) + 1):
        cur = levels[d - q].copy()
        for r in range(d - q + 1, d + 1):
            nb = 2 * d + 1 - r
            nxt = np.zeros((nb, P))
            for i in range(nb):
                nxt[i] = r * (ratio(cur[i], T[:, i + r] - T[:, i]) - ratio(cur[i + 1], T[:, i + r + 1] - T[:, i + 1]))
            cur = nxt
        vals[q] = cur.T
    return span - d, vals


def test_values(disc: Discretization, i: int, s) -> np.ndarray:
    """B_i(s) (closed curves: the cyclic function B_i + B_{i+N_h} for i < d)."""
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    first, v = local_basis(disc.test_knots, disc.d, s)
    out = np.zeros(len(s))
    for r in range(disc.d + 1):
        j = first + r
        hit = (j == i) | (j == i + disc.Nh) if disc.closed else (j == i)
        out += np.where(hit, v[0, :, r], 0.0)
    return out


def fine_values(disc: Discretization, s, idx) -> np.ndarray:
    """B-bar_j(s_p) for j in idx: (len(idx), len(s))."""
    first, v = local_basis(disc.fine_knots, disc.d, s)
    pos = {int(j): a for a, j in enumerate(idx)}
    out = np.zeros((len(idx), len(first)))
    for p in range(len(first)):
        for r in range(disc.d + 1):
            a = pos.get(int(first[p] + r))
            if a is not None:
                out[a, p] = v[0, p, r]
    return out


def regular_rule(disc: Discretization, i: int):
    """(N^(i), w^(i)) of Algorithm 1."""
    Ji = disc.overlapping_fine(i)
    Ni = disc.support_nodes(i)
    x, w = np.polynomial.legendre.leggauss(disc.d + 1)
    elems = []
    for lo, hi in disc._test_support(i):
        elems.extend(range(int(round(lo)), int(round(hi))))
    e = np.array(elems)[:, None]
    tq = (disc.a + disc.hf * (e + (x[None, :] + 1.0) / 2.0)).ravel()
    wq = np.tile(w * disc.hf / 2.0, len(elems))
    mu = fine_values(disc, tq, Ji) @ (wq * test_values(disc, i, tq))
    Bi = fine_values(disc, disc.eta[Ni], Ji)
    wi, *_ = np.linalg.lstsq(Bi, mu, rcond=None)
    return Ni, wi


def gram_band(disc: Discretization) -> np.ndarray:
    """Upper banded Cholesky factor of G = (B)(B)^T (half-bandwidth d)."""
    d = disc.d
    first, v = local_basis(disc.fine_knots, d, disc.eta)
    ab = np.zeros((d + 1, disc.NE))
    for a in range(d + 1):
        for b in range(a, d + 1):
            np.add.at(ab[d - (b - a)], first + b, v[0, :, a] * v[0, :, b])
    return sla.cholesky_banded(ab)


def element_pieces(disc: Discretization) -> np.ndarray:
    """C[e, r, k]: B-bar_{e+r}(tau_e + u h_f) = sum_k C[e,r,k] u^k (right-sided
    Taylor coefficients at the element's left end)."""
    d, M = disc.d, disc.M
    left = disc.a + disc.hf * np.arange(M)
    first, v = local_basis(disc.fine_knots, d, left, nder=d)
    assert np.array_equal(first, np.arange(M))
    C = np.zeros((M, d + 1, d + 1))
    for k in range(d + 1):
        C[:, :, k] = v[k] * disc.hf ** k / factorial(k)
    return C


def moments_at(disc: Discretization, s, C: np.ndarray) -> np.ndarray:
    """mu_j(s) = int_I B-bar_j(t) K2(s, t) dt, (len(s), N_E) (eq. mod_mom_gen)."""
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    d, M, hf = disc.d, disc.M, disc.hf
    tau = disc.a + hf * np.arange(M)
    out = np.zeros((len(s), disc.NE))
    for p, sp in enumerate(s):
        E = np.zeros((d + 1, M))                         # E[k, e] = int_e u^k K2(s, t) dt
        for sh in k2_images(disc):
            L = local_log_moments((sp + sh - tau) / hf, d)
            for k in range(d + 1):
                E[k] += hf * (np.log(hf) / (k + 1) + L[k])
        if disc.closed:
            for k in range(d + 1):
                E[k] -= 2.0 * np.log(disc.L) * hf / (k + 1)
        for r in range(d + 1):
            np.add.at(out[p], np.arange(M) + r, np.einsum("ek,ke->e", C[:, r, :], E))
    return out


class EntrySampler:
    """A[i, j] one by one for a curve and discretisation of any size."""

    def __init__(self, curve, n_elems: int, degree: int, n_ref: int):
        self.curve = curve
        self.disc = make_discretization(curve, n_elems, degree, n_ref)
        self.cb = gram_band(self.disc)
        self.C = element_pieces(self.disc)
        self._rules = {}

    def rule(self, i: int):
        if i not in self._rules:
            self._rules[i] = regular_rule(self.disc, i)
        return self._rules[i]

    def singular(self, rows, cols) -> np.ndarray:
        """W^s[rows][:, cols] (Algorithm 2)."""
        disc = self.disc
        Mu = moments_at(disc, disc.eta[rows], self.C)
        Z = sla.cho_solve_banded((self.cb, False), Mu.T)           # (N_E, len(rows))
        first, v = local_basis(disc.fine_knots, disc.d, disc.eta[cols])
        out = np.zeros((len(rows), len(cols)))
        for r in range(disc.d + 1):
            out += v[0, :, r][None, :] * Z[first + r, :].T
        return out

    def entry(self, i: int, j: int) -> float:
        disc = self.disc
        Ni, wi = self.rule(i)
        Nj, wj = self.rule(j)
        fi, _, Ji = geometry_at(self.curve, disc.eta[Ni])
        fj, _, Jj = geometry_at(self.curve, disc.eta[Nj])
        C0 = kernel_K1(disc, fi, Ji, disc.eta[Ni], fj, disc.eta[Nj])
        Ws = self.singular(Ni, Nj)
        inner = C0 @ (Jj * wj) + Ws @ (Jj * test_values(disc, j, disc.eta[Nj]))
        return float(-((Ji * wi) @ inner) / (2.0 * np.pi))


# ----------------------------------------------------------------------------
# Whole rows of A at large size
# ----------------------------------------------------------------------------
def regular_rules_sparse(disc: Discretization, cols=None):
    """The regular rules w^(i) of Algorithm 1 for test functions `cols`
    (default all), as (i, N^(i), w^(i)) triples: `regular_rule` per function."""
    cols = range(disc.n) if cols is None else cols
    return [(int(i),) + regular_rule(disc, int(i)) for i in cols]


class RowSampler:
    """Rows A[i, :] one by one at any size, from the same definitions as the
    dense oracle restricted to what a row touches (eqs. IK1e2, IK1e2_bis):

        A[i, :] = -(1/2 pi) sum_{n in N^(i)} J_n w^(i)_n
                  ( sum_{n'} K1(eta_n, eta_n') P[n', :] + sum_{n'} W^s[n][n'] Q[n', :] )

    with P[n', j] = J_n' w^(j)_n' (all n regular rules, kept sparse),
    Q[n', j] = J_n' B_j(eta_n') (d + 1 non-zeros per node, cyclic wrap for
    closed curves) and the singular rules W^s[n][:] of Algorithm 2 for the
    nodes n in N^(i).  `rules` may hand in the (i, N^(i), w^(i)) triples of
    `regular_rules_sparse` (computed elsewhere, e.g. in parallel)."""

    def __init__(self, curve, n_elems: int, degree: int, n_ref: int, rules=None):
        import scipy.sparse as sp
        self.curve = curve
        disc = self.disc = make_discretization(curve, n_elems, degree, n_ref)
        self.entry_sampler = EntrySampler(curve, n_elems, degree, n_ref)
        f, _, J = geometry_at(curve, disc.eta)
        self.f, self.J = f, J
        if rules is None:
            rules = regular_rules_sparse(disc)
        rows, cols, vals = [], [], []
        self.rule = {}
        for i, Ni, wi in rules:
            self.rule[i] = (Ni, wi)
            rows.append(Ni)
            cols.append(np.full(len(Ni), i))
            vals.append(J[Ni] * wi)
        self.P = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(disc.Nq, disc.n))
        first, v = local_basis(disc.test_knots, disc.d, disc.eta)
        qr, qc, qv = [], [], []
        for r in range(disc.d + 1):
            j = first + r
            if disc.closed:
                j = np.where(j >= disc.Nh, j - disc.Nh, j)
            keep = v[0, :, r] != 0.0
            qr.append(np.nonzero(keep)[0])
            qc.append(j[keep])
            qv.append(J[keep] * v[0, keep, r])
        self.Q = sp.csr_matrix((np.concatenate(qv), (np.concatenate(qr), np.concatenate(qc))),
                               shape=(disc.Nq, disc.n))

    def row(self, i: int) -> np.ndarray:
        disc = self.disc
        Ni, wi = self.rule[i]
        C0 = kernel_K1(disc, self.f[:, Ni], self.J[Ni], disc.eta[Ni], self.f, disc.eta)   # (|N^(i)|, Nq)
        Ws = self.entry_sampler.singular(Ni, np.arange(disc.Nq))                          # (|N^(i)|, Nq)
        inner = (self.P.T @ C0.T).T + (self.Q.T @ Ws.T).T                                  # (|N^(i)|, n)
        return -((self.J[Ni] * wi) @ inner) / (2.0 * np.pi)
