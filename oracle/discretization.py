"""Discretisation spaces, node vector and index sets (oracle; test infrastructure only).

Follows Sect. 3 (test/trial space) and Sect. 4 (exactness space, nodes) of the paper.

* Test/trial space S: degree-d B-splines on N_h uniform elements of I = [a, b].
  Open arc: clamped ("multiple auxiliary") knots, dimension N_h + d.
  Closed curve: periodic extended knots, the first d functions wrapped onto
  the last d (the cyclic basis B^(c) of Sect. 3), dimension N_h.
* Exactness space S-bar: degree-d splines on the uniform refinement with
  M = N_ref N_h elements, N_E = M + d functions B-bar_j, restricted to I
  (Sect. 4: "obtained by uniform subdivision of each element into N_ref").
  The same (non-wrapped) space is used for closed curves: only the
  trial/test functions wrap.
* Node vector eta (Sect. 4): d+2 uniformly spaced points in the first and
  in the last element of the refined partition, midpoints and breakpoints
  in every inner element; N_quad = 2d + 2 M - 1.
* Index sets of Sect. 4.1 with the paper's footnote that a support is the
  (relatively open) set where the function is non-zero:
    J^(i) = {j : supp(B-bar_j) meets supp(B_i)},  N^(i) = {n : B_i(eta_n) != 0}.
  For the clamped end functions of an open arc the end point belongs to the
  support (B_1(a) = 1), so the end node is in N^(1).
"""
from __future__ import annotations

import numpy as np

from . import bspline


class Discretization:
    def __init__(self, a: float, b: float, n_elems: int, d: int, n_ref: int, closed: bool):
        if closed and n_elems < d + 1:
            raise ValueError("closed curves need at least d+1 elements")
        self.a, self.b = float(a), float(b)
        self.Nh, self.d, self.Nref, self.closed = int(n_elems), int(d), int(n_ref), bool(closed)
        self.L = self.b - self.a
        self.h = self.L / self.Nh
        self.M = self.Nh * self.Nref
        self.hf = self.L / self.M
        self.n = self.Nh if closed else self.Nh + d           # N_DoF
        self.NE = self.M + d                                   # N_E
        d_, M = self.d, self.M
        if closed:
            # periodic extended knots of S: t_k = a + (k - d) h, k = 0..N_h + 2d
            self.test_knots = self.a + self.h * (np.arange(self.Nh + 2 * d_ + 1) - d_)
        else:
            self.test_knots = np.concatenate([[self.a] * d_, self.a + self.h * np.arange(self.Nh + 1),
                                              [self.b] * d_])
            self.test_knots[d_ + self.Nh] = self.b
        # exactness space: uniform extended knots (closed) or clamped (open);
        # both span the same space of degree-d splines on the refined partition.
        if closed:
            self.fine_knots = self.a + self.hf * (np.arange(M + 2 * d_ + 1) - d_)
        else:
            self.fine_knots = np.concatenate([[self.a] * d_, self.a + self.hf * np.arange(M + 1),
                                              [self.b] * d_])
            self.fine_knots[d_ + M] = self.b
        # node vector eta, with positions also kept in units of hf from a
        first = np.linspace(0.0, 1.0, d_ + 2)
        last = (M - 1) + np.linspace(0.0, 1.0, d_ + 2)
        inner = []
        for e in range(1, M - 1):
            if e >= 2:
                inner.append(float(e))          # breakpoint between elements e-1 and e
            inner.append(e + 0.5)               # midpoint of element e
        if M == 1:
            pos = first
        else:
            pos = np.concatenate([first, np.array(inner), last])
        self.node_pos = pos                                    # in units of hf
        self.eta = self.a + self.hf * pos
        self.eta[-1] = self.b
        self.Nq = len(self.eta)
        assert self.Nq == 2 * d_ + 2 * M - 1

    # ------------------------------------------------------------------ bases
    def test_basis(self, s, nder: int = 0) -> np.ndarray:
        """Test/trial functions B_i at s: array (nder+1, n, len(s)).
        Closed: B_i + B_{i+N_h} for i < d (cyclic basis of Sect. 3)."""
        B = bspline.basis_all(self.test_knots, self.d, s, nder)
        if not self.closed:
            return B
        out = B[:, :self.Nh].copy()
        out[:, :self.d] += B[:, self.Nh:self.Nh + self.d]
        return out

    def fine_basis(self, s, nder: int = 0) -> np.ndarray:
        """Exactness-space B-splines B-bar_j at s: (nder+1, N_E, len(s))."""
        return bspline.basis_all(self.fine_knots, self.d, s, nder)

    def collocation(self) -> np.ndarray:
        """(B)_{j,n} = B-bar_j(eta_n), shape (N_E, N_quad) (Algorithms 1 and 2)."""
        return self.fine_basis(self.eta)[0]

    # -------------------------------------------------------------- supports
    def _test_support(self, i: int) -> list[tuple[float, float]]:
        """Support of B_i as intervals in units of hf from a (within [0, M])."""
        lo = (i - self.d) * self.Nref if self.closed else None
        if self.closed:
            hi = lo + (self.d + 1) * self.Nref
            out = []
            for shift in (-self.M, 0, self.M):
                l, h = max(lo + shift, 0), min(hi + shift, self.M)
                if h > l:
                    out.append((float(l), float(h)))
            return out
        # clamped: support [t_i, t_{i+d+1}] mapped to hf units
        l = (self.test_knots[i] - self.a) / self.hf
        h = (self.test_knots[i + self.d + 1] - self.a) / self.hf
        return [(float(np.round(l)), float(np.round(h)))]

    def support_nodes(self, i: int) -> np.ndarray:
        """N^(i): indices of nodes where B_i is non-zero."""
        p = self.node_pos
        mask = np.zeros(self.Nq, dtype=bool)
        for l, h in self._test_support(i):
            mask |= (p > l + 1e-9) & (p < h - 1e-9)
        if self.closed:
            # the seam point a == b: B_i is non-zero there iff the periodic
            # support contains it in its interior
            sup = self._test_support(i)
            touches_a = any(l <= 1e-9 for l, h in sup)
            touches_b = any(h >= self.M - 1e-9 for l, h in sup)
            if touches_a and touches_b:
                mask[0] = mask[-1] = True
        else:
            if i == 0:
                mask[0] = True                 # B_1(a) = 1 for clamped knots
            if i == self.n - 1:
                mask[-1] = True
        return np.nonzero(mask)[0]

    def overlapping_fine(self, i: int) -> np.ndarray:
        """J^(i): exactness functions whose support meets that of B_i."""
        j = np.arange(self.NE)
        fl = np.maximum((self.fine_knots[j] - self.a) / self.hf, 0.0)
        fh = np.minimum((self.fine_knots[j + self.d + 1] - self.a) / self.hf, float(self.M))
        hit = np.zeros(self.NE, dtype=bool)
        for l, h in self._test_support(i):
            hit |= (np.minimum(fh, h) - np.maximum(fl, l)) > 1e-9
        return np.nonzero(hit)[0]

    # -------------------------------------------------------------- quadrature
    def fine_gauss(self, g: int) -> tuple[np.ndarray, np.ndarray]:
        """Composite Gauss-Legendre rule with g points on each refined element."""
        x, w = np.polynomial.legendre.leggauss(g)
        e = np.arange(self.M)[:, None]
        t = self.a + self.hf * (e + (x[None, :] + 1.0) / 2.0)
        return t.ravel(), np.tile(w * self.hf / 2.0, self.M)
