"""Weighted quadrature rules (oracle; test infrastructure only).

* Algorithm 1 (Sect. 4.1, eqs. reg_quad / reg_exactness): for every test
  function B_i, weights w^(i) on the nodes N^(i) such that
      sum_{n in N^(i)} w^(i)_n B-bar_j(eta_n) = mu^(i)_j = int_I B-bar_j B_i,
  for all j in J^(i), taken as the minimum Euclidean norm solution.
* Modified moments (eq. mod_mom_gen): mu_j(s) = int_I B-bar_j(t) K2(s, t) dt.
  The paper computes them with the B-spline recurrence (eq. recIq) started
  from the closed-form base integrals  int z^j ln|z| dz = z^{j+1}/(j+1) (ln|z| - 1/(j+1)).
  The oracle evaluates the same integral, element by element, from its
  definition: on each refined element the B-spline is a polynomial in the
  local coordinate u = (t - tau_e)/h_e, and
      int_e u^k ln|t - s| dt = h_e [ln(h_e)/(k+1) + int_0^1 u^k ln|u - c| du],
  c = (s - tau_e)/h_e.  The last integral is the paper's closed-form base
  integral in local coordinates when |c - 1/2| <= 5/2 (the near field), and a
  16-point Gauss-Legendre rule otherwise (the integrand is then analytic on
  an ellipse with parameter > 7.8 around [0, 1], so the rule is exact to
  below 1e-28 relative).  The recurrence itself is kept as a test: in
  absolute powers of t it cancels catastrophically as h -> 0.
* Kernel K2 (Sect. 3.1): ln|t - s| for an open arc.  For a closed curve
  f(a) = f(b), so ln||f(s)-f(t)|| is also singular at the corners (s,t) =
  (a,b), (b,a) of I x I; the singular part is then taken as the periodic
  three-image log
      K2(s,t) = ln|t-s| + ln|t-s+L| + ln|t-s-L| - 2 ln L,   L = b - a,
  which keeps K1 = ln||f(s)-f(t)|| - K2 smooth on I x I and keeps every
  moment a sum of the paper's closed forms (shifted abscissae).
* Algorithm 2 (Sect. 4.2, eqs. sing_quad / sing_exactness): for every node
  eta_m, weights w^{eta_m} in R^{N_quad} with (B) w = mu(eta_m), minimum norm.
  The paper factorises (B) once (LU); the minimum-norm solution is unique,
  so the oracle uses w = (B)^T G^{-1} mu with G = (B)(B)^T factorised once
  by banded Cholesky (G has half-bandwidth d).
"""
from __future__ import annotations

from math import comb, factorial

import numpy as np
import scipy.linalg as sla

from .discretization import Discretization

_GAUSS_FAR = np.polynomial.legendre.leggauss(16)


# --------------------------------------------------------------------------
# Algorithm 1: regular weighted rules
# --------------------------------------------------------------------------
def regular_rules(disc: Discretization) -> np.ndarray:
    """W, shape (N_quad, n): column i holds w^(i) (zero outside N^(i))."""
    Bc = disc.collocation()                              # (N_E, N_quad)
    tq, wq = disc.fine_gauss(disc.d + 1)                 # exact for degree 2d
    Bf = disc.fine_basis(tq)[0]                          # (N_E, nq)
    Bt = disc.test_basis(tq)[0]                          # (n, nq)
    W = np.zeros((disc.Nq, disc.n))
    for i in range(disc.n):
        Ji = disc.overlapping_fine(i)
        Ni = disc.support_nodes(i)
        mu = Bf[Ji] @ (wq * Bt[i])                       # mu^(i)_j = int B-bar_j B_i
        Bi = Bc[np.ix_(Ji, Ni)]
        w, *_ = np.linalg.lstsq(Bi, mu, rcond=None)      # minimum-norm solution
        W[Ni, i] = w
    return W


# --------------------------------------------------------------------------
# Modified moments
# --------------------------------------------------------------------------
def _base_integral(z, j):
    """int_0^z x^j ln|x| dx = z^{j+1}/(j+1) (ln|z| - 1/(j+1)), 0 at z = 0."""
    z = np.asarray(z, dtype=np.float64)
    az = np.abs(z)
    safe = np.where(az > 0, az, 1.0)
    v = z ** (j + 1) / (j + 1) * (np.log(safe) - 1.0 / (j + 1))
    return np.where(az > 0, v, 0.0)


def local_log_moments(c, kmax: int) -> np.ndarray:
    """L_k(c) = int_0^1 u^k ln|u - c| du for k = 0..kmax; c array.

    Near field (|c - 1/2| <= 5/2): substitute z = u - c and expand u^k
    binomially, giving the closed-form base integrals between -c and 1-c.
    Far field: Gauss-Legendre, 16 points.  Returns (kmax+1, len(c))."""
    c = np.atleast_1d(np.asarray(c, dtype=np.float64))
    out = np.zeros((kmax + 1, len(c)))
    near = np.abs(c - 0.5) <= 2.5
    if near.any():
        cn = c[near]
        for k in range(kmax + 1):
            acc = np.zeros(len(cn))
            for j in range(k + 1):
                acc += comb(k, j) * cn ** (k - j) * (_base_integral(1.0 - cn, j) - _base_integral(-cn, j))
            out[k, near] = acc
    far = ~near
    if far.any():
        x, w = _GAUSS_FAR
        u = (x + 1.0) / 2.0
        cf = c[far]
        lg = np.log(np.abs(u[:, None] - cf[None, :]))           # (16, nf)
        for k in range(kmax + 1):
            out[k, far] = (w / 2.0 * u ** k) @ lg
    return out


def k2_images(disc: Discretization) -> list[float]:
    """Abscissa shifts of the log terms in K2: [0] (open) or [0, -L, +L] (closed)."""
    return [0.0, -disc.L, disc.L] if disc.closed else [0.0]


def piece_coefficients(disc: Discretization) -> np.ndarray:
    """C[j, e, k]: B-bar_j(tau_e + u h_f) = sum_k C[j,e,k] u^k on element e.

    Taylor coefficients at the element's left end, from the right-sided
    derivatives: C[j,e,k] = h_f^k / k! * B-bar_j^(k)(tau_e^+)."""
    d, M = disc.d, disc.M
    left = disc.a + disc.hf * np.arange(M)
    D = disc.fine_basis(left, nder=d)          # right-sided: span of t = tau_e is element e
    C = np.zeros((disc.NE, M, d + 1))
    for k in range(d + 1):
        C[:, :, k] = D[k] * disc.hf ** k / factorial(k)
    return C


def moments(disc: Discretization, s, C: np.ndarray | None = None) -> np.ndarray:
    """mu_j(s) = int_I B-bar_j(t) K2(s,t) dt for all j (eq. mod_mom_gen,
    with the closed-curve K2 above).  s: array of abscissae in I.
    Returns (len(s), N_E)."""
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    d, M, hf = disc.d, disc.M, disc.hf
    if C is None:
        C = piece_coefficients(disc)
    images = k2_images(disc)
    out = np.zeros((len(s), disc.NE))
    tau = disc.a + hf * np.arange(M)
    for e in range(M):
        # E[k, p] = int_e u^k K2(s_p, t) dt
        E = np.zeros((d + 1, len(s)))
        for sh in images:
            c = (s + sh - tau[e]) / hf
            L = local_log_moments(c, d)
            for k in range(d + 1):
                E[k] += hf * (np.log(hf) / (k + 1) + L[k])
        if disc.closed:
            for k in range(d + 1):
                E[k] -= 2.0 * np.log(disc.L) * hf / (k + 1)
        js = np.nonzero(np.abs(C[:, e, :]).sum(axis=1) > 0)[0]
        out[:, js] += E.T @ C[js, e, :].T
    return out


# --------------------------------------------------------------------------
# Algorithm 2: singular weighted rules
# --------------------------------------------------------------------------
def gram_factor(disc: Discretization):
    """Banded Cholesky factor of G = (B)(B)^T (upper form, half-bandwidth d)."""
    Bc = disc.collocation()
    G = Bc @ Bc.T
    d = disc.d
    ab = np.zeros((d + 1, disc.NE))
    for r in range(d + 1):
        ab[d - r, r:] = np.diagonal(G, r)
    return sla.cholesky_banded(ab), Bc


def singular_rules(disc: Discretization, rows=None) -> np.ndarray:
    """W^s, shape (len(rows), N_quad): row m holds w^{eta_m} (Algorithm 2).
    rows: node indices (default all)."""
    cb, Bc = gram_factor(disc)
    if rows is None:
        rows = np.arange(disc.Nq)
    rows = np.asarray(rows)
    Mu = moments(disc, disc.eta[rows])                  # (len(rows), N_E)
    Z = sla.cho_solve_banded((cb, False), Mu.T)         # G^{-1} mu, (N_E, len(rows))
    return (Bc.T @ Z).T
