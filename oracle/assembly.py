"""Matrix, right-hand side, solve and errors (oracle; test infrastructure only).

* Matrix entries (Sect. 3.1, eq. final_1, split eq. IK12): the Galerkin
  matrix of the single-layer operator is  A = -(I_K1 + I_K2) / (2 pi)
  (the coefficient -1/(2 pi) of eq. bilf), with
      K1(s,t) = ln||f(s) - f(t)|| - K2(s,t)
  extended by continuity: K1(s,s) = ln J(s) (eq. F1_lim), and at the closed
  curve's corners (s,t) = (a,b), (b,a): K1 = ln J - ln 2.
* I_K1 by eq. IK1e2: the regular rules in both variables,
      I_K1 = P^T C0 P,  P = diag(J(eta)) W,  C0[n1,n2] = K1(eta_n1, eta_n2).
* I_K2 by eq. IK1e2_bis: regular outer rule, singular inner rule, used for
  every (i, j) (Sect. 5 says the singular rule was used for far pairs too):
      I_K2 = P^T W^s Q,  Q[n, j] = J(eta_n) B_j(eta_n).
* Right-hand side (Sect. 5): b1_i = sum_n P[n,i] u_D(eta_n);
  b2_i = sum_n P[n,i] sum_g w_g Kbar(eta_n, t_g) u_D(t_g) with a composite
  Gauss rule (t_g, w_g), G_RHS points per refined element, and
  Kbar(s,t) = d/dn_y ln|x-y| J(t) = (f(t)-f(s)) . (f2'(t), -f1'(t)) / |f(t)-f(s)|^2
  (outward normal of a counter-clockwise curve).  Interior problem (eq.
  seconda_BIE): beta = b1/2 - b2/(2 pi).  Open arc (eq. prima_BIE): beta = b1.
* Solve: A is symmetric positive definite in the continuous setting (eq.
  sistlin); the discrete A is symmetric only up to quadrature error, so the
  oracle solves with (A + A^T)/2 by Cholesky (LAPACK potrf/potrs).
* Errors (Sect. 6): E_M = max error on 500 uniform points of I, E_R = relative
  L^2(I) error.
* Representation formula (Sect. 2): with the density q_h = sum_j alpha_j B_j,
      u(x) = -(1/2 pi) int ln|x - y| q_h dgamma + (1/2 pi) int dln|x - y|/dn_y u_D dgamma
  for x inside a closed curve (direct method), and only the first term for an
  open arc (indirect method, density phi_h), both by the composite Gauss rule
  of the right-hand side (G_RHS points per refined element).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import bspline, rules
from .discretization import Discretization

G_RHS = 8                      # Gauss points per refined element for the b2 inner integral


def make_discretization(curve, n_elems: int, degree: int, n_ref: int) -> Discretization:
    a, b = curve.interval
    return Discretization(a, b, n_elems, degree, n_ref, curve.closed)


def geometry_at(curve, s):
    """f, f', J at parameter values s (Sect. 3, eq. J)."""
    f, f1 = bspline.curve_eval(curve, s, nder=1)
    J = np.hypot(f1[0], f1[1])
    return f, f1, J


def kernel_K1(disc: Discretization, f_s, J_s, s, f_t, t, corner_mask=None):
    """K1(s_p, t_q) for all pairs: (len(s), len(t)).  Entries with s = t take
    ln J(s) (eq. F1_lim); closed-curve corners take ln J(s) - ln 2."""
    dx = f_t[0][None, :] - f_s[0][:, None]
    dy = f_t[1][None, :] - f_s[1][:, None]
    x = t[None, :] - s[:, None]
    if disc.closed:
        L = disc.L
        D = np.abs(x) * np.abs(x + L) * np.abs(x - L) / (L * L)
    else:
        D = np.abs(x)
    num = dx * dx + dy * dy
    with np.errstate(divide="ignore", invalid="ignore"):
        K1 = 0.5 * np.log(num / (D * D))
    diag = x == 0.0
    K1 = np.where(diag, np.log(J_s)[:, None], K1)
    if disc.closed:
        corner = np.abs(np.abs(x) - disc.L) == 0.0
        K1 = np.where(corner, (np.log(J_s) - np.log(2.0))[:, None], K1)
    return K1


def assemble(curve, n_elems: int, degree: int, n_ref: int = 2, keep: bool = False) -> dict:
    """Full assembly of A (small and moderate sizes).  Returns a dict with
    A, AK1, AK2 (= I_K1, I_K2) and, if keep, the intermediate arrays."""
    disc = make_discretization(curve, n_elems, degree, n_ref)
    W = rules.regular_rules(disc)                        # (Nq, n)
    Ws = rules.singular_rules(disc)                      # (Nq, Nq)
    f, f1, J = geometry_at(curve, disc.eta)
    P = J[:, None] * W
    Q = J[:, None] * disc.test_basis(disc.eta)[0].T
    C0 = kernel_K1(disc, f, J, disc.eta, f, disc.eta)
    AK1 = P.T @ (C0 @ P)
    AK2 = P.T @ (Ws @ Q)
    A = -(AK1 + AK2) / (2.0 * np.pi)
    out = dict(A=A, AK1=AK1, AK2=AK2, disc=disc)
    if keep:
        out.update(W=W, Ws=Ws, P=P, Q=Q, C0=C0, f=f, f1=f1, J=J)
    return out


def assemble_rows(curve, n_elems: int, degree: int, n_ref: int, rows) -> dict:
    """Rows `rows` of I_K1, I_K2 and A, computed from only the singular-rule
    rows and kernel rows they need (sampled parity checks at large size;
    the test basis is evaluated densely, so n up to a few thousand)."""
    disc = make_discretization(curve, n_elems, degree, n_ref)
    rows = np.asarray(rows)
    W = rules.regular_rules(disc)
    f, f1, J = geometry_at(curve, disc.eta)
    P = J[:, None] * W
    Q = J[:, None] * disc.test_basis(disc.eta)[0].T
    need = np.unique(np.concatenate([disc.support_nodes(i) for i in rows]))
    Ws = rules.singular_rules(disc, need)                # (len(need), Nq)
    C0 = kernel_K1(disc, f[:, need], J[need], disc.eta[need], f, disc.eta)
    Pn = P[need][:, rows]                                # (len(need), len(rows))
    AK1 = Pn.T @ (C0 @ P)
    AK2 = Pn.T @ (Ws @ Q)
    return dict(AK1=AK1, AK2=AK2, A=-(AK1 + AK2) / (2.0 * np.pi), disc=disc)


# ----------------------------------------------------------------------------
# Right-hand side
# ----------------------------------------------------------------------------
def rhs_points(curve, n_elems: int, degree: int, n_ref: int = 2):
    """Parameter values where u_D is sampled: the nodes eta, then the
    composite Gauss points t_g of the b2 inner rule (with weights)."""
    disc = make_discretization(curve, n_elems, degree, n_ref)
    tg, wg = disc.fine_gauss(G_RHS)
    return disc.eta, tg, wg


def kernel_Kbar(f_s, f_t, f1_t):
    """Kbar(s_p, t_q) = (f(t)-f(s)).(f2'(t), -f1'(t)) / |f(t)-f(s)|^2."""
    dx = f_t[0][None, :] - f_s[0][:, None]
    dy = f_t[1][None, :] - f_s[1][:, None]
    return (dx * f1_t[1][None, :] - dy * f1_t[0][None, :]) / (dx * dx + dy * dy)


def build_rhs(curve, n_elems: int, degree: int, n_ref: int, uD_nodes, uD_gauss, magnitude: bool = False):
    """beta (n x nrhs).  uD_nodes: (Nq, nrhs) values of u_D at eta;
    uD_gauss: (Ng, nrhs) values at the Gauss points (closed curves only).
    With magnitude=True returns (beta, S, K): S holds the same sums taken over
    the absolute values of their terms, the scale of the rounding error of
    any evaluation of them (|fl(sum x) - sum x| <= N eps sum |x|); K bounds
    the first-order change of beta when every coordinate of f at the nodes and
    f, f' at the Gauss points changes by one unit in the last place (relative
    2^-53): since |d Kbar / d(f(t) - f(s))| <= 3 |f'(t)| / r^2 with
    r = |f(t) - f(s)|,
        K_i = (1/2pi) sum_n |P[n,i]| sum_g w_g |u_D(t_g)| 3 |f'(t_g)| (|f(s_n)| + |f(t_g)|) / r^2
    times 2^-53 (zero for an open arc)."""
    disc = make_discretization(curve, n_elems, degree, n_ref)
    W = rules.regular_rules(disc)
    f, f1, J = geometry_at(curve, disc.eta)
    P = J[:, None] * W
    uD_nodes = np.asarray(uD_nodes, np.float64).reshape(disc.Nq, -1)
    b1 = P.T @ uD_nodes
    if not disc.closed:
        return (b1, np.abs(P).T @ np.abs(uD_nodes), np.zeros_like(b1)) if magnitude else b1
    tg, wg = disc.fine_gauss(G_RHS)
    ft, f1t, _ = geometry_at(curve, tg)
    Kb = kernel_Kbar(f, ft, f1t)                         # (Nq, Ng)
    uD_gauss = np.asarray(uD_gauss, np.float64).reshape(len(tg), -1)
    b2 = P.T @ (Kb @ (wg[:, None] * uD_gauss))
    beta = 0.5 * b1 - b2 / (2.0 * np.pi)
    if not magnitude:
        return beta
    return (beta,) + _rhs_scales(P, uD_nodes, f, ft, f1t, Kb, wg, uD_gauss)


def build_rhs_rows(curve, n_elems: int, degree: int, n_ref: int, rows, uD_nodes, uD_gauss, magnitude: bool = False):
    """Entries `rows` of beta (len(rows) x nrhs) by the same sums as build_rhs,
    restricted to the nodes N^(i) where P[n, i] can be non-zero (sampled
    parity checks at large size).  magnitude=True as in build_rhs."""
    disc = make_discretization(curve, n_elems, degree, n_ref)
    W = rules.regular_rules(disc)
    rows = np.asarray(rows)
    need = np.unique(np.concatenate([disc.support_nodes(i) for i in rows]))
    f, f1, J = geometry_at(curve, disc.eta[need])
    P = J[:, None] * W[need][:, rows]                    # (len(need), len(rows))
    uD_nodes = np.asarray(uD_nodes, np.float64).reshape(disc.Nq, -1)
    b1 = P.T @ uD_nodes[need]
    if not disc.closed:
        return (b1, np.abs(P).T @ np.abs(uD_nodes[need]), np.zeros_like(b1)) if magnitude else b1
    tg, wg = disc.fine_gauss(G_RHS)
    ft, f1t, _ = geometry_at(curve, tg)
    Kb = kernel_Kbar(f, ft, f1t)                         # (len(need), Ng)
    uD_gauss = np.asarray(uD_gauss, np.float64).reshape(len(tg), -1)
    b2 = P.T @ (Kb @ (wg[:, None] * uD_gauss))
    beta = 0.5 * b1 - b2 / (2.0 * np.pi)
    if not magnitude:
        return beta
    return (beta,) + _rhs_scales(P, uD_nodes[need], f, ft, f1t, Kb, wg, uD_gauss)


def _rhs_scales(P, uN, f, ft, f1t, Kb, wg, ug):
    """(S, K) of build_rhs(magnitude=True) for a closed curve."""
    aP = np.abs(P).T
    wu = wg[:, None] * np.abs(ug)
    S = 0.5 * (aP @ np.abs(uN)) + (aP @ (np.abs(Kb) @ wu)) / (2.0 * np.pi)
    dx = ft[0][None, :] - f[0][:, None]
    dy = ft[1][None, :] - f[1][:, None]
    sens = 3.0 * np.hypot(f1t[0], f1t[1])[None, :] * \
        (np.hypot(f[0], f[1])[:, None] + np.hypot(ft[0], ft[1])[None, :]) / (dx * dx + dy * dy)
    K = 2.0 ** -53 * (aP @ (sens @ wu)) / (2.0 * np.pi)
    return S, K


# ----------------------------------------------------------------------------
# Solve and errors
# ----------------------------------------------------------------------------
def solve(A: np.ndarray, beta: np.ndarray) -> np.ndarray:
    """alpha from (A + A^T)/2 alpha = beta by Cholesky."""
    As = 0.5 * (A + A.T)
    c = sla.cho_factor(As, lower=True)
    return sla.cho_solve(c, beta)


# ----------------------------------------------------------------------------
# Representation formula (post-processing)
# ----------------------------------------------------------------------------
def density_at(disc: Discretization, alpha, s) -> np.ndarray:
    """q_h(s) = sum_j alpha_j B_j(s) for each data set: (nrhs, len(s))."""
    alpha = np.asarray(alpha, np.float64).reshape(-1, disc.n)
    return alpha @ disc.test_basis(s)[0]


def potential_sum(x, f_t, f1_t, w, q, uD=None) -> np.ndarray:
    """Quadrature form of the representation formula (Sect. 2) at points x
    (2, P), from the rule (t_g, w_g): f_t = f(t_g), f1_t = f'(t_g), densities
    q (nrhs, Ng) and, for a closed curve, u_D (nrhs, Ng) at t_g:
      u(x) = -(1/2 pi) sum_g w_g J(t_g) ln|x - f(t_g)| q_g
             + (1/2 pi) sum_g w_g Kbar(x, t_g) u_D(t_g).
    Returns (nrhs, P)."""
    J = np.hypot(f1_t[0], f1_t[1])
    dx = f_t[0][None, :] - x[0][:, None]                 # (P, Ng)
    dy = f_t[1][None, :] - x[1][:, None]
    logr = 0.5 * np.log(dx * dx + dy * dy)
    u = -(logr @ (w * J * q).T) / (2.0 * np.pi)
    if uD is not None:
        Kb = kernel_Kbar(x, f_t, f1_t)                   # (P, Ng)
        u = u + (Kb @ (w * uD).T) / (2.0 * np.pi)
    return u.T


def eval_potential(curve, n_elems: int, degree: int, n_ref: int, alpha, uD_gauss, points) -> np.ndarray:
    """u at `points` (P, 2) from the solution alpha (nrhs, n) and, for a
    closed curve, u_D at the right-hand side's Gauss points (nrhs, Ng).
    Valid away from the curve (a few refined elements or more)."""
    disc = make_discretization(curve, n_elems, degree, n_ref)
    tg, wg = disc.fine_gauss(G_RHS)
    ft, f1t, _ = geometry_at(curve, tg)
    q = density_at(disc, alpha, tg)
    uD = None
    if disc.closed:
        uD = np.asarray(uD_gauss, np.float64).reshape(-1, len(tg))
    x = np.asarray(points, np.float64).reshape(-1, 2).T
    return potential_sum(x, ft, f1t, wg, q, uD)


def outward_normal(f1):
    J = np.hypot(f1[0], f1[1])
    return np.stack([f1[1] / J, -f1[0] / J])


def errors(disc: Discretization, alpha: np.ndarray, exact) -> tuple[float, float]:
    """(E_R, E_M) of q_h = sum_j alpha_j B_j against exact(s) (Sect. 6)."""
    tg, wg = disc.fine_gauss(10)
    qh = alpha @ disc.test_basis(tg)[0]
    qe = exact(tg)
    ER = float(np.sqrt(np.sum(wg * (qh - qe) ** 2) / np.sum(wg * qe ** 2)))
    su = np.linspace(disc.a, disc.b, 500)
    EM = float(np.max(np.abs(alpha @ disc.test_basis(su)[0] - exact(su))))
    return ER, EM
