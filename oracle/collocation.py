"""Collocation form of the single-layer equation (oracle; test infrastructure only).

The paper remarks (Sect. 7) that its quadrature rules serve collocation BEM
as they are: the outer integral of the Galerkin form is dropped, the equation
is imposed at one collocation point per unknown, and the inner integrals use
the same rules.  On a closed curve (interior Dirichlet problem, direct
method) the equation at a boundary point x = f(s) is

    -(1/2 pi) int ln|x - y| q(y) dgamma_y = u_D(x)/2 - (1/2 pi) int d/dn_y ln|x - y| u_D(y) dgamma_y,

(the pointwise form of eq. seconda_BIE).  With the collocation points at
nodes eta_m (so that the singular rule w^{eta_m} of Algorithm 2 applies):

    Ac[i, j] = -(1/2 pi) (C0 P + W^s Q)[m_i, j]   (the inner sums of eqs. IK1e2, IK1e2_bis),
    beta_c[i] = u_D(eta_{m_i})/2 - v(eta_{m_i})/(2 pi),
    v(eta_m) = sum_g w_g Kbar(eta_m, t_g) u_D(t_g)   (the b2 inner rule of Sect. 5).

The paper fixes no collocation points; m_i is the node nearest the centre of
the support of B_i (the Greville abscissa of the uniform cyclic basis),
a + h (i + (1 - d)/2) modulo |I|, measured periodically in exact integer units
of h_f / (2(d+1)), ties to the smaller node index.  Ac is not symmetric: the
solve is an LU factorisation with partial pivoting (LAPACK getrf/getrs).
Closed curves only.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import rules
from .assembly import G_RHS, geometry_at, kernel_Kbar, kernel_K1, make_discretization
from .discretization import Discretization


def collocation_nodes(disc: Discretization) -> np.ndarray:
    """Node index m_i for each test function i (closed curves)."""
    if not disc.closed:
        raise ValueError("collocation is defined here for closed curves only")
    den = 2 * (disc.d + 1)
    pos = np.rint(disc.node_pos * den).astype(np.int64)          # node offsets from a, units h_f/den
    period = disc.M * den
    i = np.arange(disc.Nh, dtype=np.int64)
    centre = np.mod((2 * i + 1 - disc.d) * disc.Nref * den // 2, period)
    dist = np.abs(centre[:, None] - pos[None, :])
    dist = np.minimum(dist, period - dist)
    m = np.argmin(dist, axis=1)                                  # first minimum: smaller index
    assert len(np.unique(m)) == len(m)
    return m


def collocation_matrix(curve, n_elems: int, degree: int, n_ref: int = 2, rows=None):
    """(Ac, m): the n x n collocation matrix (or its rows `rows`) and the
    collocation nodes of those rows."""
    disc = make_discretization(curve, n_elems, degree, n_ref)
    m = collocation_nodes(disc)
    if rows is not None:
        m = m[np.asarray(rows)]
    W = rules.regular_rules(disc)
    Ws = rules.singular_rules(disc, m)                           # rows w^{eta_m}
    f, f1, J = geometry_at(curve, disc.eta)
    P = J[:, None] * W
    Q = J[:, None] * disc.test_basis(disc.eta)[0].T
    C0 = kernel_K1(disc, f[:, m], J[m], disc.eta[m], f, disc.eta)
    Ac = -(C0 @ P + Ws @ Q) / (2.0 * np.pi)
    return Ac, m


def collocation_rhs(curve, n_elems: int, degree: int, n_ref: int, uD_nodes, uD_gauss) -> np.ndarray:
    """beta_c (n x nrhs) from u_D at the nodes (Nq, nrhs) and at the Gauss
    points of the right-hand side's rule (Ng, nrhs)."""
    disc = make_discretization(curve, n_elems, degree, n_ref)
    m = collocation_nodes(disc)
    f, _, _ = geometry_at(curve, disc.eta[m])
    tg, wg = disc.fine_gauss(G_RHS)
    ft, f1t, _ = geometry_at(curve, tg)
    uD_nodes = np.asarray(uD_nodes, np.float64).reshape(disc.Nq, -1)
    uD_gauss = np.asarray(uD_gauss, np.float64).reshape(len(tg), -1)
    v = kernel_Kbar(f, ft, f1t) @ (wg[:, None] * uD_gauss)
    return 0.5 * uD_nodes[m] - v / (2.0 * np.pi)


def collocation_solve(Ac: np.ndarray, beta: np.ndarray) -> np.ndarray:
    """alpha from Ac alpha = beta by LU with partial pivoting."""
    return sla.lu_solve(sla.lu_factor(Ac), beta)
