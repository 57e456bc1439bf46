"""B-spline and NURBS evaluation (oracle; test infrastructure only).

Sect. 3 of the paper represents the boundary as f(s) = sum_i Q_i B_{i,d}(s) on
an extended knot vector T = {t_1 <= ... <= t_{N+d+1}} with I = [t_{d+1}, t_{N+1}].
The B-splines are those of the Cox-de Boor recurrence (quoted in Sect. 4.2):

    B_{j,0}(t) = 1 on [t_j, t_{j+1}), else 0
    B_{j,r}(t) = (t - t_j)/(t_{j+r} - t_j) B_{j,r-1}(t)
               + (t_{j+r+1} - t)/(t_{j+r+1} - t_{j+1}) B_{j+1,r-1}(t)

(addends with a zero denominator are dropped).  The right end point b of I
is assigned to the last non-empty knot interval, so that the basis is
continuous from the left there.  Indices here are 0-based.
"""
from __future__ import annotations

import numpy as np


def _span(knots: np.ndarray, d: int, n_basis: int, x: np.ndarray) -> np.ndarray:
    """Knot-interval index k with t_k <= x < t_{k+1}, d <= k <= n_basis-1;
    x = t_{n_basis} (right end of I) maps to the last non-empty interval."""
    k = np.searchsorted(knots, x, side="right") - 1
    k = np.clip(k, d, n_basis - 1)
    # step back over empty intervals (repeated knots) at the right end
    while True:
        bad = knots[k + 1] <= knots[k]
        if not bad.any():
            return k
        k = np.where(bad, k - 1, k)


def basis_all(knots, d: int, x, nder: int = 0) -> np.ndarray:
    """Values and derivatives of every B-spline of degree d on `knots` at x.

    Returns an array of shape (nder+1, n_basis, len(x)); entry [r, i, p] is
    the r-th derivative of B_{i,d} at x[p].  Plain Cox-de Boor recurrence on
    the degree-0 indicators of the knot interval containing each point;
    derivatives by the standard formula
        B'_{i,r} = r (B_{i,r-1}/(t_{i+r}-t_i) - B_{i+1,r-1}/(t_{i+r+1}-t_{i+1})).
    """
    t = np.asarray(knots, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n_basis = len(t) - d - 1
    span = _span(t, d, n_basis, x)
    # degree-0 indicators on the full knot vector
    levels = []
    B = np.zeros((len(t) - 1, len(x)))
    B[span, np.arange(len(x))] = 1.0
    levels.append(B)
    for r in range(1, d + 1):
        prev = levels[-1]
        nb = len(t) - r - 1
        Bn = np.zeros((nb, len(x)))
        for i in range(nb):
            den1 = t[i + r] - t[i]
            den2 = t[i + r + 1] - t[i + 1]
            if den1 > 0:
                Bn[i] += (x - t[i]) / den1 * prev[i]
            if den2 > 0:
                Bn[i] += (t[i + r + 1] - x) / den2 * prev[i + 1]
        levels.append(Bn)
    out = np.zeros((nder + 1, n_basis, len(x)))
    out[0] = levels[d]
    for q in range(1, nder + 1):
        # q-th derivative of degree-d B-splines from degree (d-q) values:
        # apply the derivative formula q times, starting from level d-q.
        if q > d:
            break
        cur = levels[d - q].copy()
        for r in range(d - q + 1, d + 1):
            nb = len(t) - r - 1
            nxt = np.zeros((nb, len(x)))
            for i in range(nb):
                den1 = t[i + r] - t[i]
                den2 = t[i + r + 1] - t[i + 1]
                if den1 > 0:
                    nxt[i] += r * cur[i] / den1
                if den2 > 0:
                    nxt[i] -= r * cur[i + 1] / den2
            cur = nxt
        out[q] = cur[:n_basis]
    return out


def curve_eval(curve, s, nder: int = 1):
    """Point, first and (optionally) second derivative of the (rational) curve.

    Returns a list [f, f', f'' ...] of arrays of shape (2, len(s)).  For a
    NURBS curve f = N/W with N = sum w_i Q_i B_i and W = sum w_i B_i, the
    derivatives follow from the quotient rule:
        f'  = (N' - W' f) / W
        f'' = (N'' - 2 W' f' - W'' f) / W
    """
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    Bd = basis_all(curve.knots, curve.degree, s, nder)
    w = np.ones(len(curve.ctrl)) if curve.weights is None else np.asarray(curve.weights, np.float64)
    Q = np.asarray(curve.ctrl, np.float64)
    Nd = [(Q * w[:, None]).T @ Bd[r] for r in range(nder + 1)]    # (2, len(s))
    Wd = [w @ Bd[r] for r in range(nder + 1)]                     # (len(s),)
    f = Nd[0] / Wd[0]
    out = [f]
    if nder >= 1:
        f1 = (Nd[1] - Wd[1] * f) / Wd[0]
        out.append(f1)
    if nder >= 2:
        f2 = (Nd[2] - 2 * Wd[1] * out[1] - Wd[2] * f) / Wd[0]
        out.append(f2)
    return out
