"""Seeded synthetic inputs: boundary curves, discretisation sizes and Dirichlet data.

This module builds INPUTS only -- control polygons, knot vectors, request mixes
and manufactured harmonic data.  It holds none of the assembly method's
arithmetic (no quadrature rule, no kernel, no moment), so both the CUDA path
and the CPU oracle may take their inputs from here.

Curves follow the representation of Sect. 3 of the paper: a degree-d spline
(optionally rational) f(s) = sum_i Q_i B_{i,d}(s) on an extended knot vector T,
with s in I = [T[d], T[N]].  Closed curves repeat the first d control points at
the end (the periodic convention of Sect. 3) or, for the clamped NURBS circle,
repeat the first control point.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Curve:
    """A spline / NURBS boundary curve.

    degree  : polynomial degree of the geometry basis
    knots   : extended knot vector T, length n_ctrl + degree + 1 (float64)
    ctrl    : control points Q, shape (n_ctrl, 2) (float64)
    weights : NURBS weights, shape (n_ctrl,), or None for a plain B-spline
    closed  : True for a closed boundary (interior problem)
    """
    degree: int
    knots: np.ndarray
    ctrl: np.ndarray
    weights: np.ndarray | None
    closed: bool

    @property
    def interval(self) -> tuple[float, float]:
        n = len(self.ctrl)
        return float(self.knots[self.degree]), float(self.knots[n])


def nurbs_circle(r: float = 0.5) -> Curve:
    """Exact quadratic NURBS circle of radius r: 9 control points on the
    circumscribed square, clamped knots with double interior knots at 1/4,
    1/2, 3/4, weights alternating 1 and sqrt(2)/2.  Counter-clockwise."""
    knots = np.array([0, 0, 0, .25, .25, .5, .5, .75, .75, 1, 1, 1], dtype=np.float64)
    ctrl = r * np.array([[1, 0], [1, 1], [0, 1], [-1, 1], [-1, 0],
                         [-1, -1], [0, -1], [1, -1], [1, 0]], dtype=np.float64)
    s2 = math.sqrt(2.0) / 2.0
    w = np.array([1, s2, 1, s2, 1, s2, 1, s2, 1], dtype=np.float64)
    return Curve(2, knots, ctrl, w, True)


def _periodic_cubic_interpolant(points: np.ndarray) -> Curve:
    """Periodic uniform cubic B-spline through `points` (m x 2) at the
    breakpoints s_j = j/m of [0, 1].

    On uniform knots a cubic B-spline takes the values 1/6, 2/3, 1/6 at the
    three breakpoints inside its support, so the control points c solve the
    circulant system (c_j + 4 c_{j+1} + c_{j+2}) / 6 = X_j (indices mod m).
    """
    m = len(points)
    circ = np.zeros((m, m))
    for j in range(m):
        circ[j, j % m] += 1.0 / 6.0
        circ[j, (j + 1) % m] += 4.0 / 6.0
        circ[j, (j + 2) % m] += 1.0 / 6.0
    c = np.linalg.solve(circ, points)
    d = 3
    ctrl = np.concatenate([c, c[:d]], axis=0)            # last d repeat the first d
    knots = (np.arange(m + 2 * d + 1, dtype=np.float64) - d) / m
    return Curve(d, knots, ctrl, None, True)


def star_curve(n_ctrl: int = 256, r0: float = 0.4, amp: float = 0.2, k: int = 5) -> Curve:
    """Star r(theta) = r0 (1 + amp cos(k theta)) interpolated by a periodic
    cubic B-spline with n_ctrl control points (counter-clockwise)."""
    th = 2.0 * np.pi * np.arange(n_ctrl) / n_ctrl
    r = r0 * (1.0 + amp * np.cos(k * th))
    return _periodic_cubic_interpolant(np.stack([r * np.cos(th), r * np.sin(th)], axis=1))


def random_star(rng: np.random.Generator, n_ctrl: int = 256, r0: float = 0.4) -> Curve:
    """Random star r(theta) = r0 (1 + sum_{k=2..6} a_k cos(k theta + phi_k)),
    a_k ~ U(0, 0.04), phi_k ~ U(0, 2 pi), periodic cubic interpolant."""
    a = rng.uniform(0.0, 0.04, size=5)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=5)
    th = 2.0 * np.pi * np.arange(n_ctrl) / n_ctrl
    r = r0 * (1.0 + sum(a[i] * np.cos((i + 2) * th + phi[i]) for i in range(5)))
    return _periodic_cubic_interpolant(np.stack([r * np.cos(th), r * np.sin(th)], axis=1))


def parabola_arc() -> Curve:
    """Open arc x1 = t, x2 = 1 - t^2, t in [-1, 1]: quadratic Bezier with
    knots [-1,-1,-1,1,1,1] and control points (-1,0), (0,2), (1,0)."""
    knots = np.array([-1, -1, -1, 1, 1, 1], dtype=np.float64)
    ctrl = np.array([[-1, 0], [0, 2], [1, 0]], dtype=np.float64)
    return Curve(2, knots, ctrl, None, False)


# ---------------------------------------------------------------------------
# Manufactured harmonic Dirichlet data (value and gradient); flux q = grad u . n
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Harmonic:
    kind: str                    # "x2-y2" | "log"
    x0: tuple[float, float] = (2.0, 1.0)

    def value(self, x: np.ndarray, y: np.ndarray) -> np.ndarray:
        if self.kind == "x2-y2":
            return x * x - y * y
        if self.kind == "log":
            return 0.5 * np.log((x - self.x0[0]) ** 2 + (y - self.x0[1]) ** 2)
        if self.kind == "one":
            return np.ones_like(x)
        raise ValueError(self.kind)

    def grad(self, x: np.ndarray, y: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
        if self.kind == "x2-y2":
            return 2 * x, -2 * y
        if self.kind == "log":
            dx, dy = x - self.x0[0], y - self.x0[1]
            r2 = dx * dx + dy * dy
            return dx / r2, dy / r2
        if self.kind == "one":
            return np.zeros_like(x), np.zeros_like(y)
        raise ValueError(self.kind)


def rhs_source(k: int, nrhs: int) -> Harmonic:
    """k-th of nrhs point-source data u = log|x - x0_k|, x0_k on radius 2.5."""
    ang = 2.0 * np.pi * k / max(nrhs, 1)
    return Harmonic("log", (2.5 * math.cos(ang), 2.5 * math.sin(ang)))


# ---------------------------------------------------------------------------
# Workload configurations (sizes and seeds)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Problem:
    name: str
    curve: Curve
    n_elems: int          # N_h, uniform discretisation elements (closed: DoF = N_h)
    degree: int           # p, degree of the discretisation space
    n_ref: int            # N_ref, refinement of the exactness space
    data: Harmonic


def config_circle() -> Problem:
    """Disk of radius 0.5, exact NURBS circle, periodic cubic, n = 64, u = x^2 - y^2."""
    return Problem("circle_r0.5_n64_p3", nurbs_circle(0.5), 64, 3, 2, Harmonic("x2-y2"))


def config_star(n: int = 2048, p: int = 3) -> Problem:
    """Star r = 0.4(1 + 0.2 cos 5 theta), 256-point periodic cubic, u = log|x-(2,1)|."""
    return Problem(f"star256_n{n}_p{p}", star_curve(), n, p, 2, Harmonic("log", (2.0, 1.0)))


def batch_mix(count: int = 1024, seed: int = 4, n_lo: int = 64, n_hi: int = 4096) -> list[Problem]:
    """Uneven batch: random stars, n log-uniform in [n_lo, n_hi], p in {2,3,4}."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(count):
        curve = random_star(rng)
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        p = int(rng.integers(2, 5))
        out.append(Problem(f"batch{r}_n{n}_p{p}", curve, n, p, 2, Harmonic("log", (2.0, 1.0))))
    return out


def serve_arrivals(rate_hz: float = 2000.0, duration_s: float = 10.0, seed: int = 5,
                   n_lo: int = 128, n_hi: int = 16384) -> list[tuple[float, Problem, int]]:
    """Poisson arrivals of (time, problem, nrhs) requests."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s:
            break
        curve = random_star(rng)
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        p = int(rng.integers(2, 5))
        nrhs = int(rng.integers(1, 9))
        out.append((t, Problem(f"req{len(out)}_n{n}_p{p}", curve, n, p, 2, Harmonic("log")), nrhs))
    return out
