// Device B-spline helpers (Cox-de Boor recurrence, Sect. 4.2 of the paper).
#pragma once
#include <cuda_runtime.h>

namespace igs {

// Knot interval k (deg <= k <= nb-1) with knots[k] <= t < knots[k+1]; t at the
// right end of I maps to the last non-empty interval.
__device__ __forceinline__ int find_span(const double* __restrict__ knots, int nb, int deg, double t) {
    if (t >= knots[nb]) {
        int k = nb - 1;
        while (k > deg && !(knots[k] < knots[k + 1])) --k;
        return k;
    }
    if (t <= knots[deg]) {
        int k = deg;
        while (k < nb - 1 && !(knots[k] < knots[k + 1])) ++k;
        return k;
    }
    int lo = deg, hi = nb;              // knots[lo] <= t < knots[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (t >= knots[mid]) lo = mid; else hi = mid;
    }
    return lo;
}

// Values of the DEG+1 B-splines non-zero on knot interval `span` at t:
// N[r] = B_{span-DEG+r, DEG}(t).  Triangular form of the Cox-de Boor
// recurrence; the degree is a template parameter so that every loop is
// unrolled and every array index is static.
template <int DEG>
__device__ __forceinline__ void basis_fixed(const double* __restrict__ knots, int span, double t, double* N) {
    double left[DEG + 1], right[DEG + 1], V[DEG + 1];
    V[0] = 1.0;
#pragma unroll
    for (int j = 1; j <= DEG; ++j) {
        left[j] = t - knots[span + 1 - j];
        right[j] = knots[span + j] - t;
        double saved = 0.0;
#pragma unroll
        for (int r = 0; r < j; ++r) {
            const double tmp = V[r] / (right[r + 1] + left[j - r]);
            V[r] = saved + right[r + 1] * tmp;
            saved = left[j - r] * tmp;
        }
        V[j] = saved;
    }
#pragma unroll
    for (int r = 0; r <= DEG; ++r) N[r] = V[r];
}

// Values N[r] and first derivatives dN[r] of B_{span-DEG+r, DEG} at t, from
// B'_{i,p} = p (B_{i,p-1}/(t_{i+p}-t_i) - B_{i+1,p-1}/(t_{i+p+1}-t_{i+1})).
template <int DEG>
__device__ __forceinline__ void basis_fixed_d1(const double* __restrict__ knots, int span, double t, double* N,
                                               double* dN) {
    double lower[DEG + 1];
    lower[DEG] = 0.0;
    basis_fixed<DEG - 1>(knots, span, t, lower);            // B_{span-DEG+1+r, DEG-1}
    basis_fixed<DEG>(knots, span, t, N);
#pragma unroll
    for (int r = 0; r <= DEG; ++r) {
        const int i = span - DEG + r;
        double v = 0.0;
        if (r >= 1) {
            const double den = knots[i + DEG] - knots[i];
            if (den > 0) v += lower[r - 1] / den;
        }
        if (r <= DEG - 1) {
            const double den = knots[i + DEG + 1] - knots[i + 1];
            if (den > 0) v -= lower[r] / den;
        }
        dN[r] = DEG * v;
    }
}

// Runtime-degree front end (1 <= deg <= 7): dispatch to the unrolled version.
__device__ __forceinline__ void basis_funs(const double* __restrict__ knots, int span, int deg, double t, double* N) {
    switch (deg) {
        case 1: basis_fixed<1>(knots, span, t, N); break;
        case 2: basis_fixed<2>(knots, span, t, N); break;
        case 3: basis_fixed<3>(knots, span, t, N); break;
        case 4: basis_fixed<4>(knots, span, t, N); break;
        case 5: basis_fixed<5>(knots, span, t, N); break;
        case 6: basis_fixed<6>(knots, span, t, N); break;
        default: basis_fixed<7>(knots, span, t, N); break;
    }
}

// Uniform cardinal pieces: value of B-bar_{e+r} at local coordinate u in
// element e is N_d(d - r + u) = sum_k piece[(d-r)(d+1)+k] u^k.
__device__ __forceinline__ double piece_eval(const double* __restrict__ piece, int d, int l, double u) {
    double v = piece[l * (d + 1) + d];
    for (int k = d - 1; k >= 0; --k) v = v * u + piece[l * (d + 1) + k];
    return v;
}

}  // namespace igs

namespace igs {
// NURBS point, derivative and speed at parameter s (Sect. 3, eq. J):
// f = N/W with N = sum w_i Q_i B_i, W = sum w_i B_i; f' = (N' - W' f)/W.
// out: x, y, x', y', J.
template <int DEG>
__device__ __forceinline__ void curve_point(int nb, const double* __restrict__ knots, const double* __restrict__ ctrl,
                                            const double* __restrict__ w, double s, double* out) {
    const int span = find_span(knots, nb, DEG, s);
    double N[DEG + 1], dN[DEG + 1];
    basis_fixed_d1<DEG>(knots, span, s, N, dN);
    double nx = 0, ny = 0, W = 0, dnx = 0, dny = 0, dW = 0;
#pragma unroll
    for (int r = 0; r <= DEG; ++r) {
        const int i = span - DEG + r;
        const double wi = w[i];
        const double px = ctrl[2 * i], py = ctrl[2 * i + 1];
        nx += wi * px * N[r]; ny += wi * py * N[r]; W += wi * N[r];
        dnx += wi * px * dN[r]; dny += wi * py * dN[r]; dW += wi * dN[r];
    }
    const double fx = nx / W, fy = ny / W;
    const double fx1 = (dnx - dW * fx) / W, fy1 = (dny - dW * fy) / W;
    out[0] = fx;
    out[1] = fy;
    out[2] = fx1;
    out[3] = fy1;
    out[4] = sqrt(fx1 * fx1 + fy1 * fy1);
}

// Runtime geometry degree -> compile-time evaluator.
__device__ __forceinline__ void curve_point_any(int deg, int nb, const double* __restrict__ knots,
                                                const double* __restrict__ ctrl, const double* __restrict__ w,
                                                double s, double* out) {
    switch (deg) {
        case 1: curve_point<1>(nb, knots, ctrl, w, s, out); break;
        case 2: curve_point<2>(nb, knots, ctrl, w, s, out); break;
        case 3: curve_point<3>(nb, knots, ctrl, w, s, out); break;
        case 4: curve_point<4>(nb, knots, ctrl, w, s, out); break;
        case 5: curve_point<5>(nb, knots, ctrl, w, s, out); break;
        case 6: curve_point<6>(nb, knots, ctrl, w, s, out); break;
        default: curve_point<7>(nb, knots, ctrl, w, s, out); break;
    }
}
}  // namespace igs

