// Host planner: integer description of the discretisation (Sect. 3 and 4).
//
// * Test space: N_h uniform elements; closed curves use the cyclic basis of
//   Sect. 3 (n = N_h), open arcs clamped knots (n = N_h + d).  Test function i
//   is the B-spline with support [t_i, t_{i+d+1}] of the extended knot vector,
//   i.e. coarse elements i-d .. i; for a closed curve the indices i >= N_h are
//   the wrapped copies of i - N_h ("unrolled" indices).
// * Exactness space: uniform B-splines on M = N_ref N_h refined elements,
//   restricted to I; B-bar_j covers refined elements j-d .. j, j = 0 .. M+d-1.
// * Nodes (Sect. 4): d+2 uniform points in the first and last refined element,
//   breakpoints and midpoints in the inner ones, N_quad = 2d + 2M - 1.
// * N^(i) (Sect. 4.1): nodes where B_i is non-zero (the paper's footnote: the
//   support is the set where the function does not vanish).  For a closed
//   curve the seam nodes eta = a and eta = b both belong to the wrapped
//   functions; node ranges are stored in "unrolled" node indices u, with
//   physical node u mod N_quad, so that every N^(i) is one contiguous range.
#include <algorithm>
#include <cmath>
#include <sstream>

#include "igs_internal.h"

namespace igs {

static double binom(int n, int k) {
    double r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

int build_plan(Plan& p, double a, double b, int Nh, int d, int Nref, int closed, std::string& err) {
    std::ostringstream os;
    if (d < 2 || d > kMaxDegree) { os << "degree must be in [2," << kMaxDegree << "]"; err = os.str(); return IGS_E_INVALID_ARG; }
    if (Nref < 1 || Nref > kMaxNref) { os << "n_ref must be in [1," << kMaxNref << "]"; err = os.str(); return IGS_E_INVALID_ARG; }
    if (!(b > a)) { err = "empty parameter interval"; return IGS_E_INVALID_ARG; }
    if (closed && Nh < 2 * (d + 1)) { err = "closed curves need n_elems >= 2(degree+1)"; return IGS_E_INVALID_ARG; }
    if (Nh < 1 || (long long)Nh * Nref < 3) { err = "need n_elems * n_ref >= 3"; return IGS_E_INVALID_ARG; }
    if ((long long)Nh * Nref > (1 << 26)) { err = "problem too large"; return IGS_E_INVALID_ARG; }

    p.d = d; p.Nh = Nh; p.Nref = Nref; p.closed = closed ? 1 : 0;
    p.n = closed ? Nh : Nh + d;
    p.M = Nh * Nref;
    p.Nq = 2 * d + 2 * p.M - 1;
    p.NE = p.M + d;
    p.den = 2 * (d + 1);
    p.a = a; p.b = b; p.L = b - a; p.h = p.L / Nh; p.hf = p.L / p.M;
    const int M = p.M, Nq = p.Nq, den = p.den, n = p.n;
    const int cunit = den * Nref;                 // one coarse element in position units

    // node positions (units of h_f / den)
    p.pos_num.resize(Nq);
    for (int m = 0; m <= d + 1; ++m) p.pos_num[m] = 2 * m;
    for (int k = 0; k <= 2 * M - 6; ++k) p.pos_num[d + 2 + k] = (3 + k) * (d + 1);
    for (int k = 0; k <= d + 1; ++k) p.pos_num[d + 2 * M - 3 + k] = 2 * (d + 1) * (M - 1) + 2 * k;
    for (int m = 1; m < Nq; ++m)
        if (p.pos_num[m] <= p.pos_num[m - 1]) { err = "internal: node order"; return IGS_E_INVALID_ARG; }

    p.jfirst.resize(Nq); p.member.resize(Nq); p.fspan.resize(Nq);
    for (int m = 0; m < Nq; ++m) {
        const int P = p.pos_num[m];
        p.jfirst[m] = P / cunit;
        const bool onbreak = (P % cunit) == 0;
        const int cnt = onbreak ? d : d + 1;
        p.member[m] = (1 << cnt) - 1;
        p.fspan[m] = std::min(P / den, M - 1);
    }
    if (!closed) {
        p.member[0] = 1;                          // only B_1(a) = 1 (clamped)
        p.member[Nq - 1] = 1 << (d - 1);          // only B_n(b) = 1: n-1 = N_h + d - 1 = jfirst + d - 1
    }

    // N^(i) as unrolled node ranges
    p.lo.assign(n, INT32_MAX); p.hi.assign(n, INT32_MIN);
    std::vector<int> cnt(n, 0);
    for (int m = 0; m < Nq; ++m) {
        for (int r = 0; r <= d; ++r) {
            if (!((p.member[m] >> r) & 1)) continue;
            int iu = p.jfirst[m] + r;
            int i = iu, u = m;
            if (closed && iu >= n) { i = iu - n; u = m - Nq; }
            if (i < 0 || i >= n) { err = "internal: band index"; return IGS_E_INVALID_ARG; }
            p.lo[i] = std::min(p.lo[i], u);
            p.hi[i] = std::max(p.hi[i], u);
            cnt[i]++;
        }
    }
    p.max_nodes_i = 0;
    for (int i = 0; i < n; ++i) {
        if (cnt[i] == 0 || p.hi[i] - p.lo[i] + 1 != cnt[i]) { err = "internal: N^(i) not contiguous"; return IGS_E_INVALID_ARG; }
        p.max_nodes_i = std::max(p.max_nodes_i, cnt[i]);
    }

    // J^(i) and the refined elements of supp(B_i)
    p.jlo1.resize(n); p.jhi1.resize(n); p.jlo2.resize(n); p.jhi2.resize(n);
    p.elo1.resize(n); p.ehi1.resize(n); p.elo2.resize(n); p.ehi2.resize(n);
    p.max_fine_i = 0;
    for (int i = 0; i < n; ++i) {
        int e0, e1, f0 = 0, f1 = 0;
        if (closed) {
            e0 = (i - d) * Nref; e1 = (i + 1) * Nref;
            if (e0 < 0) { f0 = e0 + M; f1 = M; e0 = 0; }
        } else {
            e0 = std::max(0, i - d) * Nref;
            e1 = (std::min(Nh - 1, i) + 1) * Nref;
        }
        p.elo1[i] = e0; p.ehi1[i] = e1; p.jlo1[i] = e0; p.jhi1[i] = e1 - 1 + d;
        if (f1 > f0) { p.elo2[i] = f0; p.ehi2[i] = f1; p.jlo2[i] = f0; p.jhi2[i] = f1 - 1 + d; }
        else { p.elo2[i] = 0; p.ehi2[i] = 0; p.jlo2[i] = 0; p.jhi2[i] = -1; }
        int nf = (p.jhi1[i] - p.jlo1[i] + 1) + (p.jhi2[i] - p.jlo2[i] + 1);
        p.max_fine_i = std::max(p.max_fine_i, nf);
    }

    // node range touching each exactness function: positions in [(j-d), (j+1)] h_f
    p.gfirst.resize(p.NE); p.glast.resize(p.NE);
    for (int j = 0; j < p.NE; ++j) {
        int lo = (j - d) * den, hi = (j + 1) * den;
        auto itl = std::lower_bound(p.pos_num.begin(), p.pos_num.end(), lo);
        auto ith = std::upper_bound(p.pos_num.begin(), p.pos_num.end(), hi);
        p.gfirst[j] = int(itl - p.pos_num.begin());
        p.glast[j] = int(ith - p.pos_num.begin()) - 1;
    }

    // cardinal B-spline pieces N_d(l + u) = sum_k piece[l][k] u^k (truncated-power formula)
    p.piece.assign((d + 1) * (d + 1), 0.0);
    double dfact = 1;
    for (int k = 2; k <= d; ++k) dfact *= k;
    for (int l = 0; l <= d; ++l)
        for (int i = 0; i <= l; ++i) {
            double sgn = (i % 2) ? -1.0 : 1.0;
            for (int k = 0; k <= d; ++k)
                p.piece[l * (d + 1) + k] += sgn * binom(d + 1, i) * binom(d, k) * std::pow(double(l - i), d - k) / dfact;
        }

    // far-field series: int_0^1 u^k ln|u - c| du = ln|c - 1/2|/(k+1) - sum_q S[k][q] (c - 1/2)^{-q}
    p.series.assign((d + 1) * kSeries, 0.0);
    auto mom = [](int q) { return (q % 2) ? 0.0 : 2.0 * std::pow(0.5, q + 1) / (q + 1); };
    for (int k = 0; k <= d; ++k)
        for (int q = 1; q < kSeries; ++q) {
            double s = 0;
            for (int i = 0; i <= k; ++i) s += binom(k, i) * std::pow(0.5, k - i) * mom(i + q);
            p.series[k * kSeries + q] = s / q;
        }
    return IGS_OK;
}

// Collocation node of each test function of a closed curve (the collocation
// form of the single-layer equation): the node nearest the centre of the
// support of B_i, i.e. (2i + 1 - d) N_ref den / 2 in units h_f / den, modulo
// the period M den, by periodic distance, ties to the smaller node index.
int collocation_nodes(const Plan& P, std::vector<int>& out, std::string& err) {
    if (!P.closed) { err = "collocation nodes are defined for closed curves only"; return IGS_E_INVALID_ARG; }
    const int64_t period = (int64_t)P.M * P.den;
    const std::vector<int>& pos = P.pos_num;
    out.assign(P.n, -1);
    for (int i = 0; i < P.n; ++i) {
        int64_t c = ((int64_t)(2 * i + 1 - P.d) * P.Nref * P.den) / 2;
        c %= period;
        if (c < 0) c += period;
        // the nearest nodes lie on either side of c, or at the two ends (the same point a = b)
        const int lb = int(std::lower_bound(pos.begin(), pos.end(), (int)c) - pos.begin());
        const int cand[4] = {0, lb - 1, lb, P.Nq - 1};
        int best = -1;
        int64_t bd = 0;
        for (int q = 0; q < 4; ++q) {
            const int m = cand[q];
            if (m < 0 || m >= P.Nq) continue;
            int64_t dist = c - pos[m];
            if (dist < 0) dist = -dist;
            dist = std::min(dist, period - dist);
            if (best < 0 || dist < bd || (dist == bd && m < best)) { best = m; bd = dist; }
        }
        out[i] = best;
    }
    std::vector<int> sorted(out);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) {
        err = "collocation nodes are not distinct for this discretisation";
        return IGS_E_INVALID_ARG;
    }
    return IGS_OK;
}

}  // namespace igs
