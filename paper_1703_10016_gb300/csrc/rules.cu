// Weighted quadrature rules on the device (FP64): Sect. 4, Algorithms 1 and 2.
#include <cmath>
#include <mutex>
#include <set>
#include <type_traits>

#include "bspline_dev.cuh"
#include "igs_internal.h"

namespace igs {

constexpr int kMaxLocalNodes = 64;   // |N^(i)| bound (d <= 5, N_ref <= 4)
constexpr int kMaxLocalFine = 40;    // |J^(i)| bound

// Gauss-Legendre nodes/weights on [0,1] for 1..6 points (row g-1), filled by the host.
__constant__ double c_gauss_x[6][6];
__constant__ double c_gauss_w[6][6];

// --------------------------------------------------------------- nodes, bands
// eta_m = a + h_f * pos_m; exactness functions at the node from the cardinal
// pieces; test functions jfirst..jfirst+d (cyclic: cardinal pieces in coarse
// coordinates; clamped: Cox-de Boor on the clamped knot vector).
__global__ void k_nodes_bands(int Nq, int d, int den, int Nref, int M, int closed, double a, double b, double hf,
                              const int* __restrict__ pos, const int* __restrict__ jfirst,
                              const int* __restrict__ member, const int* __restrict__ fspan,
                              const double* __restrict__ piece, const double* __restrict__ tknots, int ntb,
                              double* __restrict__ eta, double* __restrict__ Bf, double* __restrict__ Bt) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Nq) return;
    const int P = pos[m];
    double t = (m == Nq - 1) ? b : a + hf * (double(P) / den);
    eta[m] = t;
    // exactness functions e..e+d at local coordinate u in element e
    const int e = fspan[m];
    const double u = double(P - e * den) / den;
    for (int r = 0; r <= d; ++r) Bf[m * (d + 1) + r] = piece_eval(piece, d, d - r, u);
    // test functions
    const int cunit = den * Nref;
    const int jf = jfirst[m];
    if (closed) {
        const double uc = double(P - jf * cunit) / cunit;
        for (int r = 0; r <= d; ++r)
            Bt[m * (d + 1) + r] = ((member[m] >> r) & 1) ? piece_eval(piece, d, d - r, uc) : 0.0;
    } else {
        double N[kMaxDegree + 1];
        int span = find_span(tknots, ntb, d, t);
        basis_funs(tknots, span, d, t, N);
        for (int r = 0; r <= d; ++r) {
            int idx = jf + r - (span - d);
            double v = (idx >= 0 && idx <= d) ? N[idx] : 0.0;
            Bt[m * (d + 1) + r] = ((member[m] >> r) & 1) ? v : 0.0;
        }
    }
}

// ----------------------------------------------------------------- Algorithm 1
// One thread per test function i: mu^(i)_j = int B-bar_j B_i by Gauss with d+1
// points per refined element (exact), local collocation matrix (B)^(i), and the
// minimum-norm solution of (B)^(i) w = mu^(i) by Householder QR of (B)^(i)T.
__device__ double test_value(int closed, int d, int Nref, int n, const double* piece, const double* tknots, int ntb,
                             int iu, double pos_c, double t) {
    if (closed) {
        double loc = pos_c - (iu - d);                // position inside the support [0, d+1]
        if (loc <= 0.0 || loc >= d + 1) return 0.0;
        int l = (int)floor(loc);
        if (l > d) l = d;
        return piece_eval(piece, d, l, loc - l);
    }
    double N[kMaxDegree + 1];
    int span = find_span(tknots, ntb, d, t);
    basis_funs(tknots, span, d, t, N);
    int idx = iu - (span - d);
    return (idx >= 0 && idx <= d) ? N[idx] : 0.0;
}

__global__ void __launch_bounds__(64) k_regular(int n, int Nq, int d, int Nref, int M, int closed, double a, double hf,
                                                const int* __restrict__ lo, const int* __restrict__ hi,
                                                const int* __restrict__ jr, const int* __restrict__ jfirst,
                                                const int* __restrict__ fspan, const double* __restrict__ Bf,
                                                const double* __restrict__ piece, const double* __restrict__ tknots,
                                                int ntb, double* __restrict__ W, int* __restrict__ flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double A[kMaxLocalNodes][kMaxLocalFine];    // (B)^(i)T, Householder vectors below the diagonal
    double mu[kMaxLocalFine], diag[kMaxLocalFine], beta[kMaxLocalFine], z[kMaxLocalNodes];
    int fj[kMaxLocalFine];
    const int u0 = lo[i], nN = hi[i] - lo[i] + 1;
    const int* R = jr + 8 * i;
    int nJ = 0;
    for (int j = R[0]; j <= R[1]; ++j) fj[nJ++] = j;
    for (int j = R[2]; j <= R[3]; ++j) fj[nJ++] = j;
    if (nN > kMaxLocalNodes || nJ > kMaxLocalFine || nJ > nN) { atomicOr(flag, 1); return; }

    // mu^(i)_j over the refined elements of supp(B_i)
    for (int q = 0; q < nJ; ++q) mu[q] = 0.0;
    const int g = d + 1;
    for (int part = 0; part < 2; ++part) {
        const int e0 = R[4 + 2 * part], e1 = R[5 + 2 * part];
        const int iu = (closed && part == 1) ? i + n : i;          // wrapped copy near b
        for (int e = e0; e < e1; ++e) {
            for (int k = 0; k < g; ++k) {
                const double x = c_gauss_x[g - 1][k], wq = c_gauss_w[g - 1][k] * hf;
                const double t = a + hf * (e + x);
                const double bi = test_value(closed, d, Nref, n, piece, tknots, ntb, iu, (e + x) / Nref, t);
                if (bi == 0.0) continue;
                for (int r = 0; r <= d; ++r) {
                    const int j = e + r;                           // B-bar_{e+r} on element e
                    const double bj = piece_eval(piece, d, d - r, x);
                    for (int q = 0; q < nJ; ++q)
                        if (fj[q] == j) { mu[q] += wq * bj * bi; break; }
                }
            }
        }
    }
    // local matrix, transposed: A[ul][q] = B-bar_{fj[q]}(eta_{m(ul)})
    for (int ul = 0; ul < nN; ++ul) {
        int m = (u0 + ul) % Nq;
        if (m < 0) m += Nq;
        const int e = fspan[m];
        for (int q = 0; q < nJ; ++q) {
            const int r = fj[q] - e;
            A[ul][q] = (r >= 0 && r <= d) ? Bf[m * (d + 1) + r] : 0.0;
        }
    }
    // Householder QR of A (nN x nJ)
    for (int k = 0; k < nJ; ++k) {
        double nrm = 0.0;
        for (int r = k; r < nN; ++r) nrm += A[r][k] * A[r][k];
        nrm = sqrt(nrm);
        if (nrm == 0.0) { atomicOr(flag, 2); return; }
        const double alpha = (A[k][k] > 0) ? -nrm : nrm;
        A[k][k] -= alpha;
        double vn = 0.0;
        for (int r = k; r < nN; ++r) vn += A[r][k] * A[r][k];
        beta[k] = (vn > 0) ? 2.0 / vn : 0.0;
        diag[k] = alpha;
        for (int c = k + 1; c < nJ; ++c) {
            double s = 0.0;
            for (int r = k; r < nN; ++r) s += A[r][k] * A[r][c];
            s *= beta[k];
            for (int r = k; r < nN; ++r) A[r][c] -= s * A[r][k];
        }
    }
    // R^T y = mu
    for (int k = 0; k < nJ; ++k) {
        double s = mu[k];
        for (int c = 0; c < k; ++c) s -= A[c][k] * z[c];
        z[k] = s / diag[k];
    }
    for (int r = nJ; r < nN; ++r) z[r] = 0.0;
    // w = H_0 ... H_{nJ-1} [y; 0]
    for (int k = nJ - 1; k >= 0; --k) {
        double s = 0.0;
        for (int r = k; r < nN; ++r) s += A[r][k] * z[r];
        s *= beta[k];
        for (int r = k; r < nN; ++r) z[r] -= s * A[r][k];
    }
    // scatter into the node bands: slot r with jfirst[m] + r = unrolled index of i
    for (int ul = 0; ul < nN; ++ul) {
        const int u = u0 + ul;
        int m = u % Nq;
        if (m < 0) m += Nq;
        const int iu = (u < 0) ? i + n : i;
        const int r = iu - jfirst[m];
        if (r < 0 || r > d) { atomicOr(flag, 4); continue; }
        W[m * (d + 1) + r] = z[ul];
    }
}

// ----------------------------------------------------------------- Gram matrix
// G = (B)(B)^T, upper band G[j][r] = sum_m B-bar_j(eta_m) B-bar_{j+r}(eta_m).
__global__ void k_gram(int NE, int d, const int* __restrict__ gfirst, const int* __restrict__ glast,
                       const int* __restrict__ fspan, const double* __restrict__ Bf, double* __restrict__ G) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= NE) return;
    double acc[kMaxDegree + 1];
    for (int r = 0; r <= d; ++r) acc[r] = 0.0;
    for (int m = gfirst[j]; m <= glast[j]; ++m) {
        const int e = fspan[m];
        const int rj = j - e;
        if (rj < 0 || rj > d) continue;
        const double bj = Bf[m * (d + 1) + rj];
        for (int r = 0; r <= d; ++r) {
            const int rk = rj + r;
            if (rk <= d) acc[r] += bj * Bf[m * (d + 1) + rk];
        }
    }
    for (int r = 0; r <= d; ++r) G[j * (d + 1) + r] = acc[r];
}

// Banded Cholesky G = L L^T (L(j, j-r) stored at L[j][r]), one block.  G is
// Toeplitz away from the ends of I (uniform knots), and the rows of the
// Cholesky factor of a banded Toeplitz SPD matrix converge geometrically to a
// fixed row.  Thread 0 runs the recurrence until two consecutive rows agree to
// 4e-16 (relative) on equal rows of G; the block then copies that row over
// the following rows whose G rows are identical, and thread 0 finishes the
// rows after them.  Without convergence the recurrence simply runs to the end.
__device__ void chol_row(int j, int d, const double* __restrict__ G, double* __restrict__ L, int* flag) {
    const int k0 = (j - d > 0) ? j - d : 0;
    for (int k = k0; k <= j; ++k) {
        double s = G[k * (d + 1) + (j - k)];
        for (int p = k0; p < k; ++p) s -= L[j * (d + 1) + (j - p)] * L[k * (d + 1) + (k - p)];
        if (k < j) {
            L[j * (d + 1) + (j - k)] = s / L[k * (d + 1)];
        } else {
            if (!(s > 0.0)) { atomicOr(flag, 8); s = 1.0; }
            L[j * (d + 1)] = sqrt(s);
        }
    }
}

__device__ bool same_g_row(const double* G, int d, int a, int b) {
    for (int r = 0; r <= d; ++r)
        if (G[a * (d + 1) + r] != G[b * (d + 1) + r]) return false;
    return true;
}

__global__ void __launch_bounds__(256) k_chol_band(int NE, int d, const double* __restrict__ G, double* __restrict__ L,
                                                   int* __restrict__ flag) {
    __shared__ int s_conv, s_end;
    const int tid = threadIdx.x;
    if (tid == 0) {
        int conv = -1;
        for (int j = 0; j < NE; ++j) {
            chol_row(j, d, G, L, flag);
            if (j >= 4 * (d + 1) && same_g_row(G, d, j, j - 1)) {
                bool same = true;
                for (int r = 0; r <= d && same; ++r) {
                    const double a = L[j * (d + 1) + r], b = L[(j - 1) * (d + 1) + r];
                    same = fabs(a - b) <= 4e-16 * fabs(a);
                }
                if (same) { conv = j; break; }
            }
        }
        s_conv = conv;
        s_end = NE;
    }
    __syncthreads();
    const int conv = s_conv;
    if (conv < 0) return;
    // first row after conv whose G row differs from G[conv]
    for (int t = conv + 1 + tid; t < NE; t += blockDim.x)
        if (!same_g_row(G, d, t, conv)) atomicMin(&s_end, t);
    __syncthreads();
    const int end = s_end;
    for (int idx = tid; idx < (end - conv - 1) * (d + 1); idx += blockDim.x) {
        const int t = conv + 1 + idx / (d + 1), r = idx % (d + 1);
        L[t * (d + 1) + r] = L[conv * (d + 1) + r];
    }
    __syncthreads();
    if (tid == 0)
        for (int j = end; j < NE; ++j) chol_row(j, d, G, L, flag);
}

// ----------------------------------------------------------------- moments
// L_k(c) = int_0^1 u^k ln|u - c| du, k = 0..d: closed form of the paper's base
// integrals in local coordinates near the element, log series far from it.
__device__ __forceinline__ double base_F(double z, int j) {
    if (z == 0.0) return 0.0;
    double zp = z;
    for (int q = 0; q < j; ++q) zp *= z;
    return zp / (j + 1) * (log(fabs(z)) - 1.0 / (j + 1));
}

__device__ void local_log_moments(double c, int d, const double* __restrict__ series, double* Lk) {
    const double del = c - 0.5;
    if (fabs(del) <= 2.5) {
        // z = u - c: u^k = sum_i C(k,i) c^{k-i} z^i
        double F1[kMaxDegree + 1], F0[kMaxDegree + 1];
        for (int i = 0; i <= d; ++i) { F1[i] = base_F(1.0 - c, i); F0[i] = base_F(-c, i); }
        for (int k = 0; k <= d; ++k) {
            double s = 0.0, binom = 1.0, cp = 1.0;
            // sum over i = k..0 with c^{k-i}
            for (int i = k; i >= 0; --i) {
                s += binom * cp * (F1[i] - F0[i]);
                // next: i-1, binom C(k, i-1) = C(k,i) * i / (k-i+1), cp *= c
                binom = binom * i / (k - i + 1);
                cp *= c;
            }
            Lk[k] = s;
        }
    } else {
        const double lg = log(fabs(del)), rho = 1.0 / del;
        for (int k = 0; k <= d; ++k) {
            const double* S = series + k * kSeries;
            double acc = 0.0;
            for (int q = kSeries - 1; q >= 1; --q) acc = (acc + S[q]) * rho;
            Lk[k] = lg / (k + 1) - acc;
        }
    }
}

// Element moments by relative position.  E_{m,e,k} = int_e ((t - tau_e)/h_f)^k
// K2(t - eta_m) dt depends on eta_m and the element only through the offset
// du = pos_m - e den (positions in units of h_f/den, all integers), so one
// table over du in [-(M-1) den, M den] holds every moment the rules need:
// Et[(du - dmin)(d+1) + k], all K2 images included.
__global__ void k_etable(int ntab, int dmin, int d, int den, int M, int closed, double hf, double L,
                         const double* __restrict__ series, double* __restrict__ Et) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntab) return;
    const double c = double(dmin + t) / den;                  // (eta - tau_e) / h_f
    const double lhf = log(hf);
    double acc[kMaxDegree + 1];
    for (int k = 0; k <= d; ++k) acc[k] = 0.0;
    const int nimg = closed ? 3 : 1;
    for (int im = 0; im < nimg; ++im) {
        const double shift = (im == 0) ? 0.0 : (im == 1 ? -double(M) : double(M));
        double Lk[kMaxDegree + 1];
        local_log_moments(c + shift, d, series, Lk);
        for (int k = 0; k <= d; ++k) acc[k] += hf * (lhf / (k + 1) + Lk[k]);
    }
    if (closed) {
        const double c2 = 2.0 * log(L) * hf;
        for (int k = 0; k <= d; ++k) acc[k] -= c2 / (k + 1);
    }
    for (int k = 0; k <= d; ++k) Et[(size_t)t * (d + 1) + k] = acc[k];
}

// mu_j(eta_m) = sum over the elements e = j-d+l of B-bar_j's support of
// sum_k piece[l][k] E_{m,e,k} (eq. mod_mom_gen), for j in a block of 128 and
// the node rows[blockIdx.y] (or blockIdx.y); output Z[j][col].
__global__ void __launch_bounds__(128) k_mu_tab(int NE, int M, int d, int den, int dmin, const int* __restrict__ pos,
                                                const int* __restrict__ rows, const double* __restrict__ piece,
                                                const double* __restrict__ Et, double* __restrict__ Z, int ldz) {
    const int col = blockIdx.y;
    const int m = rows ? rows[col] : col;
    const int j = blockIdx.x * 128 + threadIdx.x;
    if (j >= NE) return;
    const int P = pos[m];
    double mu = 0.0;
    for (int l = 0; l <= d; ++l) {
        const int e = j - d + l;
        if (e < 0 || e >= M) continue;
        const double* E = Et + (size_t)(P - e * den - dmin) * (d + 1);
        for (int k = 0; k <= d; ++k) mu += piece[l * (d + 1) + k] * E[k];
    }
    Z[(size_t)j * ldz + col] = mu;
}

// z = G^{-1} mu in place, one thread per column (node).  The last d values of
// each substitution stay in a register window and the sum takes the most
// recent value last, so one step's dependency chain is one FMA and one
// multiply.  Everything a chunk of steps reads from memory (right-hand side,
// factor band, reciprocal diagonal) is loaded one chunk ahead, before the
// current chunk's stores, so no step waits on a memory round trip.
constexpr int kSubChunk = 8;
template <int D>
struct SubChunk {
    double z[kSubChunk];
    double l[kSubChunk][D];
    double rd[kSubChunk];
};
// forward: rows j0 .. j0+7, band entries L[j][r] (r = 1..D) of row j
template <int D>
__device__ __forceinline__ void sub_load_fwd(SubChunk<D>& c, int j0, int NE, const double* __restrict__ L,
                                             const double* __restrict__ rd, const double* Z, int ldz, int col) {
#pragma unroll
    for (int t = 0; t < kSubChunk; ++t) {
        const int j = j0 + t;
        const bool in = j < NE;
        c.z[t] = in ? Z[(size_t)j * ldz + col] : 0.0;
        c.rd[t] = in ? rd[j] : 0.0;
#pragma unroll
        for (int r = 1; r <= D; ++r) c.l[t][r - 1] = (in && j - r >= 0) ? L[j * (D + 1) + r] : 0.0;
    }
}
// backward: rows j0, j0-1, ..., band entries L[j+r][r] (column j of L)
template <int D>
__device__ __forceinline__ void sub_load_bwd(SubChunk<D>& c, int j0, int NE, const double* __restrict__ L,
                                             const double* __restrict__ rd, const double* Z, int ldz, int col) {
#pragma unroll
    for (int t = 0; t < kSubChunk; ++t) {
        const int j = j0 - t;
        const bool in = j >= 0;
        c.z[t] = in ? Z[(size_t)j * ldz + col] : 0.0;
        c.rd[t] = in ? rd[j] : 0.0;
#pragma unroll
        for (int r = 1; r <= D; ++r) c.l[t][r - 1] = (in && j + r < NE) ? L[(j + r) * (D + 1) + r] : 0.0;
    }
}
template <int D>
__device__ void gsolve_col(int NE, const double* __restrict__ L, const double* __restrict__ rd, double* __restrict__ Z,
                           int ldz, int c) {
    double win[D];
    SubChunk<D> cur, nxt;
#pragma unroll
    for (int r = 0; r < D; ++r) win[r] = 0.0;              // win[r] = z[j - 1 - r] before step j
    sub_load_fwd<D>(cur, 0, NE, L, rd, Z, ldz, c);
    for (int j0 = 0; j0 < NE; j0 += kSubChunk) {
        sub_load_fwd<D>(nxt, j0 + kSubChunk, NE, L, rd, Z, ldz, c);
#pragma unroll
        for (int t = 0; t < kSubChunk; ++t) {
            const int j = j0 + t;
            if (j < NE) {
                double s = cur.z[t];
#pragma unroll
                for (int r = D; r >= 1; --r) s -= cur.l[t][r - 1] * win[r - 1];
                const double v = s * cur.rd[t];
#pragma unroll
                for (int r = D - 1; r > 0; --r) win[r] = win[r - 1];
                win[0] = v;
                Z[(size_t)j * ldz + c] = v;
            }
        }
        cur = nxt;
    }
#pragma unroll
    for (int r = 0; r < D; ++r) win[r] = 0.0;              // win[r] = y[j + 1 + r] before step j
    sub_load_bwd<D>(cur, NE - 1, NE, L, rd, Z, ldz, c);
    for (int j0 = NE - 1; j0 >= 0; j0 -= kSubChunk) {
        sub_load_bwd<D>(nxt, j0 - kSubChunk, NE, L, rd, Z, ldz, c);
#pragma unroll
        for (int t = 0; t < kSubChunk; ++t) {
            const int j = j0 - t;
            if (j >= 0) {
                double s = cur.z[t];
#pragma unroll
                for (int r = D; r >= 1; --r) s -= cur.l[t][r - 1] * win[r - 1];
                const double v = s * cur.rd[t];
#pragma unroll
                for (int r = D - 1; r > 0; --r) win[r] = win[r - 1];
                win[0] = v;
                Z[(size_t)j * ldz + c] = v;
            }
        }
        cur = nxt;
    }
}

__global__ void k_gsolve(int NE, int d, int ncol, const double* __restrict__ L, const double* __restrict__ rd,
                         double* __restrict__ Z, int ldz) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    switch (d) {
        case 2: gsolve_col<2>(NE, L, rd, Z, ldz, c); break;
        case 3: gsolve_col<3>(NE, L, rd, Z, ldz, c); break;
        case 4: gsolve_col<4>(NE, L, rd, Z, ldz, c); break;
        default: gsolve_col<5>(NE, L, rd, Z, ldz, c); break;
    }
}

// ------------------------------------------- partitioned solve with G = L L^T
// Many-right-hand-side-free form of the two banded substitutions for a few
// dense right-hand sides (the boundary rows of W^s): rows are split into P
// blocks of kPart rows (the last block takes the remainder, so every block
// has at least d rows).  Forward, block p: L_pp y_p = mu_p - L_p,p-1 y_p-1,
// where L_p,p-1 reaches only the last d entries t_p-1 of y_p-1, so
//     y_p = u_p - sum_k t_p-1[k] V_p[k],   u_p = L_pp^{-1} mu_p,
//     V_p[k] = L_pp^{-1} (column m-k of L_p,p-1)   (k = 1..d, "spikes").
// The spikes depend on L only; the local solves run in parallel over blocks;
// only the d interface values per block are carried sequentially.  Backward
// likewise with L^T and the first d entries of the next block.  Algebraically
// this is the block form of the same substitutions (no truncation).
constexpr int kPart = 64;

__host__ __device__ inline int part_count(int NE) { return NE / kPart; }       // >= 1 when NE >= kPart
__device__ __forceinline__ int part_len(int NE, int P, int p) { return p == P - 1 ? NE - p * kPart : kPart; }

// V[(p*D + k-1)*2kPart + i] = V_p[k][i] (forward), W likewise (backward, k = 0..D-1)
template <int D>
__global__ void k_spikes(int NE, const double* __restrict__ L, const double* __restrict__ rd, double* __restrict__ V,
                         double* __restrict__ W) {
    const int P = part_count(NE);
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 2 * P * D) return;
    const bool fwd = q < P * D;
    const int p = (fwd ? q : q - P * D) / D, k = (fwd ? q : q - P * D) % D;
    const int r0 = p * kPart, len = part_len(NE, P, p);
    double* out = (fwd ? V : W) + (size_t)(p * D + k) * 2 * kPart;
    double win[D];
#pragma unroll
    for (int r = 0; r < D; ++r) win[r] = 0.0;
    if (fwd) {
        if (p == 0) return;
        // column (r0 - 1 - k) of L restricted to rows of block p: L[r0+i][r0-1-k], band offset i+1+k
        for (int i = 0; i < len; ++i) {
            const int j = r0 + i;
            double s = (i + 1 + k <= D) ? L[j * (D + 1) + i + 1 + k] : 0.0;
#pragma unroll
            for (int r = D; r >= 1; --r)
                if (i - r >= 0) s -= L[j * (D + 1) + r] * win[r - 1];
            const double v = s * rd[j];
#pragma unroll
            for (int r = D - 1; r > 0; --r) win[r] = win[r - 1];
            win[0] = v;
            out[i] = v;
        }
    } else {
        if (p == P - 1) return;
        // row (r0 + len + k) of L restricted to columns of block p, transposed:
        // rhs_i = L[r0+len+k][r0+i], band offset len+k-i
        for (int i = len - 1; i >= 0; --i) {
            const int j = r0 + i, off = len + k - i;
            double s = (off <= D) ? L[(r0 + len + k) * (D + 1) + off] : 0.0;
#pragma unroll
            for (int r = D; r >= 1; --r)
                if (i + r < len) s -= L[(j + r) * (D + 1) + r] * win[r - 1];
            const double v = s * rd[j];
#pragma unroll
            for (int r = D - 1; r > 0; --r) win[r] = win[r - 1];
            win[0] = v;
            out[i] = v;
        }
    }
}

// Local substitutions in place, one thread per (block, column): forward
// L_pp u_p = mu_p (dir 0) or backward L_pp^T u_p = y_p (dir 1), no coupling.
template <int D>
__global__ void k_part_local(int NE, int ncol, int dir, const double* __restrict__ L, const double* __restrict__ rd,
                             double* __restrict__ Z, int ldz) {
    const int P = part_count(NE);
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= P * ncol) return;
    const int p = q / ncol, c = q % ncol;
    const int r0 = p * kPart, len = part_len(NE, P, p);
    double win[D];
#pragma unroll
    for (int r = 0; r < D; ++r) win[r] = 0.0;
    if (dir == 0) {
        for (int i = 0; i < len; ++i) {
            const int j = r0 + i;
            double s = Z[(size_t)j * ldz + c];
#pragma unroll
            for (int r = D; r >= 1; --r)
                if (i - r >= 0) s -= L[j * (D + 1) + r] * win[r - 1];
            const double v = s * rd[j];
#pragma unroll
            for (int r = D - 1; r > 0; --r) win[r] = win[r - 1];
            win[0] = v;
            Z[(size_t)j * ldz + c] = v;
        }
    } else {
        for (int i = len - 1; i >= 0; --i) {
            const int j = r0 + i;
            double s = Z[(size_t)j * ldz + c];
#pragma unroll
            for (int r = D; r >= 1; --r)
                if (i + r < len) s -= L[(j + r) * (D + 1) + r] * win[r - 1];
            const double v = s * rd[j];
#pragma unroll
            for (int r = D - 1; r > 0; --r) win[r] = win[r - 1];
            win[0] = v;
            Z[(size_t)j * ldz + c] = v;
        }
    }
}

// Interface values, one warp, lane (c, k) for columns c0 <= c < c0 + nc and
// k < D (nc * D <= 32).  Forward: t_p[k] = y_p[len_p-1-k] = u_p[len_p-1-k] -
// sum_k' V_p[k'][len_p-1-k] t_p-1[k'] for p = 1..P-1 (t_0 from u_0); the
// values of t_p-1 come from the lanes of the same column by shuffles.
// Backward: s_p[k] = z_p[k] = u_p[k] - sum_k' W_p[k'][k] s_p+1[k'] for
// p = P-2..0.  T[(p*ncol + c)*D + k] receives the carried values.
template <int D>
__global__ void k_part_iface(int NE, int ncol, int c0, int nc, int dir, const double* __restrict__ Z, int ldz,
                             const double* __restrict__ VW, double* __restrict__ T) {
    const int P = part_count(NE);
    const int lane = threadIdx.x;
    const bool act = lane < nc * D;
    const int c = c0 + (act ? lane / D : 0), k = act ? lane % D : 0;
    const int base = lane - k;                                 // lane of (c, 0)
    if (dir == 0) {
        double t = act ? Z[(size_t)(kPart - 1 - k) * ldz + c] : 0.0;
        if (act) T[(size_t)(0 * ncol + c) * D + k] = t;
        for (int p = 1; p < P; ++p) {
            const int r0 = p * kPart, len = part_len(NE, P, p);
            const int i = len - 1 - k;
            double s = act ? Z[(size_t)(r0 + i) * ldz + c] : 0.0;
            double vk[D];
#pragma unroll
            for (int kk = 0; kk < D; ++kk) vk[kk] = act ? VW[(size_t)(p * D + kk) * 2 * kPart + i] : 0.0;
#pragma unroll
            for (int kk = 0; kk < D; ++kk) {
                // t_p-1[kk + 1 in 1-based] = y_p-1[m - 1 - kk]: spike kk couples entry m-1-kk
                const double tk = __shfl_sync(0xffffffffu, t, base + kk);
                s -= vk[kk] * tk;
            }
            t = s;
            if (act) T[(size_t)(p * ncol + c) * D + k] = t;
        }
    } else {
        const int rl = (P - 1) * kPart;
        double t = act ? Z[(size_t)(rl + k) * ldz + c] : 0.0;
        if (act) T[(size_t)((P - 1) * ncol + c) * D + k] = t;
        for (int p = P - 2; p >= 0; --p) {
            const int r0 = p * kPart;
            double s = act ? Z[(size_t)(r0 + k) * ldz + c] : 0.0;
            double wk[D];
#pragma unroll
            for (int kk = 0; kk < D; ++kk) wk[kk] = act ? VW[(size_t)(p * D + kk) * 2 * kPart + k] : 0.0;
#pragma unroll
            for (int kk = 0; kk < D; ++kk) {
                const double tk = __shfl_sync(0xffffffffu, t, base + kk);
                s -= wk[kk] * tk;
            }
            t = s;
            if (act) T[(size_t)(p * ncol + c) * D + k] = t;
        }
    }
}

// Corrections: forward y_p = u_p - sum_k V_p[k] t_p-1[k] (p >= 1); backward
// z_p = u_p - sum_k W_p[k] s_p+1[k] (p <= P-2).  One thread per (row, column).
template <int D>
__global__ void k_part_correct(int NE, int ncol, int dir, const double* __restrict__ VW, const double* __restrict__ T,
                               double* __restrict__ Z, int ldz) {
    const int P = part_count(NE);
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (size_t)NE * ncol) return;
    const int j = (int)(q / ncol), c = (int)(q % ncol);
    const int p = min(j / kPart, P - 1), i = j - p * kPart;
    const int pn = dir == 0 ? p - 1 : p + 1;                   // block whose interface values couple in
    if (pn < 0 || pn >= P) return;
    double s = Z[(size_t)j * ldz + c];
#pragma unroll
    for (int k = 0; k < D; ++k) s -= VW[(size_t)(p * D + k) * 2 * kPart + i] * T[(size_t)(pn * ncol + c) * D + k];
    Z[(size_t)j * ldz + c] = s;
}

// z = G^{-1} z for ncol columns of Z (ldz), partitioned (NE >= 2 kPart).
static void part_gsolve(igs_prob p, cudaStream_t s, int NE, int d, int ncol, const double* L, const double* rd,
                        double* Z, int ldz, int& launches) {
    const int P = part_count(NE);
    double* V = (double*)dev_alloc(p, sizeof(double) * (size_t)P * d * 2 * kPart);
    double* W = (double*)dev_alloc(p, sizeof(double) * (size_t)P * d * 2 * kPart);
    double* T = (double*)dev_alloc(p, sizeof(double) * (size_t)P * ncol * d);
    auto run = [&](auto dtag) {
        constexpr int D = decltype(dtag)::value;
        k_spikes<D><<<(2 * P * D + 127) / 128, 128, 0, s>>>(NE, L, rd, V, W);
        for (int dir = 0; dir < 2; ++dir) {
            const double* VW = dir == 0 ? V : W;
            k_part_local<D><<<(P * ncol + 127) / 128, 128, 0, s>>>(NE, ncol, dir, L, rd, Z, ldz);
            for (int c0 = 0; c0 < ncol; c0 += 32 / D)
                k_part_iface<D><<<1, 32, 0, s>>>(NE, ncol, c0, std::min(ncol - c0, 32 / D), dir, Z, ldz, VW, T);
            k_part_correct<D><<<(unsigned)(((size_t)NE * ncol + 255) / 256), 256, 0, s>>>(NE, ncol, dir, VW, T, Z, ldz);
        }
        launches += 5 + 2 * ((ncol + 32 / D - 1) / (32 / D));
    };
    switch (d) {
        case 2: run(std::integral_constant<int, 2>()); break;
        case 3: run(std::integral_constant<int, 3>()); break;
        case 4: run(std::integral_constant<int, 4>()); break;
        default: run(std::integral_constant<int, 5>()); break;
    }
    IGS_CUDA(cudaGetLastError());
    dev_free(p, V);
    dev_free(p, W);
    dev_free(p, T);
}

// Reciprocals of the Cholesky diagonal: the substitutions multiply instead of
// dividing (an FP64 division is a long dependent sequence on this GPU).
__global__ void k_recip_diag(int NE, int d, const double* __restrict__ L, double* __restrict__ rd) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < NE) rd[j] = 1.0 / L[j * (d + 1)];
}

// WsT[nn][m] = w^{eta_m}_{nn} = sum_r B-bar_{e+r}(eta_nn) z_m[e+r], e = fspan[nn].
__global__ void k_ws(int Nq, int d, const int* __restrict__ fspan, const double* __restrict__ Bf,
                     const double* __restrict__ Z, int ldz, double* __restrict__ WsT, float* __restrict__ WsT32) {
    const int nn = blockIdx.y;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Nq) return;
    const int e = fspan[nn];
    double s = 0.0;
    for (int r = 0; r <= d; ++r) s += Bf[nn * (d + 1) + r] * Z[(size_t)(e + r) * ldz + m];
    WsT[(size_t)nn * Nq + m] = s;
    if (WsT32) WsT32[(size_t)nn * Nq + m] = (float)s;
}

// --------------------------------------------------- compressed singular rules
// Column m' of W^s is Mu y with y = G^{-1} (B)[:, m'] (G symmetric).  y decays
// geometrically away from m', so only the elements where it is above 1e-20
// of its maximum contribute.  Away from the ends of [a, b] the columns are
// shifted copies of one another (uniform knots; period 2 in the node index),
// which the Toeplitz sequences record.

// y_c = G^{-1} (B)[:, cols[c]], one thread per column; Y[c][j] (zeroed by the
// caller).  The solution decays geometrically away from the column's
// elements: each substitution stops once d+1 consecutive values are below
// 1e-40 of the largest so far (the rest is zero to far below the 1e-20 cut
// applied afterwards).  Register window and chunked reads as in gsolve_col.
template <int D>
__device__ void ycols_col(int NE, int e0, const double* __restrict__ bf, const double* __restrict__ L,
                          const double* __restrict__ rd, double* __restrict__ y) {
    double win[D];
#pragma unroll
    for (int r = 0; r < D; ++r) win[r] = 0.0;              // win[r] = y[j - 1 - r] (zero before e0)
    double big = 0.0;
    int small = 0, jstop = NE - 1;
    for (int j = e0; j < NE; ++j) {
        double s = (j - e0 <= D) ? bf[j - e0] : 0.0;
        // only band entries of rows with a predecessor are read (the factor
        // stores nothing left of column 0)
#pragma unroll
        for (int r = D; r >= 1; --r)
            if (j - r >= e0) s -= L[j * (D + 1) + r] * win[r - 1];
        const double v = s * rd[j];
#pragma unroll
        for (int r = D - 1; r > 0; --r) win[r] = win[r - 1];
        win[0] = v;
        y[j] = v;
        big = fmax(big, fabs(v));
        small = (j > e0 + D && fabs(v) <= 1e-40 * big) ? small + 1 : 0;
        if (small > D) { jstop = j; break; }
    }
#pragma unroll
    for (int r = 0; r < D; ++r) win[r] = 0.0;              // win[r] = y[j + 1 + r] (zero past jstop)
    small = 0;
    double yc[kSubChunk];
#pragma unroll
    for (int t = 0; t < kSubChunk; ++t) yc[t] = (jstop - t >= 0) ? y[jstop - t] : 0.0;
    for (int j0 = jstop; j0 >= 0; j0 -= kSubChunk) {
        double yn[kSubChunk];
#pragma unroll
        for (int t = 0; t < kSubChunk; ++t) yn[t] = (j0 - kSubChunk - t >= 0) ? y[j0 - kSubChunk - t] : 0.0;
        bool stop = false;
#pragma unroll
        for (int t = 0; t < kSubChunk; ++t) {
            const int j = j0 - t;
            if (j >= 0 && !stop) {
                double s = yc[t];
#pragma unroll
                for (int r = D; r >= 1; --r)
                    if (j + r <= jstop) s -= L[(j + r) * (D + 1) + r] * win[r - 1];
                const double v = s * rd[j];
#pragma unroll
                for (int r = D - 1; r > 0; --r) win[r] = win[r - 1];
                win[0] = v;
                y[j] = v;
                big = fmax(big, fabs(v));
                small = (j < e0 && fabs(v) <= 1e-40 * big) ? small + 1 : 0;
                stop = small > D;
            }
        }
        if (stop) break;
#pragma unroll
        for (int t = 0; t < kSubChunk; ++t) yc[t] = yn[t];
    }
}

__global__ void k_ycols(int ncols, int NE, int d, const int* __restrict__ cols, const int* __restrict__ fspan,
                        const double* __restrict__ Bf, const double* __restrict__ L, const double* __restrict__ rd,
                        double* __restrict__ Y) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    const int mp = cols[c], e0 = fspan[mp];
    const double* bf = Bf + mp * (d + 1);
    double* y = Y + (size_t)c * NE;
    switch (d) {
        case 2: ycols_col<2>(NE, e0, bf, L, rd, y); break;
        case 3: ycols_col<3>(NE, e0, bf, L, rd, y); break;
        case 4: ycols_col<4>(NE, e0, bf, L, rd, y); break;
        default: ycols_col<5>(NE, e0, bf, L, rd, y); break;
    }
}

// Element range of each column and its per-element coefficients
// Yc[c][e - elo][k] = sum_l piece[l][k] y_c[e + d - l]; one block per column.
__global__ void __launch_bounds__(128) k_yc(int NE, int M, int d, int cap, const double* __restrict__ Y,
                                            const double* __restrict__ piece, int* __restrict__ erange,
                                            double* __restrict__ Yc, int* __restrict__ flag) {
    __shared__ double smax[128];
    __shared__ int slo[128], shi[128];
    const int c = blockIdx.x, tid = threadIdx.x;
    const double* y = Y + (size_t)c * NE;
    double mx = 0.0;
    for (int j = tid; j < NE; j += blockDim.x) mx = fmax(mx, fabs(y[j]));
    smax[tid] = mx;
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (tid < w) smax[tid] = fmax(smax[tid], smax[tid + w]);
        __syncthreads();
    }
    const double tol = 1e-20 * smax[0];
    int lo = NE, hi = -1;
    for (int j = tid; j < NE; j += blockDim.x)
        if (fabs(y[j]) > tol) { lo = min(lo, j); hi = max(hi, j); }
    slo[tid] = lo;
    shi[tid] = hi;
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (tid < w) { slo[tid] = min(slo[tid], slo[tid + w]); shi[tid] = max(shi[tid], shi[tid + w]); }
        __syncthreads();
    }
    const int elo = max(0, slo[0] - d), ehi = min(M - 1, shi[0]);
    if (ehi - elo + 1 > cap || shi[0] < 0) {
        if (tid == 0) { atomicOr(flag, 16); erange[2 * c] = 0; erange[2 * c + 1] = -1; }
        return;
    }
    if (tid == 0) { erange[2 * c] = elo; erange[2 * c + 1] = ehi; }
    for (int e = elo + tid; e <= ehi; e += blockDim.x)
        for (int k = 0; k <= d; ++k) {
            double s = 0.0;
            for (int l = 0; l <= d; ++l) {
                const int j = e + d - l;
                if (j >= 0 && j < NE) s += piece[l * (d + 1) + k] * y[j];
            }
            Yc[((size_t)c * cap + (e - elo)) * (d + 1) + k] = s;
        }
}

// Wc[c][m] = W^s[m][cols[c]] = sum_{e in range(c)} sum_k E_{m,e,k} Yc[c][e][k].
// The element row of the table for element q+1 is loaded while element q is
// contracted (the FP64 pipe, not the L2 latency, sets the pace).
template <int D>
__device__ __forceinline__ double wcols_sum(const double* __restrict__ E, int cnt, int den,
                                            const double* __restrict__ sY) {
    constexpr int D1 = D + 1;
    double cur[D1], nxt[D1];
#pragma unroll
    for (int k = 0; k < D1; ++k) cur[k] = E[k];
    double acc = 0.0;
    for (int q = 0; q < cnt; ++q) {
        E -= (size_t)den * D1;
        if (q + 1 < cnt) {
#pragma unroll
            for (int k = 0; k < D1; ++k) nxt[k] = E[k];
        }
#pragma unroll
        for (int k = 0; k < D1; ++k) acc += cur[k] * sY[q * D1 + k];
#pragma unroll
        for (int k = 0; k < D1; ++k) cur[k] = nxt[k];
    }
    return acc;
}

__global__ void __launch_bounds__(256) k_wcols(int Nq, int d, int den, int dmin, int cap, const int* __restrict__ pos,
                                               const double* __restrict__ Et, const int* __restrict__ erange,
                                               const double* __restrict__ Yc, double* __restrict__ Wc) {
    extern __shared__ double sY[];
    const int c = blockIdx.y;
    const int elo = erange[2 * c], cnt = erange[2 * c + 1] - elo + 1;
    const int D1 = d + 1;
    for (int t = threadIdx.x; t < cnt * D1; t += blockDim.x) sY[t] = Yc[(size_t)c * cap * D1 + t];
    __syncthreads();
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Nq) return;
    if (cnt <= 0) {
        Wc[(size_t)c * Nq + m] = 0.0;
        return;
    }
    const double* E = Et + (size_t)(pos[m] - elo * den - dmin) * D1;
    double acc;
    switch (d) {
        case 2: acc = wcols_sum<2>(E, cnt, den, sY); break;
        case 3: acc = wcols_sum<3>(E, cnt, den, sY); break;
        case 4: acc = wcols_sum<4>(E, cnt, den, sY); break;
        default: acc = wcols_sum<5>(E, cnt, den, sY); break;
    }
    Wc[(size_t)c * Nq + m] = acc;
}

// Boundary rows: WsRow[r][m'] = sum_r' B-bar_{e+r'}(eta_m') z_r[e+r'], e = fspan[m'].
__global__ void k_wrows(int Nq, int d, int nrow, const int* __restrict__ fspan, const double* __restrict__ Bf,
                        const double* __restrict__ Z, double* __restrict__ Wr) {
    const int r = blockIdx.y;
    const int mp = blockIdx.x * blockDim.x + threadIdx.x;
    if (mp >= Nq) return;
    const int e = fspan[mp];
    double s = 0.0;
    for (int q = 0; q <= d; ++q) s += Bf[mp * (d + 1) + q] * Z[(size_t)(e + q) * nrow + r];
    Wr[(size_t)r * Nq + mp] = s;
}

// Interior Toeplitz sequences from the two left anchor columns (node indices
// aL0 = B and aL1 = B + 1): T[p][delta + Nq - 1] = W^s[m][m'] for interior m'
// of parity p = (m' - B) & 1 and m - m' = delta.  delta >= 0 reads the anchor
// of parity p directly; delta < 0 reads it through the centrosymmetry
// W^s[m][m'] = W^s[Nq-1-m][Nq-1-m'], where the reflected column Nq-1-m' has
// parity (Nq - 1 - p) & 1.
__global__ void k_toeplitz(int Nq, int R, int aL0, int aL1, const double* __restrict__ WcL0,
                           const double* __restrict__ WcL1, double* __restrict__ T) {
    const size_t len = 2 * (size_t)Nq - 1;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2 * len) return;
    const int p = int(idx / len);
    const int delta = int(idx % len) - (Nq - 1);
    const int q = (delta >= 0) ? p : ((Nq - 1 - p) & 1);
    const int m = (q ? aL1 : aL0) + (delta >= 0 ? delta : -delta);
    T[idx] = (m <= Nq - R - 1) ? (q ? WcL1 : WcL0)[m] : 0.0;
}

// Right-end boundary columns (or rows) from the left-end ones.  The nodes, the
// knots and ln|u - v| are symmetric under u -> a + b - u, so W^s is
// centrosymmetric: W^s[m][m'] = W^s[Nq-1-m][Nq-1-m'].  dst has 2K rows of
// length Nq; rows c0 .. 2K-1 are written, dst[c] = src[c] for c < K and
// dst[c][m] = src[2K-1-c][Nq-1-m] for c >= K.  With c0 = K, src may be dst.
__global__ void k_mirror(int Nq, int K, int c0, const double* src, double* dst) {
    const int c = c0 + blockIdx.y;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Nq) return;
    dst[(size_t)c * Nq + m] = (c < K) ? src[(size_t)c * Nq + m] : src[(size_t)(2 * K - 1 - c) * Nq + (Nq - 1 - m)];
}

__global__ void k_to_f32(size_t count, const double* __restrict__ x, float* __restrict__ y) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) y[i] = (float)x[i];
}

// Dense expansion for diagnostics: Ws[m][m'] = W^s[m][m'].
__global__ void k_ws_expand(WsView<double> v, double* __restrict__ Ws) {
    const int mp = blockIdx.x * blockDim.x + threadIdx.x, m = blockIdx.y;
    if (mp >= v.Nq) return;
    Ws[(size_t)m * v.Nq + mp] = ws_at(v, m, mp);
}

void ws_expand(igs_prob p, double* d_out) {
    const int Nq = p->plan.Nq;
    WsView<double> v{p->d_WsT, p->d_WsRow, p->d_WsToe, Nq, p->ws_B, p->ws_R};
    k_ws_expand<<<dim3((Nq + 255) / 256, Nq), 256, 0, p->geom->ctx->stream>>>(v, d_out);
    IGS_CUDA(cudaGetLastError());
}

// Boundary columns kept explicitly at each end: the columns' departure from
// the interior shift pattern falls below 3e-13 of max|W^s| within 66, 88, 114
// and 134 nodes for d = 2..5 (independent of N_ref); 24(d+1)+16 leaves margin.
static int ws_boundary_columns(int d) { return 24 * (d + 1) + 16; }

// ------------------------------------------------------------------ driver
static void upload_gauss() {
    // once per device; concurrent first calls (serving threads) are serialised
    static std::mutex mu;
    static std::set<int> done;
    int dev = 0;
    IGS_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (done.count(dev)) return;
    double gx[6][6] = {}, gw[6][6] = {};
    for (int g = 1; g <= 6; ++g) {
        // Golub-Welsch free: Newton on Legendre polynomials
        for (int k = 0; k < g; ++k) {
            double x = cos(kPi * (k + 0.75) / (g + 0.5));
            for (int it = 0; it < 100; ++it) {
                double p0 = 1, p1 = x;
                for (int q = 2; q <= g; ++q) { double p2 = ((2 * q - 1) * x * p1 - (q - 1) * p0) / q; p0 = p1; p1 = p2; }
                double pn = (g == 1) ? x : p1, pm = (g == 1) ? 1 : p0;
                double dp = g * (x * pn - pm) / (x * x - 1);
                double dx = pn / dp;
                x -= dx;
                if (fabs(dx) < 1e-16) break;
            }
            double p0 = 1, p1 = x;
            for (int q = 2; q <= g; ++q) { double p2 = ((2 * q - 1) * x * p1 - (q - 1) * p0) / q; p0 = p1; p1 = p2; }
            double pn = (g == 1) ? x : p1, pm = (g == 1) ? 1 : p0;
            double dp = g * (x * pn - pm) / (x * x - 1);
            gx[g - 1][k] = (1.0 - x) / 2.0;
            gw[g - 1][k] = 1.0 / ((1 - x * x) * dp * dp);      // 2/((1-x^2)P'^2) / 2
        }
    }
    IGS_CUDA(cudaMemcpyToSymbol(c_gauss_x, gx, sizeof(gx)));
    IGS_CUDA(cudaMemcpyToSymbol(c_gauss_w, gw, sizeof(gw)));
    done.insert(dev);
}

void rules_build(igs_prob p) {
    const Plan& P = p->plan;
    cudaStream_t s = p->geom->ctx->stream;
    const int d = P.d, Nq = P.Nq, NE = P.NE, n = P.n, D1 = d + 1;
    upload_gauss();
    cudaEvent_t e0, e1;
    IGS_CUDA(cudaEventCreate(&e0));
    IGS_CUDA(cudaEventCreate(&e1));
    IGS_CUDA(cudaEventRecord(e0, s));
    int launches = 0;

    p->d_eta = (double*)dev_alloc(p, sizeof(double) * Nq);
    p->d_Bf = (double*)dev_alloc(p, sizeof(double) * Nq * D1);
    p->d_Bt = (double*)dev_alloc(p, sizeof(double) * Nq * D1);
    p->d_W = (double*)dev_alloc(p, sizeof(double) * Nq * D1);
    p->d_G = (double*)dev_alloc(p, sizeof(double) * NE * D1);
    double* d_L = (double*)dev_alloc(p, sizeof(double) * NE * D1);
    IGS_CUDA(cudaMemsetAsync(d_L, 0, sizeof(double) * NE * D1, s));    // band entries left of column 0 stay 0
    IGS_CUDA(cudaMemsetAsync(p->d_W, 0, sizeof(double) * Nq * D1, s));
    IGS_CUDA(cudaMemsetAsync(p->d_flag, 0, sizeof(int), s));

    // test knot vector
    std::vector<double> tk;
    if (P.closed) {
        for (int k = 0; k <= P.Nh + 2 * d; ++k) tk.push_back(P.a + P.h * (k - d));
    } else {
        for (int k = 0; k < d; ++k) tk.push_back(P.a);
        for (int k = 0; k <= P.Nh; ++k) tk.push_back(k == P.Nh ? P.b : P.a + P.h * k);
        for (int k = 0; k < d; ++k) tk.push_back(P.b);
    }
    double* d_tk = (double*)dev_alloc(p, sizeof(double) * tk.size());
    IGS_CUDA(cudaMemcpyAsync(d_tk, tk.data(), sizeof(double) * tk.size(), cudaMemcpyHostToDevice, s));
    const int ntb = int(tk.size()) - d - 1;

    k_nodes_bands<<<(Nq + 127) / 128, 128, 0, s>>>(Nq, d, P.den, P.Nref, P.M, P.closed, P.a, P.b, P.hf, p->d_pos,
                                                   p->d_jfirst, p->d_member, p->d_fspan, p->d_piece, d_tk, ntb,
                                                   p->d_eta, p->d_Bf, p->d_Bt);
    ++launches;
    k_regular<<<(n + 63) / 64, 64, 0, s>>>(n, Nq, d, P.Nref, P.M, P.closed, P.a, P.hf, p->d_lo, p->d_hi, p->d_jr,
                                           p->d_jfirst, p->d_fspan, p->d_Bf, p->d_piece, d_tk, ntb, p->d_W, p->d_flag);
    ++launches;
    k_gram<<<(NE + 127) / 128, 128, 0, s>>>(NE, d, p->d_gfirst, p->d_glast, p->d_fspan, p->d_Bf, p->d_G);
    ++launches;
    k_chol_band<<<1, 256, 0, s>>>(NE, d, p->d_G, d_L, p->d_flag);
    ++launches;
    double* d_rd = (double*)dev_alloc(p, sizeof(double) * NE);
    k_recip_diag<<<(NE + 255) / 256, 256, 0, s>>>(NE, d, d_L, d_rd);
    ++launches;
    IGS_CUDA(cudaGetLastError());

    // element-moment table over all node/element offsets
    const int den = P.den, M = P.M;
    const int dmin = -(M - 1) * den;
    const int ntab = (2 * M - 1) * den + 1;
    double* d_Et = (double*)dev_alloc(p, sizeof(double) * (size_t)ntab * D1);
    k_etable<<<(ntab + 127) / 128, 128, 0, s>>>(ntab, dmin, d, den, M, P.closed, P.hf, P.L, p->d_series, d_Et);
    ++launches;

    const bool mixed = p->precision == IGS_MIXED;
    const int B = ws_boundary_columns(d), R = d + 2;
    if (Nq < 2 * B + 2 * R + 64) {
        // dense: Z = G^{-1} Mu^T, column m' of W^s for every node
        p->ws_B = Nq;
        p->ws_R = 0;
        p->d_Z = (double*)dev_alloc(p, sizeof(double) * (size_t)NE * Nq);
        k_mu_tab<<<dim3((NE + 127) / 128, Nq), 128, 0, s>>>(NE, M, d, den, dmin, p->d_pos, nullptr, p->d_piece, d_Et,
                                                           p->d_Z, Nq);
        ++launches;
        k_gsolve<<<(Nq + 127) / 128, 128, 0, s>>>(NE, d, Nq, d_L, d_rd, p->d_Z, Nq);
        ++launches;
        p->d_WsT = (double*)dev_alloc(p, sizeof(double) * (size_t)Nq * Nq);
        if (mixed) p->d_WsT32 = (float*)dev_alloc(p, sizeof(float) * (size_t)Nq * Nq);
        k_ws<<<dim3((Nq + 255) / 256, Nq), 256, 0, s>>>(Nq, d, p->d_fspan, p->d_Bf, p->d_Z, Nq, p->d_WsT,
                                                       p->d_WsT32);
        ++launches;
        IGS_CUDA(cudaGetLastError());
    } else {
        // compressed: B boundary columns and R boundary rows at the left end,
        // two interior anchor columns (one per node parity); the right end
        // follows by centrosymmetry
        p->ws_B = B;
        p->ws_R = R;
        const int ncols = B + 2;
        std::vector<int> cols(ncols);
        for (int c = 0; c < ncols; ++c) cols[c] = c;
        int* d_cols = (int*)dev_alloc(p, sizeof(int) * ncols);
        IGS_CUDA(cudaMemcpyAsync(d_cols, cols.data(), sizeof(int) * ncols, cudaMemcpyHostToDevice, s));
        double* d_Y = (double*)dev_alloc(p, sizeof(double) * (size_t)ncols * NE);
        IGS_CUDA(cudaMemsetAsync(d_Y, 0, sizeof(double) * (size_t)ncols * NE, s));
        k_ycols<<<(ncols + 63) / 64, 64, 0, s>>>(ncols, NE, d, d_cols, p->d_fspan, p->d_Bf, d_L, d_rd, d_Y);
        ++launches;
        const int cap = std::min(M, 1024);
        int* d_er = (int*)dev_alloc(p, sizeof(int) * 2 * ncols);
        double* d_Yc = (double*)dev_alloc(p, sizeof(double) * (size_t)ncols * cap * D1);
        k_yc<<<ncols, 128, 0, s>>>(NE, M, d, cap, d_Y, p->d_piece, d_er, d_Yc, p->d_flag);
        ++launches;
        double* d_Wc = (double*)dev_alloc(p, sizeof(double) * (size_t)ncols * Nq);
        const size_t ysm = sizeof(double) * (size_t)cap * D1;
        ensure_dyn_smem((const void*)k_wcols, (size_t)ysm);
        k_wcols<<<dim3((Nq + 255) / 256, ncols), 256, ysm, s>>>(Nq, d, den, dmin, cap, p->d_pos, d_Et, d_er, d_Yc,
                                                               d_Wc);
        ++launches;
        // boundary rows: full rules at the first R nodes, mirrored to the last R
        std::vector<int> rows(R);
        for (int r = 0; r < R; ++r) rows[r] = r;
        int* d_rows = (int*)dev_alloc(p, sizeof(int) * R);
        IGS_CUDA(cudaMemcpyAsync(d_rows, rows.data(), sizeof(int) * R, cudaMemcpyHostToDevice, s));
        double* d_Zr = (double*)dev_alloc(p, sizeof(double) * (size_t)NE * R);
        k_mu_tab<<<dim3((NE + 127) / 128, R), 128, 0, s>>>(NE, M, d, den, dmin, p->d_pos, d_rows, p->d_piece, d_Et,
                                                          d_Zr, R);
        if (NE >= 2 * kPart) {
            part_gsolve(p, s, NE, d, R, d_L, d_rd, d_Zr, R, launches);
        } else {
            k_gsolve<<<1, R, 0, s>>>(NE, d, R, d_L, d_rd, d_Zr, R);
            ++launches;
        }
        p->d_WsRow = (double*)dev_alloc(p, sizeof(double) * (size_t)2 * R * Nq);
        k_wrows<<<dim3((Nq + 255) / 256, R), 256, 0, s>>>(Nq, d, R, p->d_fspan, p->d_Bf, d_Zr, p->d_WsRow);
        k_mirror<<<dim3((Nq + 255) / 256, R), 256, 0, s>>>(Nq, R, R, p->d_WsRow, p->d_WsRow);
        launches += 3;
        // boundary columns at both ends and the Toeplitz sequences
        p->d_WsT = (double*)dev_alloc(p, sizeof(double) * (size_t)2 * B * Nq);
        k_mirror<<<dim3((Nq + 255) / 256, 2 * B), 256, 0, s>>>(Nq, B, 0, d_Wc, p->d_WsT);
        const size_t tlen = 2 * (2 * (size_t)Nq - 1);
        p->d_WsToe = (double*)dev_alloc(p, sizeof(double) * tlen);
        k_toeplitz<<<(unsigned)((tlen + 255) / 256), 256, 0, s>>>(Nq, R, B, B + 1, d_Wc + (size_t)B * Nq,
                                                                   d_Wc + (size_t)(B + 1) * Nq, p->d_WsToe);
        launches += 2;
        if (mixed) {
            const size_t nc = (size_t)2 * B * Nq, nr = (size_t)2 * R * Nq;
            p->d_WsT32 = (float*)dev_alloc(p, sizeof(float) * nc);
            p->d_WsRow32 = (float*)dev_alloc(p, sizeof(float) * nr);
            p->d_WsToe32 = (float*)dev_alloc(p, sizeof(float) * tlen);
            k_to_f32<<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(nc, p->d_WsT, p->d_WsT32);
            k_to_f32<<<(unsigned)((nr + 255) / 256), 256, 0, s>>>(nr, p->d_WsRow, p->d_WsRow32);
            k_to_f32<<<(unsigned)((tlen + 255) / 256), 256, 0, s>>>(tlen, p->d_WsToe, p->d_WsToe32);
            launches += 3;
        }
        IGS_CUDA(cudaGetLastError());
        dev_free(p, d_cols);
        dev_free(p, d_Y);
        dev_free(p, d_er);
        dev_free(p, d_Yc);
        dev_free(p, d_Wc);
        dev_free(p, d_rows);
        dev_free(p, d_Zr);
    }
    dev_free(p, d_Et);

    int flag = 0;
    IGS_CUDA(cudaMemcpyAsync(&flag, p->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    IGS_CUDA(cudaEventRecord(e1, s));
    IGS_CUDA(cudaStreamSynchronize(s));
    float ms = 0;
    IGS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (p->d_Z) dev_free(p, p->d_Z);
    dev_free(p, d_L);
    dev_free(p, d_rd);
    dev_free(p, d_tk);
    p->timing.rules_ms = ms;
    p->launches += launches;
    if (flag) throw Error(IGS_E_INVALID_ARG, "rule construction failed (flag " + std::to_string(flag) + ")");
    p->rules_ready = 1;
}

}  // namespace igs
