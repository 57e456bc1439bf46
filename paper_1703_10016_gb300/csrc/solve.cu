// Solve (A + A^T)/2 alpha = beta (eq. sistlin; A is SPD in the continuous
// setting, symmetric only up to quadrature error in the discrete one).
//
// FP64 tier: blocked right-looking Cholesky in FP64 and two triangular solves.
// MIXED tier: the same factorisation in FP32, then iterative refinement with
// FP64 residuals r = beta - A_s alpha until ||r|| <= 1e-10 ||beta||.
// The factor L is stored in the lower triangle of F and mirrored to the upper
// triangle (U = L^T) so that both substitutions read contiguous rows.
#include <cmath>

#include "igs_internal.h"

namespace igs {

constexpr int kNB = 64;      // Cholesky panel width
constexpr int kTB = 32;      // triangular-solve block

template <typename T>
__global__ void k_symmetrize(int n, const T* __restrict__ A, T* __restrict__ F, double* __restrict__ As64) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
    if (j >= n) return;
    const double v = 0.5 * ((double)A[(size_t)i * n + j] + (double)A[(size_t)j * n + i]);
    F[(size_t)i * n + j] = (T)v;
    if (As64) As64[(size_t)i * n + j] = v;
}

// Unblocked Cholesky of the kb x kb diagonal block at (k0, k0), one CTA.
template <typename T>
__global__ void __launch_bounds__(256) k_potrf(int n, T* __restrict__ F, int k0, int kb, int* __restrict__ flag) {
    __shared__ T a[kNB][kNB + 1];
    for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
        const int i = idx / kb, l = idx % kb;
        a[i][l] = (l <= i) ? F[(size_t)(k0 + i) * n + k0 + l] : (T)0;
    }
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
        if (threadIdx.x == 0) {
            const T dj = a[j][j];
            if (!(dj > (T)0)) { atomicOr(flag, 1); a[j][j] = (T)1; }
            else a[j][j] = sqrt(dj);
        }
        __syncthreads();
        const T dj = a[j][j];
        for (int i = j + 1 + threadIdx.x; i < kb; i += blockDim.x) a[i][j] /= dj;
        __syncthreads();
        const int rem = kb - j - 1;
        for (int idx = threadIdx.x; idx < rem * rem; idx += blockDim.x) {
            const int i = j + 1 + idx / rem, l = j + 1 + idx % rem;
            if (l <= i) a[i][l] -= a[i][j] * a[l][j];
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
        const int i = idx / kb, l = idx % kb;
        if (l <= i) F[(size_t)(k0 + i) * n + k0 + l] = a[i][l];
    }
}

// Panel: F[i, k0:k0+kb] <- F[i, k0:k0+kb] L11^{-T} for rows i >= k0+kb (64 rows per CTA).
template <typename T>
__global__ void __launch_bounds__(64) k_trsm(int n, T* __restrict__ F, int k0, int kb) {
    __shared__ T L11[kNB][kNB + 1];
    __shared__ T X[64][kNB + 1];
    const int r0 = k0 + kb + blockIdx.x * 64;
    for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
        const int i = idx / kb, l = idx % kb;
        L11[i][l] = (l <= i) ? F[(size_t)(k0 + i) * n + k0 + l] : (T)0;
    }
    for (int idx = threadIdx.x; idx < 64 * kb; idx += blockDim.x) {
        const int rr = idx / kb, c = idx % kb;
        X[rr][c] = (r0 + rr < n) ? F[(size_t)(r0 + rr) * n + k0 + c] : (T)0;
    }
    __syncthreads();
    const int rr = threadIdx.x;
    if (r0 + rr < n) {
        for (int c = 0; c < kb; ++c) {
            T s = X[rr][c];
            for (int l = 0; l < c; ++l) s -= X[rr][l] * L11[c][l];
            X[rr][c] = s / L11[c][c];
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 64 * kb; idx += blockDim.x) {
        const int r = idx / kb, c = idx % kb;
        if (r0 + r < n) F[(size_t)(r0 + r) * n + k0 + c] = X[r][c];
    }
}

// Trailing update of the lower triangle: F[i][j] -= sum_l F[i][k0+l] F[j][k0+l],
// 64 x 64 tiles, 256 threads with 4 x 4 outputs each.
template <typename T>
__global__ void __launch_bounds__(256) k_syrk(int n, T* __restrict__ F, int k0, int kb) {
    const int ti = blockIdx.y, tj = blockIdx.x;
    if (tj > ti) return;
    const int base = k0 + kb;
    const int i0 = base + ti * 64, j0 = base + tj * 64;
    __shared__ T As[64][kNB + 1], Bs[64][kNB + 1];
    for (int idx = threadIdx.x; idx < 64 * kb; idx += blockDim.x) {
        const int r = idx / kb, l = idx % kb;
        As[r][l] = (i0 + r < n) ? F[(size_t)(i0 + r) * n + k0 + l] : (T)0;
        Bs[r][l] = (j0 + r < n) ? F[(size_t)(j0 + r) * n + k0 + l] : (T)0;
    }
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    T acc[4][4] = {};
    for (int l = 0; l < kb; ++l) {
        T av[4], bv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) { av[q] = As[ty + 16 * q][l]; bv[q] = Bs[tx + 16 * q][l]; }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] += av[r] * bv[c];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int i = i0 + ty + 16 * r, j = j0 + tx + 16 * c;
            if (i < n && j < n && j <= i) F[(size_t)i * n + j] -= acc[r][c];
        }
}

template <typename T>
__global__ void k_mirror(int n, T* __restrict__ F) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
    if (j < i) F[(size_t)j * n + i] = F[(size_t)i * n + j];
}

// Forward (lower=1: L y = b) or backward (lower=0: U x = y, U = L^T in the upper
// triangle) substitution for nrhs vectors, one CTA of 1024 threads; X holds b
// on entry and the solution on exit (X[k*n + i]).
template <typename T>
__global__ void __launch_bounds__(1024) k_trsv(int n, const T* __restrict__ F, T* __restrict__ X, int nrhs, int lower) {
    __shared__ T xb[8][kTB];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int nblk = (n + kTB - 1) / kTB;
    for (int bb = 0; bb < nblk; ++bb) {
        const int blk = lower ? bb : nblk - 1 - bb;
        const int b0 = blk * kTB, bn = min(kTB, n - b0);
        // 1. update: X[b0+w] -= sum over solved columns (warp w owns row b0+w, lanes stride columns)
        const int c_lo = lower ? 0 : b0 + bn, c_hi = lower ? b0 : n;
        if (warp < bn) {
            const int row = b0 + warp;
            T part[8];
            for (int k = 0; k < nrhs; ++k) part[k] = (T)0;
            for (int c = c_lo + lane; c < c_hi; c += 32) {
                const T f = F[(size_t)row * n + c];
                for (int k = 0; k < nrhs; ++k) part[k] += f * X[(size_t)k * n + c];
            }
            for (int k = 0; k < nrhs; ++k) {
                T v = part[k];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) xb[k][warp] = X[(size_t)k * n + row] - v;
            }
        }
        __syncthreads();
        // 2. triangular block solve (warp k handles right-hand side k)
        if (warp < nrhs) {
            const int k = warp;
            T xv = (lane < bn) ? xb[k][lane] : (T)0;
            for (int q = 0; q < bn; ++q) {
                const int c = lower ? q : bn - 1 - q;
                const int row = b0 + c;
                const T diag = F[(size_t)row * n + row];
                T xc = __shfl_sync(0xffffffffu, xv, c) / diag;
                if (lane == c) xv = xc;
                // eliminate from the not-yet-solved rows of the block
                const bool pending = lower ? (lane > c && lane < bn) : (lane < c);
                if (pending) xv -= F[(size_t)(b0 + lane) * n + row] * xc;
            }
            if (lane < bn) X[(size_t)k * n + b0 + lane] = xv;
        }
        __syncthreads();
    }
}

// r = beta - As alpha (FP64), one warp per row; also |r|^2 and |beta|^2 per rhs.
__global__ void k_resid(int n, int nrhs, const double* __restrict__ As, const double* __restrict__ alpha,
                        const double* __restrict__ beta, double* __restrict__ r, double* __restrict__ norms) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
    if (warp >= n) return;
    const int i = warp;
    double s[8];
    for (int k = 0; k < nrhs; ++k) s[k] = 0.0;
    for (int j = lane; j < n; j += 32) {
        const double a = As[(size_t)i * n + j];
        for (int k = 0; k < nrhs; ++k) s[k] += a * alpha[(size_t)k * n + j];
    }
    for (int k = 0; k < nrhs; ++k) {
        double v = s[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) {
            const double rv = beta[(size_t)k * n + i] - v;
            r[(size_t)k * n + i] = rv;
            atomicAdd(&norms[2 * k], rv * rv);
            atomicAdd(&norms[2 * k + 1], beta[(size_t)k * n + i] * beta[(size_t)k * n + i]);
        }
    }
}

template <typename T>
__global__ void k_cast_in(int cnt, const double* __restrict__ src, T* __restrict__ dst, const double* __restrict__ scale,
                          int n) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cnt) return;
    const double sc = scale ? scale[2 * (q / n)] : 0.0;
    const double inv = (sc > 0) ? 1.0 / sqrt(sc) : 1.0;
    dst[q] = (T)(src[q] * inv);
}

template <typename T>
__global__ void k_accum(int cnt, const T* __restrict__ dx, double* __restrict__ x, const double* __restrict__ scale,
                        int n, int first) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cnt) return;
    const double sc = scale ? scale[2 * (q / n)] : 0.0;
    const double f = (sc > 0) ? sqrt(sc) : 1.0;
    const double v = (double)dx[q] * f;
    x[q] = first ? v : x[q] + v;
}

template <typename T>
static void factor(igs_prob p, cudaStream_t s) {
    const int n = p->plan.n;
    T* F = (T*)p->d_F;
    IGS_CUDA(cudaMemsetAsync(p->d_flag, 0, sizeof(int), s));
    for (int k0 = 0; k0 < n; k0 += kNB) {
        const int kb = std::min(kNB, n - k0);
        k_potrf<T><<<1, 256, 0, s>>>(n, F, k0, kb, p->d_flag);
        const int rem = n - k0 - kb;
        if (rem > 0) {
            k_trsm<T><<<(rem + 63) / 64, 64, 0, s>>>(n, F, k0, kb);
            const int nt = (rem + 63) / 64;
            k_syrk<T><<<dim3(nt, nt), 256, 0, s>>>(n, F, k0, kb);
            p->launches += 2;
        }
        p->launches++;
    }
    k_mirror<T><<<dim3((n + 255) / 256, n), 256, 0, s>>>(n, F);
    p->launches++;
    IGS_CUDA(cudaGetLastError());
    int flag = 0;
    IGS_CUDA(cudaMemcpyAsync(&flag, p->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    IGS_CUDA(cudaStreamSynchronize(s));
    if (flag) throw Error(IGS_E_NOT_SPD, "Cholesky met a non-positive pivot");
}

template <typename T>
static void prepare_factor(igs_prob p, cudaStream_t s) {
    const int n = p->plan.n;
    if (!p->d_F) p->d_F = dev_alloc(p, sizeof(T) * (size_t)n * n);
    if (!p->d_As64) p->d_As64 = (double*)dev_alloc(p, sizeof(double) * (size_t)n * n);
    k_symmetrize<T><<<dim3((n + 255) / 256, n), 256, 0, s>>>(n, (const T*)p->d_A, (T*)p->d_F, p->d_As64);
    p->launches++;
    IGS_CUDA(cudaGetLastError());
    factor<T>(p, s);
    p->factored = 1;
}

template <typename T>
static void refine(igs_prob p, double* d_beta, int nrhs, double* d_alpha, double* resid, cudaStream_t s, int max_it,
                   double tol) {
    const int n = p->plan.n;
    const int cnt = n * nrhs;
    T* d_x = (T*)dev_alloc(p, sizeof(T) * cnt);
    double* d_r = (double*)dev_alloc(p, sizeof(double) * cnt);
    double* d_norm = (double*)dev_alloc(p, sizeof(double) * 2 * nrhs);
    std::vector<double> hn(2 * nrhs);
    int it = 0;
    const double* src = d_beta;
    const double* scale = nullptr;
    for (;;) {
        k_cast_in<T><<<(cnt + 255) / 256, 256, 0, s>>>(cnt, src, d_x, scale, n);
        k_trsv<T><<<1, 1024, 0, s>>>(n, (const T*)p->d_F, d_x, nrhs, 1);
        k_trsv<T><<<1, 1024, 0, s>>>(n, (const T*)p->d_F, d_x, nrhs, 0);
        k_accum<T><<<(cnt + 255) / 256, 256, 0, s>>>(cnt, d_x, d_alpha, scale, n, it == 0);
        IGS_CUDA(cudaMemsetAsync(d_norm, 0, sizeof(double) * 2 * nrhs, s));
        k_resid<<<(n * 32 + 255) / 256, 256, 0, s>>>(n, nrhs, p->d_As64, d_alpha, d_beta, d_r, d_norm);
        p->launches += 5;
        IGS_CUDA(cudaGetLastError());
        IGS_CUDA(cudaMemcpyAsync(hn.data(), d_norm, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, s));
        IGS_CUDA(cudaStreamSynchronize(s));
        ++it;
        double worst = 0;
        for (int k = 0; k < nrhs; ++k) {
            const double rel = hn[2 * k + 1] > 0 ? std::sqrt(hn[2 * k] / hn[2 * k + 1]) : std::sqrt(hn[2 * k]);
            if (resid) resid[k] = rel;
            worst = std::max(worst, rel);
        }
        if (worst <= tol || it >= max_it) break;
        src = d_r;
        scale = d_norm;
    }
    p->timing.ir_iterations = it;
    dev_free(p, d_x);
    dev_free(p, d_r);
    dev_free(p, d_norm);
    double worst = 0;
    for (int k = 0; k < nrhs; ++k) worst = std::max(worst, hn[2 * k + 1] > 0 ? std::sqrt(hn[2 * k] / hn[2 * k + 1]) : 0.0);
    if (worst > tol && max_it > 1) throw Error(IGS_E_NOT_CONVERGED, "iterative refinement did not reach 1e-10");
}

void solve_system(igs_prob p, double* d_beta, int nrhs, double* d_alpha, double* resid) {
    cudaStream_t s = p->geom->ctx->stream;
    if (nrhs < 1 || nrhs > 8) throw Error(IGS_E_INVALID_ARG, "nrhs must be in [1, 8]");
    cudaEvent_t e0, e1, e2;
    IGS_CUDA(cudaEventCreate(&e0)); IGS_CUDA(cudaEventCreate(&e1)); IGS_CUDA(cudaEventCreate(&e2));
    IGS_CUDA(cudaEventRecord(e0, s));
    const bool mixed = p->precision == IGS_MIXED;
    if (!p->factored) {
        if (mixed) prepare_factor<float>(p, s);
        else prepare_factor<double>(p, s);
    }
    IGS_CUDA(cudaEventRecord(e1, s));
    if (mixed) refine<float>(p, d_beta, nrhs, d_alpha, resid, s, 30, 1e-10);
    else refine<double>(p, d_beta, nrhs, d_alpha, resid, s, 1, 1e-10);
    IGS_CUDA(cudaEventRecord(e2, s));
    IGS_CUDA(cudaEventSynchronize(e2));
    float f_ms = 0, s_ms = 0;
    cudaEventElapsedTime(&f_ms, e0, e1);
    cudaEventElapsedTime(&s_ms, e1, e2);
    p->timing.factor_ms = f_ms;
    p->timing.solve_ms = s_ms;
    cudaEventDestroy(e0); cudaEventDestroy(e1); cudaEventDestroy(e2);
}

}  // namespace igs
