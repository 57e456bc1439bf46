// Solve (A + A^T)/2 alpha = beta (eq. sistlin; A is SPD in the continuous
// setting, symmetric only up to quadrature error in the discrete one).
//
// Blocked right-looking Cholesky with 64-wide panels, one graph-captured
// launch sequence per problem:
//   k_panel  CTA 0 factors the 64 x 64 diagonal block and stores L11; every
//            other CTA factors the diagonal block stacked on its 64-row slice
//            of the panel, which yields L21 = A21 L11^{-T} for that slice;
//   k_syrk   trailing update of the lower triangle, 64 x 64 tiles; the tile
//            column that holds the next panel goes first, the rest runs on a
//            second captured stream beside the next panel (look-ahead); in the
//            MIXED tier that rest runs on the tensor cores (k_syrk_tc).
// FP64 tier: all in FP64, then one substitution pair.  MIXED tier: the same in
// FP32 on D A_s D with D = diag(A_s)^-1/2 (unit diagonal, every factor entry at
// most 1 in magnitude), then iterative refinement with FP64 residuals
// r = beta - A_s alpha until ||r|| <= 1e-10 ||beta||.  The triangular solves go by 64-row blocks in solve
// order: the inverted diagonal block (computed once per factorisation, in
// parallel), then a rank-64 update of the rows not yet solved.
#include <cuda_fp16.h>

#include <cmath>

#include "igs_internal.h"

namespace igs {

constexpr int kNB = 64;      // Cholesky panel width / triangular-solve block

// Tiles of 64 x 64 over the lower triangle of tile pairs (bi >= bj), CTAs
// numbered over that triangle.
constexpr int kTT = 64;
__device__ __forceinline__ void tri_decode(int t, int& ti, int& tj);

// dscale[i] = 1 / sqrt(A_ii) in FP32: the unit-diagonal scaling D of the MIXED
// tier's factorisation (a non-positive diagonal keeps 1 and the factorisation
// flags it).  The refinement applies the same FP32 values, so the factor is
// that of D As D with D exactly as stored.
__global__ void k_diag_scale(int n, const float* __restrict__ A, float* __restrict__ dscale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float a = A[(size_t)i * n + i];
    dscale[i] = a > 0.0f ? rsqrtf(a) : 1.0f;
}

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int N = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int N = 2; };

template <typename T>
__device__ __forceinline__ T vget(const typename Vec16<T>::type& v, int q);
template <> __device__ __forceinline__ float vget<float>(const float4& v, int q) {
    return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}
template <> __device__ __forceinline__ double vget<double>(const double2& v, int q) { return q == 0 ? v.x : v.y; }

// A^T from A through 32 x 32 shared-memory tiles (for a matrix assembled
// without its transpose, e.g. by the batched form).
template <typename T>
__global__ void __launch_bounds__(256) k_transpose(int n, const T* __restrict__ A, T* __restrict__ AT) {
    __shared__ T t[32][33];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    for (int r = threadIdx.x / 32; r < 32; r += 8) {
        const int i = i0 + r, j = j0 + threadIdx.x % 32;
        if (i < n && j < n) t[r][threadIdx.x % 32] = A[(size_t)i * n + j];
    }
    __syncthreads();
    for (int r = threadIdx.x / 32; r < 32; r += 8) {
        const int i = j0 + r, j = i0 + threadIdx.x % 32;
        if (i < n && j < n) AT[(size_t)i * n + j] = t[threadIdx.x % 32][r];
    }
}

// FP64 tier: As = (A + A^T)/2 from A and A^T (both row-major, written by the
// assembly), one 16-byte vector of each per thread: a streaming kernel, every
// access coalesced.  F gets the lower triangle of As, As64 the whole As (for
// the residual).  Grid (row chunks, rows).
template <typename T>
__global__ void __launch_bounds__(256) k_symmetrize(int n, const T* __restrict__ A, const T* __restrict__ AT,
                                                    T* __restrict__ F, double* __restrict__ As64) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N;
    const int i = blockIdx.y;
    const size_t rowoff = (size_t)i * n;
    if ((n % VN) == 0) {
        const int j = (blockIdx.x * blockDim.x + threadIdx.x) * VN;
        if (j >= n) return;
        const V a = *(const V*)(A + rowoff + j), at = *(const V*)(AT + rowoff + j);
#pragma unroll
        for (int u = 0; u < VN; ++u) {
            const double v = 0.5 * ((double)vget<T>(a, u) + (double)vget<T>(at, u));
            As64[rowoff + j + u] = v;
            if (j + u <= i) F[rowoff + j + u] = (T)v;
        }
    } else {
        for (int u = 0; u < VN; ++u) {
            const int j = (blockIdx.x * blockDim.x + threadIdx.x) * VN + u;
            if (j >= n) return;
            const double v = 0.5 * ((double)A[rowoff + j] + (double)AT[rowoff + j]);
            As64[rowoff + j] = v;
            if (j <= i) F[rowoff + j] = (T)v;
        }
    }
}

// MIXED tier: the lower triangle of D As D, As = (A + A^T)/2, in FP32 from A
// and A^T, four entries per thread (16-byte loads and stores); no FP64
// arithmetic (FP64 runs at 1/64 of the FP32 rate on this GPU).  Grid (column
// chunks of 1024, rows); chunks above the diagonal return at once.
__global__ void __launch_bounds__(256) k_symmetrize_lower_f(int n, const float* __restrict__ A,
                                                            const float* __restrict__ AT, float* __restrict__ F,
                                                            const float* __restrict__ dscale) {
    const int i = blockIdx.y;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (j > i) return;
    const size_t rowoff = (size_t)i * n;
    const float di = 0.5f * dscale[i];
    if ((n & 3) == 0 && j + 3 <= i) {
        const float4 a = *(const float4*)(A + rowoff + j), at = *(const float4*)(AT + rowoff + j);
        const float4 dj = *(const float4*)(dscale + j);
        float4 v;
        v.x = (a.x + at.x) * di * dj.x;
        v.y = (a.y + at.y) * di * dj.y;
        v.z = (a.z + at.z) * di * dj.z;
        v.w = (a.w + at.w) * di * dj.w;
        *(float4*)(F + rowoff + j) = v;
    } else {
        for (int u = 0; u < 4 && j + u <= i && j + u < n; ++u)
            F[rowoff + j + u] = (A[rowoff + j + u] + AT[rowoff + j + u]) * di * dscale[j + u];
    }
}

// Panel step at column k0 (width kb).  CTA 0 factors the 64 x 64 diagonal
// block and stores L11; CTA b >= 1 factors the tall block made of the
// diagonal block and rows k0 + 64 b .. + 63 below it (the diagonal part
// redundantly, so that no CTA waits for another), which turns its rows into
// L21 = A21 L11^{-T}.  Right-looking by 8-column blocks, three barriers per
// block: (1) each row's thread reads the 8 x 8 diagonal sub-block and its row,
// then factors the sub-block itself (every thread the same, in registers: no
// communication) and solves its own row against it; (2) rank-8 update of the
// columns to the right.
// A non-positive pivot sets *flag and is replaced by 1.
// NS > 1 (FP32): each CTA b >= 1 takes 64 NS rows below the diagonal block
// (PARTS threads per row in the update), so that a tall panel runs in fewer
// waves of CTAs.
// FUSE (FP32, kp >= 0): the CTA first applies the previous panel's update to
// its rows of this column block, A[i][k0 + l] -= sum_m L[i][kp + m]
// L[k0 + l][kp + m] (the right-looking update of the next column block, here
// instead of a launch of its own on the panel chain), from the previous
// panel's 64 columns of the same rows staged in shared memory.
__host__ __device__ constexpr int panel_rows(int ns) { return (1 + ns) * 64; }   // diagonal block + slices
__host__ __device__ constexpr int panel_threads(int ns, int parts) { return parts * panel_rows(ns); }
constexpr int kPB = 8;                                     // inner block width

// Programmatic dependent launch: a kernel of the panel chain lets the next
// one be scheduled at once (its CTAs park at the wait) and itself waits for
// its predecessor's completion and memory before touching shared data.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename T> __device__ __forceinline__ T rsqrt_t(T x);
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

template <typename T, int NS, int PARTS, bool FUSE>
__global__ void __launch_bounds__(panel_threads(NS, PARTS)) k_panel(int n, T* __restrict__ F, int k0, int kb, int kp,
                                                                    T* __restrict__ diagL, int* __restrict__ flag) {
    constexpr int kPanelRows = panel_rows(NS), kPanelThreads = panel_threads(NS, PARTS), kPanelParts = PARTS;
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N;
    constexpr int LP = kNB + 16 / (int)sizeof(T);          // row stride of the staged previous panel
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T (*P)[kPB] = (T (*)[kPB])smem_raw;                     // current 8 columns of L, one row of 8 per row
    T (*a)[kNB + 1] = (T (*)[kNB + 1])(P + kPanelRows);    // rows 0..63 diagonal block, then the slice
    T (*Lp)[LP] = (T (*)[LP])(a + kPanelRows);              // FUSE: the same rows of the previous panel
    const int tid = threadIdx.x;
    const int r0 = k0 + kNB + ((int)blockIdx.x - 1) * NS * kNB;
    const int nb = blockIdx.x == 0 ? 0 : min(NS * kNB, n - r0);
    const int rows = kNB + nb;
    const bool fuse = FUSE && kp >= 0;
    // all loads in flight before the first store
    constexpr int kPer = kPanelRows * kNB / kPanelThreads;
    T v[kPer], w[FUSE ? kPer : 1];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int idx = tid + q * kPanelThreads, i = idx / kNB, l = idx % kNB;
        if (i < kNB) {
            if (i < kb && l < kb) v[q] = (l <= i) ? F[(size_t)(k0 + i) * n + k0 + l] : (T)0;
            else v[q] = (i == l) ? (T)1 : (T)0;       // identity padding beyond kb
        } else {
            v[q] = (i < rows) ? F[(size_t)(r0 + i - kNB) * n + k0 + l] : (T)0;
        }
        if (FUSE && fuse) {
            const int row = i < kNB ? (i < kb ? k0 + i : -1) : (i < rows ? r0 + i - kNB : -1);
            w[FUSE ? q : 0] = row >= 0 ? F[(size_t)row * n + kp + l] : (T)0;
        }
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int idx = tid + q * kPanelThreads;
        a[idx / kNB][idx % kNB] = v[q];
        if (FUSE && fuse) Lp[idx / kNB][idx % kNB] = w[FUSE ? q : 0];
    }
    __syncthreads();
    if (FUSE && fuse) {
        // thread (ri, ci): rows ri + RG r (r < RR), columns ci + 16 c (c < 4); a
        // quarter-warp reads eight distinct staged rows (odd stride in 16-byte
        // units) or one row (broadcast)
        constexpr int RG = kPanelThreads / 16, RR = kPanelRows / RG;
        const int ri = tid / 16, ci = tid % 16;
        T acc[RR][4];
#pragma unroll
        for (int r = 0; r < RR; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = (T)0;
#pragma unroll 2
        for (int m0 = 0; m0 < kNB; m0 += VN) {
            V xr[RR], xc[4];
#pragma unroll
            for (int r = 0; r < RR; ++r) xr[r] = *(const V*)&Lp[ri + RG * r][m0];
#pragma unroll
            for (int c = 0; c < 4; ++c) xc[c] = *(const V*)&Lp[ci + 16 * c][m0];
#pragma unroll
            for (int u = 0; u < VN; ++u)
#pragma unroll
                for (int r = 0; r < RR; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] += vget<T>(xr[r], u) * vget<T>(xc[c], u);
        }
#pragma unroll
        for (int r = 0; r < RR; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) a[ri + RG * r][ci + 16 * c] -= acc[r][c];
        __syncthreads();
    }
    const int i = tid % kPanelRows, part = tid / kPanelRows;
#pragma unroll 1
    for (int c0 = 0; c0 < kNB; c0 += kPB) {
        // (1) rows i >= c0: L of the 8 x 8 diagonal sub-block, then this row's 8 entries.
        // Every participating thread reads the sub-block before any of them writes
        // its row back (the rows of the sub-block are among the rows written).
        const bool act = part == 0 && i >= c0 && i < rows;
        T d[kPB][kPB];
        T x[kPB];
        if (act) {
#pragma unroll
            for (int u = 0; u < kPB; ++u)
#pragma unroll
                for (int w = 0; w < kPB; ++w) d[u][w] = (w <= u) ? a[c0 + u][c0 + w] : (T)0;
#pragma unroll
            for (int w = 0; w < kPB; ++w) x[w] = a[i][c0 + w];
        }
        __syncthreads();
        if (act) {
#pragma unroll
            for (int w = 0; w < kPB; ++w) {
                T pv = d[w][w];
                if (!(pv > (T)0)) {
                    if (i == c0) atomicOr(flag, 1);
                    pv = (T)1;
                }
                const T r = rsqrt_t<T>(pv);
                d[w][w] = pv * r;
#pragma unroll
                for (int u = 0; u < kPB; ++u)
                    if (u > w) d[u][w] *= r;
#pragma unroll
                for (int u = 0; u < kPB; ++u)
#pragma unroll
                    for (int z = 0; z < kPB; ++z)
                        if (z > w && z <= u) d[u][z] -= d[u][w] * d[z][w];
                // own row (rows below the sub-block): forward substitution step w
                x[w] *= r;
#pragma unroll
                for (int z = 0; z < kPB; ++z)
                    if (z > w) x[z] -= x[w] * d[z][w];
            }
            // a row inside the sub-block comes out of the same substitution as its
            // row of L (its entries right of the diagonal start at zero): clear those
#pragma unroll
            for (int w = 0; w < kPB; ++w)
                if (i < kNB && c0 + w > i) x[w] = (T)0;
#pragma unroll
            for (int w = 0; w < kPB; ++w) {
                a[i][c0 + w] = x[w];
                P[i][w] = x[w];
            }
        }
        __syncthreads();
        // (2) a[i][l] -= sum_w L[i][c0+w] L[l][c0+w] for c0 + 8 <= l (<= i on the diagonal block)
        if (c0 + kPB < kNB && i >= c0 + kPB && i < rows) {
            V xi[kPB / VN];
#pragma unroll
            for (int q = 0; q < kPB / VN; ++q) xi[q] = *(const V*)&P[i][q * VN];
            const int lmax = i < kNB ? i : kNB - 1;
            // two columns per trip, both loaded before either store
#pragma unroll 1
            for (int l = c0 + kPB + part; l <= lmax; l += 2 * kPanelParts) {
                const int l2 = l + kPanelParts;
                const bool two = l2 <= lmax;
                V p1[kPB / VN], p2[kPB / VN];
#pragma unroll
                for (int q = 0; q < kPB / VN; ++q) {
                    p1[q] = *(const V*)&P[l][q * VN];
                    p2[q] = *(const V*)&P[two ? l2 : l][q * VN];
                }
                T s1 = a[i][l], s2 = a[i][two ? l2 : l];
#pragma unroll
                for (int q = 0; q < kPB / VN; ++q)
#pragma unroll
                    for (int u = 0; u < VN; ++u) {
                        s1 -= vget<T>(xi[q], u) * vget<T>(p1[q], u);
                        s2 -= vget<T>(xi[q], u) * vget<T>(p2[q], u);
                    }
                a[i][l] = s1;
                if (two) a[i][l2] = s2;
            }
        }
        __syncthreads();
    }
    if (blockIdx.x == 0) {
        for (int idx = tid; idx < kb * kNB; idx += kPanelThreads) {
            const int r = idx / kNB, l = idx % kNB;
            diagL[(size_t)(k0 + r) * kNB + l] = (l <= r) ? a[r][l] : (T)0;
        }
        return;
    }
    for (int idx = tid; idx < nb * kNB; idx += kPanelThreads) {
        const int r = idx / kNB, l = idx % kNB;
        F[(size_t)(r0 + r) * n + k0 + l] = a[kNB + r][l];
    }
}

// Trailing update of the lower triangle after panel k0:
// F[i][j] -= sum_l F[i][k0+l] F[j][k0+l] for i >= j >= k0 + kb, 64 x 64 tiles.
// `mode` picks the tiles: 0 all, 1 the first tile column only (the next
// panel's columns, updated first so that the next panel can start), 2 all
// but the first tile column (CTAs numbered over the lower triangle of tiles
// only), 3 the tile columns below gridDim.y, 4 the tile columns 1 ..
// gridDim.y, all rows below.  The panel rows are staged row-major (coalesced 16-byte loads);
// thread (tx, ty) owns rows ty + 16 r and columns tx + 16 c (r, c < 4) and
// reads 16-byte vectors along l (odd row stride in 16-byte units: the
// quarter-warps hit distinct banks).
constexpr int kST = 64;
constexpr int kSTM = kST / 16;       // rows / columns per thread
template <typename T> __host__ __device__ constexpr int syrk_ld() { return kNB + 16 / (int)sizeof(T); }

__device__ __forceinline__ void tri_decode(int t, int& ti, int& tj) {
    int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    while (r * (r + 1) / 2 > t) --r;
    ti = r;
    tj = t - r * (r + 1) / 2;
}

template <typename T>
__global__ void __launch_bounds__(256) k_syrk(int n, T* __restrict__ F, int k0, int kb, int mode) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N;
    constexpr int LD = syrk_ld<T>();
    pdl_wait();
    pdl_trigger();
    int ti, tj;
    if (mode == 1) {
        ti = blockIdx.x;
        tj = 0;
    } else if (mode == 2) {
        tri_decode(blockIdx.x, ti, tj);
        ++ti;
        ++tj;
    } else if (mode == 3) {                       // column tiles blockIdx.y < gridDim.y, all rows below
        ti = blockIdx.x;
        tj = blockIdx.y;
        if (ti < tj) return;
    } else if (mode == 4) {                       // column tiles 1 .. gridDim.y, all rows below
        ti = blockIdx.x;
        tj = blockIdx.y + 1;
        if (ti < tj) return;
    } else {
        tri_decode(blockIdx.x, ti, tj);
    }
    const int base = k0 + kb;
    const int i0 = base + ti * kST, j0 = base + tj * kST;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T (*As)[LD] = (T (*)[LD])smem_raw;
    T (*Bs)[LD] = (ti == tj) ? As : As + kST;
    const bool vec_ok = (n % VN) == 0 && kb == kNB;
    if (vec_ok) {
        constexpr int per_row = kNB / VN;
        for (int idx = threadIdx.x; idx < kST * per_row; idx += blockDim.x) {
            const int rr = idx / per_row, q = idx % per_row;
            V va = V{}, vb = V{};
            if (i0 + rr < n) va = *(const V*)(F + (size_t)(i0 + rr) * n + k0 + q * VN);
            if (ti != tj && j0 + rr < n) vb = *(const V*)(F + (size_t)(j0 + rr) * n + k0 + q * VN);
            *(V*)&As[rr][q * VN] = va;
            if (ti != tj) *(V*)&Bs[rr][q * VN] = vb;
        }
    } else {
        for (int idx = threadIdx.x; idx < kST * kNB; idx += blockDim.x) {
            const int rr = idx / kNB, l = idx % kNB;
            As[rr][l] = (i0 + rr < n && l < kb) ? F[(size_t)(i0 + rr) * n + k0 + l] : (T)0;
            if (ti != tj) Bs[rr][l] = (j0 + rr < n && l < kb) ? F[(size_t)(j0 + rr) * n + k0 + l] : (T)0;
        }
    }
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    T acc[kSTM][kSTM];
#pragma unroll
    for (int r = 0; r < kSTM; ++r)
#pragma unroll
        for (int c = 0; c < kSTM; ++c) acc[r][c] = (T)0;
#pragma unroll 4
    for (int l = 0; l < kNB; l += VN) {
        V av[kSTM], bv[kSTM];
#pragma unroll
        for (int q = 0; q < kSTM; ++q) {
            av[q] = *(const V*)&As[ty + 16 * q][l];
            bv[q] = *(const V*)&Bs[tx + 16 * q][l];
        }
#pragma unroll
        for (int u = 0; u < VN; ++u)
#pragma unroll
            for (int r = 0; r < kSTM; ++r) {
                const T ar = vget<T>(av[r], u);
#pragma unroll
                for (int c = 0; c < kSTM; ++c) acc[r][c] += ar * vget<T>(bv[c], u);
            }
    }
    // epilogue: read every C entry before writing any (all loads in flight at once)
    T cv[kSTM][kSTM];
#pragma unroll
    for (int r = 0; r < kSTM; ++r) {
        const int i = i0 + ty + 16 * r;
#pragma unroll
        for (int c = 0; c < kSTM; ++c) {
            const int j = j0 + tx + 16 * c;
            cv[r][c] = (i < n && j <= i) ? F[(size_t)i * n + j] : (T)0;
        }
    }
#pragma unroll
    for (int r = 0; r < kSTM; ++r) {
        const int i = i0 + ty + 16 * r;
#pragma unroll
        for (int c = 0; c < kSTM; ++c) {
            const int j = j0 + tx + 16 * c;
            if (i < n && j <= i) F[(size_t)i * n + j] = cv[r][c] - acc[r][c];
        }
    }
}

// Diagonal blocks back into F, and U = L^T into the upper triangle: one
// 64 x 64 tile pair per CTA (tiles align with the 64-wide diagonal blocks),
// the lower tile read row by row and written transposed through shared memory.
// Tile columns bj0 .. bj0 + w - 1 (w > 0: grid x over the tile rows from the
// diagonal down, y over the columns) or all from bj0 on (w = 0: CTAs numbered
// over that lower triangle of tiles).
template <typename T>
__global__ void __launch_bounds__(256) k_finalize(int n, T* __restrict__ F, const T* __restrict__ diagL, int bj0,
                                                  int w) {
    __shared__ T t[kTT][kTT + 1];
    int bi, bj;
    if (w > 0) {
        bj = bj0 + (int)blockIdx.y;
        bi = bj + (int)blockIdx.x;
        if (bi >= (n + kTT - 1) / kTT) return;
    } else {
        tri_decode(blockIdx.x, bi, bj);
        bi += bj0;
        bj += bj0;
    }
    const int i0 = bi * kTT, j0 = bj * kTT;
    const int c = threadIdx.x % kTT, r4 = threadIdx.x / kTT;
    for (int r = r4; r < kTT; r += 4) {
        const int i = i0 + r, j = j0 + c;
        T v = (T)0;
        if (i < n && j < n && j <= i) {
            v = (bi == bj) ? diagL[(size_t)i * kNB + c] : F[(size_t)i * n + j];
            if (bi == bj) F[(size_t)i * n + j] = v;
        }
        t[r][c] = v;
    }
    __syncthreads();
    for (int r = r4; r < kTT; r += 4) {                      // F[j0 + r][i0 + c] = L[i0 + c][j0 + r]
        const int i = j0 + r, j = i0 + c;
        if (i < n && j < n && j > i) F[(size_t)i * n + j] = t[c][r];
    }
}

// Inverses of the 64 x 64 diagonal blocks of L (one CTA per block, after the
// factorisation, off the panel critical path): li[i][c] = -(sum_{l=c}^{i-1}
// L[i][l] li[l][c]) / L[i][i], row by row, all columns of a row at once.
template <typename T>
__global__ void __launch_bounds__(256) k_diag_inverse(int n, const T* __restrict__ diagL, T* __restrict__ diagLinv) {
    __shared__ T a[kNB][kNB + 1], li[kNB][kNB + 1];
    const int b0 = blockIdx.x * kNB, bn = min(kNB, n - b0);
    const int tid = threadIdx.x;
    for (int idx = tid; idx < kNB * kNB; idx += blockDim.x) {
        const int i = idx / kNB, l = idx % kNB;
        const T v = (i < bn && l < bn) ? diagL[(size_t)(b0 + i) * kNB + l] : (T)(i == l ? 1 : 0);
        a[i][l] = v;
        li[i][l] = (i == l) ? (T)1 / v : (T)0;
    }
    __syncthreads();
    const int c = tid / 4, part = tid % 4;
    for (int i = 1; i < kNB; ++i) {
        T s = (T)0;
        if (c < i)
            for (int l = c + part; l < i; l += 4) s += a[i][l] * li[l][c];
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        if (c < i && part == 0) li[i][c] = -s * li[i][i];
        __syncthreads();
    }
    for (int idx = tid; idx < bn * kNB; idx += blockDim.x) {
        const int i = idx / kNB, l = idx % kNB;
        diagLinv[(size_t)(b0 + i) * kNB + l] = li[i][l];
    }
}

// Inverses of the 128 x 128 diagonal blocks of L from those of their two 64 x 64
// diagonal blocks (MIXED tier, for 128-row substitution blocks):
// [L0 0; L10 L1]^-1 = [L0^-1 0; -L1^-1 L10 L0^-1  L1^-1], one CTA per block.
constexpr size_t kInv128Smem = 3 * (size_t)kNB * (kNB + 1) * sizeof(float);
__global__ void __launch_bounds__(256) k_diag_inverse128(int n, const float* __restrict__ F,
                                                         const float* __restrict__ Linv, float* __restrict__ Linv128) {
    extern __shared__ float sm128[];
    float (*i0s)[kNB + 1] = (float (*)[kNB + 1])sm128;          // L0^-1
    float (*i1s)[kNB + 1] = i0s + kNB;                          // L1^-1
    float (*l10)[kNB + 1] = i1s + kNB;                          // L10, then L10 L0^-1
    const int b0 = blockIdx.x * 128, bs = min(128, n - b0), tid = threadIdx.x;
    const int b1 = b0 + kNB, bn1 = bs - kNB;                 // rows of the second 64-block (<= 0: none)
    for (int idx = tid; idx < kNB * kNB; idx += blockDim.x) {
        const int r = idx / kNB, c = idx % kNB;
        i0s[r][c] = r < bs ? Linv[(size_t)(b0 + r) * kNB + c] : 0.0f;
        i1s[r][c] = r < bn1 ? Linv[(size_t)(b1 + r) * kNB + c] : 0.0f;
        l10[r][c] = r < bn1 ? F[(size_t)(b1 + r) * n + b0 + c] : 0.0f;
    }
    __syncthreads();
    // T = L10 L0^-1 into l10 (row by row: thread (r, c-quad))
    const int r = tid / 4, q = tid % 4;
    float t[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int c = q + 4 * u;
        float v = 0.0f;
        for (int l = c; l < kNB; ++l) v += l10[r][l] * i0s[l][c];
        t[u] = v;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 16; ++u) l10[r][q + 4 * u] = t[u];
    __syncthreads();
    // X = -L1^-1 T
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int c = q + 4 * u;
        float v = 0.0f;
        for (int l = 0; l <= r; ++l) v += i1s[r][l] * l10[l][c];
        t[u] = -v;
    }
    for (int idx = tid; idx < kNB * 128; idx += blockDim.x) {
        const int rr = idx / 128, c = idx % 128;
        if (rr < bs) Linv128[(size_t)(b0 + rr) * 128 + c] = c < kNB ? i0s[rr][c] : 0.0f;
        if (rr < bn1 && c >= kNB) Linv128[(size_t)(b1 + rr) * 128 + c] = i1s[rr][c - kNB];
    }
    if (r < bn1)
#pragma unroll
        for (int u = 0; u < 16; ++u) Linv128[(size_t)(b1 + r) * 128 + q + 4 * u] = t[u];
}

// Forward (lower=1: L y = b) or backward (lower=0: L^T x = y, U = L^T in the
// upper triangle) substitution for NR vectors, one CTA of 1024 threads, by
// 64-row blocks in solve order ("right-looking"): the block is solved with the
// inverted diagonal block (a 64 x 64 matrix-vector product), then every row
// not yet solved subtracts its 64-column slice times the new block of the
// solution -- each thread streams its row slice as 16-byte vectors.  X holds b
// on entry and the solution on exit (X[k*n + i]).
constexpr int kTrsvThreads = 1024;
template <typename T, int NR>
__global__ void __launch_bounds__(kTrsvThreads) k_trsv(int n, const T* __restrict__ F, const T* __restrict__ Linv,
                                                       T* __restrict__ X, int lower) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N;
    __shared__ T rb[NR][kNB];
    __shared__ __align__(16) T yb[NR][kNB];
    const int nblk = (n + kNB - 1) / kNB;
    const bool vec_ok = (n % VN) == 0;
    for (int bb = 0; bb < nblk; ++bb) {
        const int blk = lower ? bb : nblk - 1 - bb;
        const int b0 = blk * kNB, bn = min(kNB, n - b0);
        for (int idx = threadIdx.x; idx < NR * kNB; idx += blockDim.x) {
            const int k = idx / kNB, i = idx % kNB;
            rb[k][i] = (i < bn) ? X[(size_t)k * n + b0 + i] : (T)0;
        }
        __syncthreads();
        // y = Linv r (lower) or Linv^T r (upper); four threads per output
        for (int o = threadIdx.x / 4; o < NR * kNB; o += blockDim.x / 4) {
            const int part = threadIdx.x % 4;
            const int k = o / kNB, i = o % kNB;
            T s = (T)0;
            if (i < bn) {
                if (lower)
                    for (int l = part; l <= i; l += 4) s += Linv[(size_t)(b0 + i) * kNB + l] * rb[k][l];
                else
                    for (int l = i + part; l < bn; l += 4) s += Linv[(size_t)(b0 + l) * kNB + i] * rb[k][l];
            }
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            if (part == 0) {
                yb[k][i] = (i < bn) ? s : (T)0;
                if (i < bn) X[(size_t)k * n + b0 + i] = s;
            }
        }
        __syncthreads();
        // update the rows still to solve with columns b0 .. b0+bn-1
        const int u_lo = lower ? b0 + bn : 0, u_hi = lower ? n : b0;
        for (int row = u_lo + threadIdx.x; row < u_hi; row += blockDim.x) {
            const T* frow = F + (size_t)row * n + b0;
            T acc[NR];
#pragma unroll
            for (int k = 0; k < NR; ++k) acc[k] = (T)0;
            if (vec_ok && bn == kNB) {
#pragma unroll 4
                for (int q = 0; q < kNB / VN; ++q) {
                    const V fv = *(const V*)(frow + q * VN);
#pragma unroll
                    for (int k = 0; k < NR; ++k) {
                        const V yv = *(const V*)&yb[k][q * VN];
#pragma unroll
                        for (int u = 0; u < VN; ++u) acc[k] += vget<T>(fv, u) * vget<T>(yv, u);
                    }
                }
            } else {
                for (int l = 0; l < bn; ++l) {
                    const T f = frow[l];
#pragma unroll
                    for (int k = 0; k < NR; ++k) acc[k] += f * yb[k][l];
                }
            }
#pragma unroll
            for (int k = 0; k < NR; ++k) X[(size_t)k * n + row] -= acc[k];
        }
        __syncthreads();
    }
}

template <typename T>
static void launch_trsv(int n, const T* F, const T* Linv, T* X, int nrhs, int lower, cudaStream_t s) {
    switch (nrhs) {
        case 1: k_trsv<T, 1><<<1, kTrsvThreads, 0, s>>>(n, F, Linv, X, lower); break;
        case 2: k_trsv<T, 2><<<1, kTrsvThreads, 0, s>>>(n, F, Linv, X, lower); break;
        case 3: k_trsv<T, 3><<<1, kTrsvThreads, 0, s>>>(n, F, Linv, X, lower); break;
        case 4: k_trsv<T, 4><<<1, kTrsvThreads, 0, s>>>(n, F, Linv, X, lower); break;
        case 5: k_trsv<T, 5><<<1, kTrsvThreads, 0, s>>>(n, F, Linv, X, lower); break;
        case 6: k_trsv<T, 6><<<1, kTrsvThreads, 0, s>>>(n, F, Linv, X, lower); break;
        case 7: k_trsv<T, 7><<<1, kTrsvThreads, 0, s>>>(n, F, Linv, X, lower); break;
        default: k_trsv<T, 8><<<1, kTrsvThreads, 0, s>>>(n, F, Linv, X, lower); break;
    }
}

// Multi-CTA substitution in one cooperative launch (all CTAs co-resident).
// CTA c handles the 64-row blocks blk(c), blk(c + grid), ... in solve order.
// A block waits for each block it depends on (bounded spin on a flag that the
// producer sets after writing its piece of the solution), subtracts that
// block's contribution as soon as it arrives, then applies the inverted
// diagonal block and publishes its own piece.  The L traffic is spread over
// the CTAs; the critical path is one 64 x 64 matrix-vector product per block.
// A wait that exceeds its budget (one second, or 2^22 polls) sets *err and
// ends the kernel; the blocks waiting on it then run out of budget too.
constexpr long long kSpinLimit = 1LL << 22;
constexpr unsigned long long kSpinNs = 1000000000ull;
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
template <typename T, int NR>
__global__ void __launch_bounds__(256) k_trsv_coop(int n, const T* __restrict__ F, const T* __restrict__ Linv,
                                                   T* __restrict__ X, int lower, int* __restrict__ flags, int epoch,
                                                   int* __restrict__ err) {
    __shared__ T acc[NR][kNB];
    __shared__ T yin[NR][kNB];
    __shared__ int s_abort;
    const int tid = threadIdx.x;
    const int nblk = (n + kNB - 1) / kNB;
    const int i = tid / 4, part = tid % 4;          // row of the block, column phase
    if (tid == 0) s_abort = 0;
    for (int J = blockIdx.x; J < nblk; J += gridDim.x) {
        const int blk = lower ? J : nblk - 1 - J;
        const int b0 = blk * kNB, bn = min(kNB, n - b0);
        // this thread's slice of the inverted diagonal block, fetched before any wait:
        // row i (lower) or column i (upper), entries l = part + 4 m
        T lv[kNB / 4];
#pragma unroll
        for (int m = 0; m < kNB / 4; ++m) {
            const int l = part + 4 * m;
            if (lower) lv[m] = (i < bn) ? Linv[(size_t)(b0 + i) * kNB + l] : (T)0;
            else lv[m] = (l < bn && i < bn) ? Linv[(size_t)(b0 + l) * kNB + i] : (T)0;
        }
        for (int idx = tid; idx < NR * kNB; idx += blockDim.x) {
            const int k = idx / kNB, r = idx % kNB;
            acc[k][r] = (r < bn) ? X[(size_t)k * n + b0 + r] : (T)0;
        }
        const int ndep = lower ? blk : nblk - 1 - blk;
        T fr[kNB / 4];                              // F[b0 + i][d0 + part + 4 m] of the next dependency
        auto fetch = [&](int q) {
            const int D = lower ? q : nblk - 1 - q;
            const int d0 = D * kNB, dn = min(kNB, n - d0);
#pragma unroll
            for (int m = 0; m < kNB / 4; ++m) {
                const int c = part + 4 * m;
                fr[m] = (i < bn && c < dn) ? F[(size_t)(b0 + i) * n + d0 + c] : (T)0;
            }
        };
        if (ndep > 0) fetch(0);
        __syncthreads();
        for (int q = 0; q < ndep; ++q) {
            const int D = lower ? q : nblk - 1 - q;
            const int d0 = D * kNB, dn = min(kNB, n - d0);
            if (tid == 0) {
                long long it = 0;
                const unsigned long long t0 = global_ns();
                while (atomicAdd(&flags[D], 0) != epoch) {
                    if (++it > kSpinLimit || global_ns() - t0 > kSpinNs) {
                        atomicOr(err, 1);
                        s_abort = 1;
                        break;
                    }
                    __nanosleep(32);
                }
                __threadfence();
            }
            __syncthreads();
            if (s_abort) return;
            for (int idx = tid; idx < NR * kNB; idx += blockDim.x) {
                const int k = idx / kNB, c = idx % kNB;
                yin[k][c] = (c < dn) ? __ldcg(X + (size_t)k * n + d0 + c) : (T)0;
            }
            __syncthreads();
            // acc[k][i] -= sum_c F[b0+i][d0+c] yin[k][c]  (four threads per row)
            T sk[NR];
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                T v = (T)0;
#pragma unroll
                for (int m = 0; m < kNB / 4; ++m) v += fr[m] * yin[k][part + 4 * m];
                sk[k] = v;
            }
            if (q + 1 < ndep) fetch(q + 1);
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                T v = sk[k];
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                v += __shfl_xor_sync(0xffffffffu, v, 2);
                if (part == 0 && i < bn) acc[k][i] -= v;
            }
            __syncthreads();
        }
        // own block: y = Linv acc (lower) or Linv^T acc (upper)
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            T v = (T)0;
#pragma unroll
            for (int m = 0; m < kNB / 4; ++m) v += lv[m] * acc[k][part + 4 * m];
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            if (part == 0 && i < bn) X[(size_t)k * n + b0 + i] = v;
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) atomicExch(&flags[blk], epoch);
    }
}

template <typename T, int NR>
static void coop_launch(int n, const T* F, const T* Linv, T* X, int lower, int* flags, int epoch, int* err,
                        cudaStream_t s) {
    static int max_blocks = -1;                   // co-resident CTAs of this instantiation
    if (max_blocks < 0) {
        int dev = 0, sms = 0, per = 0;
        IGS_CUDA(cudaGetDevice(&dev));
        IGS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        IGS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_trsv_coop<T, NR>, 256, 0));
        max_blocks = sms * per;
    }
    const int nblk = (n + kNB - 1) / kNB;
    const int grid = std::max(1, std::min(nblk, max_blocks));
    void* args[] = {(void*)&n, (void*)&F, (void*)&Linv, (void*)&X, (void*)&lower, (void*)&flags, (void*)&epoch,
                    (void*)&err};
    IGS_CUDA(cudaLaunchCooperativeKernel((void*)k_trsv_coop<T, NR>, dim3(grid), dim3(256), args, 0, s));
}

template <typename T>
static void launch_trsv_coop(int n, const T* F, const T* Linv, T* X, int nrhs, int lower, int* flags, int epoch,
                             int* err, cudaStream_t s) {
    switch (nrhs) {
        case 1: coop_launch<T, 1>(n, F, Linv, X, lower, flags, epoch, err, s); break;
        case 2: coop_launch<T, 2>(n, F, Linv, X, lower, flags, epoch, err, s); break;
        case 3: coop_launch<T, 3>(n, F, Linv, X, lower, flags, epoch, err, s); break;
        case 4: coop_launch<T, 4>(n, F, Linv, X, lower, flags, epoch, err, s); break;
        case 5: coop_launch<T, 5>(n, F, Linv, X, lower, flags, epoch, err, s); break;
        case 6: coop_launch<T, 6>(n, F, Linv, X, lower, flags, epoch, err, s); break;
        case 7: coop_launch<T, 7>(n, F, Linv, X, lower, flags, epoch, err, s); break;
        default: coop_launch<T, 8>(n, F, Linv, X, lower, flags, epoch, err, s); break;
    }
}

// FP32 blocked triangular solve in one cooperative launch, blocks of 64 rows,
// with the solution published as 64-bit words (value bits, epoch): a word is
// written once, atomically, so a reader that sees the current epoch holds the
// value it needs without a separate flag or fence.  Block blk waits on the
// words of each earlier block (lower) or later block (upper) in turn, applies
// that block's off-diagonal panel and finally its inverted diagonal block.
// X holds the right-hand sides on entry and the solution on exit; pub is
// [NR][n].  A wait that exceeds its budget (one second, or 2^22 polls) sets
// *err and ends the kernel; the blocks waiting on it then run out of budget.
__device__ __forceinline__ unsigned long long ld_word(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_word(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Wait until the word at w carries `tag` in its upper half; false after
// `limit` polls or `ns` nanoseconds without it.
__device__ __forceinline__ bool wait_word(const unsigned long long* w, unsigned long long tag, unsigned long long& v,
                                          long long limit, unsigned long long ns) {
    v = ld_word(w);
    if ((v & 0xffffffff00000000ull) == tag) return true;
    long long it = 0;
    const unsigned long long t0 = global_ns();
    do {
        __nanosleep(20);
        v = ld_word(w);
        if (++it > limit || global_ns() - t0 > ns) return false;
    } while ((v & 0xffffffff00000000ull) != tag);
    return true;
}

// Self-test of the bounded wait: one thread waits for a tag that nothing
// writes and records whether the wait gave up (1) or, impossibly, succeeded (0).
__global__ void k_wait_probe(const unsigned long long* w, unsigned long long ns, int* status) {
    unsigned long long v = 0;
    *status = wait_word(w, 0xabcd000000000000ull, v, 1LL << 40, ns) ? 0 : 1;
}

// The dependency tiles F[b0.., d0..] (64 x 64) do not depend on the published
// values, so they are fetched kTrsvStages - 1 tiles ahead into a shared-memory
// ring by cp.async (16-byte copies, zero fill outside the matrix; rows padded
// to kTrsvLd floats: the four column phases of eight rows hit distinct banks).
// A row of F must start on 16 bytes (n % 4 == 0); otherwise (ASYNC = false)
// the next tile is held in registers.
__host__ __device__ constexpr int trsv_stages(int RB) { return RB == 64 ? 6 : 3; }
constexpr size_t trsv_smem(int RB) { return (size_t)trsv_stages(RB) * RB * (RB + 4) * sizeof(float); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int NR, bool ASYNC, int RB>
__global__ void __launch_bounds__(4 * RB) k_trsv_pk(int n, const float* __restrict__ F, const float* __restrict__ Linv,
                                                 float* __restrict__ X, int lower, unsigned long long* pub,
                                                 int epoch, int* __restrict__ err) {
    __shared__ float acc[NR][RB];
    __shared__ float yin[NR][RB];
    extern __shared__ __align__(16) float ring[];       // [trsv_stages(RB)][RB][RB + 4] (ASYNC)
    const int tid = threadIdx.x;
    const int nblk = (n + RB - 1) / RB;
    const int i = tid / 4, part = tid % 4;          // row of the block, column phase
    const unsigned long long tag = (unsigned long long)(unsigned)epoch << 32;
    for (int J = blockIdx.x; J < nblk; J += gridDim.x) {
        const int blk = lower ? J : nblk - 1 - J;
        const int b0 = blk * RB, bn = min(RB, n - b0);
        // this thread's slice of the inverted diagonal block, fetched before any wait:
        // row i (lower) or column i (upper), entries l = part + 4 m
        float lv[RB / 4];
#pragma unroll
        for (int m = 0; m < RB / 4; ++m) {
            const int l = part + 4 * m;
            if (lower) lv[m] = (i < bn) ? Linv[(size_t)(b0 + i) * RB + l] : 0.0f;
            else lv[m] = (l < bn && i < bn) ? Linv[(size_t)(b0 + l) * RB + i] : 0.0f;
        }
        for (int idx = tid; idx < NR * RB; idx += blockDim.x) {
            const int k = idx / RB, r = idx % RB;
            acc[k][r] = (r < bn) ? X[(size_t)k * n + b0 + r] : 0.0f;
        }
        const int ndep = lower ? blk : nblk - 1 - blk;
        float fr[RB / 4];                          // F[b0 + i][d0 + part + 4 m] of the next dependency
        auto fetch = [&](int q) {                   // register path
            const int D = lower ? q : nblk - 1 - q;
            const int d0 = D * RB, dn = min(RB, n - d0);
#pragma unroll
            for (int m = 0; m < RB / 4; ++m) {
                const int c = part + 4 * m;
                fr[m] = (i < bn && c < dn) ? F[(size_t)(b0 + i) * n + d0 + c] : 0.0f;
            }
        };
        auto issue = [&](int q) {                   // ring path: tile q into stage q % trsv_stages(RB)
            if (q < ndep) {
                const int D = lower ? q : nblk - 1 - q;
                const int d0 = D * RB, dn = min(RB, n - d0);
                float* st = ring + (size_t)(q % trsv_stages(RB)) * RB * (RB + 4);
#pragma unroll
                for (int u = 0; u < RB / 16; ++u) {
                    const int ch = tid + 4 * RB * u, row = ch / (RB / 4), c4 = 4 * (ch % (RB / 4));
                    const bool ok = row < bn && c4 < dn;
                    cp_async16(st + row * (RB + 4) + c4, ok ? F + (size_t)(b0 + row) * n + d0 + c4 : F, ok ? 16 : 0);
                }
            }
            cp_async_commit();                      // empty groups keep the count uniform
        };
        if (ASYNC) {
#pragma unroll
            for (int q = 0; q < trsv_stages(RB) - 1; ++q) issue(q);
        } else if (ndep > 0) {
            fetch(0);
        }
        __syncthreads();
        for (int q = 0; q < ndep; ++q) {
            const int D = lower ? q : nblk - 1 - q;
            const int d0 = D * RB, dn = min(RB, n - d0);
            if (ASYNC) issue(q + trsv_stages(RB) - 1);
            int bad = 0;
            for (int idx = tid; idx < NR * RB; idx += blockDim.x) {
                const int k = idx / RB, c = idx % RB;
                float y = 0.0f;
                if (c < dn) {
                    unsigned long long v = 0;
                    if (!wait_word(pub + (size_t)k * n + d0 + c, tag, v, kSpinLimit, kSpinNs)) bad = 1;
                    y = __uint_as_float((unsigned)(v & 0xffffffffull));
                }
                yin[k][c] = y;
            }
            if (ASYNC) cp_async_wait<trsv_stages(RB) - 1>();    // tile q has landed (this thread's part)
            if (__syncthreads_or(bad)) {
                if (ASYNC) cp_async_wait<0>();
                if (tid == 0) atomicOr(err, 1);
                return;
            }
            if (ASYNC) {
                const float* row = ring + (size_t)(q % trsv_stages(RB)) * RB * (RB + 4) + i * (RB + 4);
#pragma unroll
                for (int m = 0; m < RB / 4; ++m) fr[m] = row[part + 4 * m];
            }
            // acc[k][i] -= sum_c F[b0+i][d0+c] yin[k][c]  (four threads per row)
            float sk[NR];
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                float v = 0.0f;
#pragma unroll
                for (int m = 0; m < RB / 4; ++m) v += fr[m] * yin[k][part + 4 * m];
                sk[k] = v;
            }
            if (!ASYNC && q + 1 < ndep) fetch(q + 1);
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                float v = sk[k];
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                v += __shfl_xor_sync(0xffffffffu, v, 2);
                if (part == 0 && i < bn) acc[k][i] -= v;
            }
            __syncthreads();
        }
        if (ASYNC) cp_async_wait<0>();              // no copy outlives its block (empty groups only)
        // own block: y = Linv acc (lower) or Linv^T acc (upper), stored and published
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            float v = 0.0f;
#pragma unroll
            for (int m = 0; m < RB / 4; ++m) v += lv[m] * acc[k][part + 4 * m];
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            if (part == 0 && i < bn) {
                X[(size_t)k * n + b0 + i] = v;
                st_word(pub + (size_t)k * n + b0 + i, tag | __float_as_uint(v));
            }
        }
        __syncthreads();
    }
}

template <int NR, bool ASYNC, int RB>
static void pk_launch_rb(int n, const float* F, const float* Linv, float* X, int lower, unsigned long long* pub,
                         int epoch, int* err, cudaStream_t s) {
    static int max_blocks = -1;                   // co-resident CTAs of this instantiation
    auto kern = k_trsv_pk<NR, ASYNC, RB>;
    const size_t smem = ASYNC ? trsv_smem(RB) : 0;
    if (max_blocks < 0) {
        int dev = 0, sms = 0, per = 0;
        IGS_CUDA(cudaGetDevice(&dev));
        IGS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        if (ASYNC) ensure_dyn_smem((const void*)kern, smem);
        IGS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 4 * RB, smem));
        max_blocks = sms * per;
    }
    const int nblk = (n + RB - 1) / RB;
    const int grid = std::max(1, std::min(nblk, max_blocks));
    void* args[] = {(void*)&n, (void*)&F, (void*)&Linv, (void*)&X, (void*)&lower, (void*)&pub, (void*)&epoch,
                    (void*)&err};
    IGS_CUDA(cudaLaunchCooperativeKernel((void*)kern, dim3(grid), dim3(4 * RB), args, smem, s));
}

// 128-row blocks (with the inverses of the 128 x 128 diagonal blocks) where a
// row of F starts on 16 bytes, else 64-row blocks
template <int NR>
static void pk_launch(int n, const float* F, const float* Linv, const float* Linv128, float* X, int lower,
                      unsigned long long* pub, int epoch, int* err, cudaStream_t s) {
    if ((n % 4) == 0 && Linv128) pk_launch_rb<NR, true, 128>(n, F, Linv128, X, lower, pub, epoch, err, s);
    else if ((n % 4) == 0) pk_launch_rb<NR, true, 64>(n, F, Linv, X, lower, pub, epoch, err, s);
    else pk_launch_rb<NR, false, 64>(n, F, Linv, X, lower, pub, epoch, err, s);
}

static void launch_trsv_pk(int n, const float* F, const float* Linv, const float* Linv128, float* X, int nrhs,
                           int lower, unsigned long long* pub, int epoch, int* err, cudaStream_t s) {
    switch (nrhs) {
        case 1: pk_launch<1>(n, F, Linv, Linv128, X, lower, pub, epoch, err, s); break;
        case 2: pk_launch<2>(n, F, Linv, Linv128, X, lower, pub, epoch, err, s); break;
        case 3: pk_launch<3>(n, F, Linv, Linv128, X, lower, pub, epoch, err, s); break;
        case 4: pk_launch<4>(n, F, Linv, Linv128, X, lower, pub, epoch, err, s); break;
        case 5: pk_launch<5>(n, F, Linv, Linv128, X, lower, pub, epoch, err, s); break;
        case 6: pk_launch<6>(n, F, Linv, Linv128, X, lower, pub, epoch, err, s); break;
        case 7: pk_launch<7>(n, F, Linv, Linv128, X, lower, pub, epoch, err, s); break;
        default: pk_launch<8>(n, F, Linv, Linv128, X, lower, pub, epoch, err, s); break;
    }
}

// r = beta - As alpha (FP64), one warp per row (lanes over columns, then a
// fixed shuffle tree).  The norms |r|^2 and |beta|^2 are summed afterwards by
// k_norms in a fixed order, so the refinement is deterministic.
template <int NR>
__global__ void k_resid(int n, const double* __restrict__ As, const double* __restrict__ alpha,
                        const double* __restrict__ beta, double* __restrict__ r) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
    if (warp >= n) return;
    const int i = warp;
    double s[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) s[k] = 0.0;
    for (int j = lane; j < n; j += 32) {
        const double a = As[(size_t)i * n + j];
#pragma unroll
        for (int k = 0; k < NR; ++k) s[k] = fma(a, alpha[(size_t)k * n + j], s[k]);
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        double v = s[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) r[(size_t)k * n + i] = beta[(size_t)k * n + i] - v;
    }
}

// norms[2k] = |r_k|^2, norms[2k+1] = |beta_k|^2: one block per data set,
// thread t sums entries t, t + 1024, ... in order, then a fixed tree.
constexpr int kNormThreads = 1024;
__global__ void __launch_bounds__(kNormThreads) k_norms(int n, const double* __restrict__ r,
                                                        const double* __restrict__ beta, double* __restrict__ norms) {
    __shared__ double s_r[kNormThreads], s_b[kNormThreads];
    const int k = blockIdx.x, t = threadIdx.x;
    double a = 0.0, b = 0.0;
    for (int i = t; i < n; i += kNormThreads) {
        const double rv = r[(size_t)k * n + i], bv = beta[(size_t)k * n + i];
        a = fma(rv, rv, a);
        b = fma(bv, bv, b);
    }
    s_r[t] = a;
    s_b[t] = b;
    __syncthreads();
    for (int h = kNormThreads / 2; h > 0; h >>= 1) {
        if (t < h) {
            s_r[t] += s_r[t + h];
            s_b[t] += s_b[t + h];
        }
        __syncthreads();
    }
    if (t == 0) {
        norms[2 * k] = s_r[0];
        norms[2 * k + 1] = s_b[0];
    }
}

// MIXED tier residual without FP64 arithmetic: r = beta - As alpha with
// As = (A + A^T)/2 read from the FP32 A and A^T, in float-float arithmetic
// (pairs hi + lo carrying about 48 bits).  Per entry: t = a + a' exactly as a
// pair (two-sum), the product with alpha_j = ah + al (the exact product th ah
// by a fused multiply-add, the cross terms rounded) and a two-sum into the
// running pair.  One warp per row, lanes over 4-column groups in order, then
// a fixed shuffle tree of pair additions: deterministic.  The final
// conversion r_i = beta_i - (sh + sl)/2 is the only FP64 arithmetic (once per
// row).  alpha_ff holds alpha as (hi, lo) pairs, [NR][n].
// (the _rn intrinsics keep the compiler from contracting these into FMAs,
// which would break the error-free transforms)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a), av = __fsub_rn(s, bv);
    e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}
__device__ __forceinline__ void ff_add(float& sh, float& sl, float ph, float pl) {
    float s, e;
    two_sum(sh, ph, s, e);
    sh = s;
    sl += e + pl;
}

__global__ void k_split_alpha(int cnt, const double* __restrict__ alpha, float2* __restrict__ aff) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cnt) return;
    const double a = alpha[q];
    const float h = (float)a;
    aff[q] = make_float2(h, (float)(a - (double)h));
}

template <int NR>
__global__ void __launch_bounds__(256) k_resid_ff(int n, const float* __restrict__ A, const float* __restrict__ AT,
                                                  const float2* __restrict__ aff, const double* __restrict__ beta,
                                                  double* __restrict__ r) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
    if (warp >= n) return;
    const int i = warp;
    const float* a_row = A + (size_t)i * n;
    const float* t_row = AT + (size_t)i * n;
    float sh[NR], sl[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) sh[k] = sl[k] = 0.0f;
    auto term = [&](float a, float at, int j) {
        float th, tl;
        two_sum(a, at, th, tl);
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            const float2 al = aff[(size_t)k * n + j];
            const float ph = __fmul_rn(th, al.x);
            const float pl = fmaf(th, al.y, fmaf(tl, al.x, fmaf(th, al.x, -ph)));
            ff_add(sh[k], sl[k], ph, pl);
        }
    };
    if ((n & 3) == 0) {
        for (int j = 4 * lane; j < n; j += 128) {
            const float4 a = *(const float4*)(a_row + j), at = *(const float4*)(t_row + j);
            term(a.x, at.x, j);
            term(a.y, at.y, j + 1);
            term(a.z, at.z, j + 2);
            term(a.w, at.w, j + 3);
        }
    } else {
        for (int j = lane; j < n; j += 32) term(a_row[j], t_row[j], j);
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        float h = sh[k], l = sl[k];
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
            ff_add(h, l, oh, ol);
        }
        if (lane == 0) r[(size_t)k * n + i] = beta[(size_t)k * n + i] - 0.5 * ((double)h + (double)l);
    }
}

static void launch_resid_ff(int n, int nrhs, const float* A, const float* AT, const double* alpha, float2* aff,
                            const double* beta, double* r, double* norms, cudaStream_t s) {
    k_split_alpha<<<(n * nrhs + 255) / 256, 256, 0, s>>>(n * nrhs, alpha, aff);
    const dim3 g((n * 32 + 255) / 256), b(256);
    switch (nrhs) {
        case 1: k_resid_ff<1><<<g, b, 0, s>>>(n, A, AT, aff, beta, r); break;
        case 2: k_resid_ff<2><<<g, b, 0, s>>>(n, A, AT, aff, beta, r); break;
        case 3: k_resid_ff<3><<<g, b, 0, s>>>(n, A, AT, aff, beta, r); break;
        case 4: k_resid_ff<4><<<g, b, 0, s>>>(n, A, AT, aff, beta, r); break;
        case 5: k_resid_ff<5><<<g, b, 0, s>>>(n, A, AT, aff, beta, r); break;
        case 6: k_resid_ff<6><<<g, b, 0, s>>>(n, A, AT, aff, beta, r); break;
        case 7: k_resid_ff<7><<<g, b, 0, s>>>(n, A, AT, aff, beta, r); break;
        default: k_resid_ff<8><<<g, b, 0, s>>>(n, A, AT, aff, beta, r); break;
    }
    k_norms<<<nrhs, kNormThreads, 0, s>>>(n, r, beta, norms);
}


static void launch_resid(int n, int nrhs, const double* As, const double* alpha, const double* beta, double* r,
                         double* norms, cudaStream_t s) {
    const dim3 g((n * 32 + 255) / 256), b(256);
    switch (nrhs) {
        case 1: k_resid<1><<<g, b, 0, s>>>(n, As, alpha, beta, r); break;
        case 2: k_resid<2><<<g, b, 0, s>>>(n, As, alpha, beta, r); break;
        case 3: k_resid<3><<<g, b, 0, s>>>(n, As, alpha, beta, r); break;
        case 4: k_resid<4><<<g, b, 0, s>>>(n, As, alpha, beta, r); break;
        case 5: k_resid<5><<<g, b, 0, s>>>(n, As, alpha, beta, r); break;
        case 6: k_resid<6><<<g, b, 0, s>>>(n, As, alpha, beta, r); break;
        case 7: k_resid<7><<<g, b, 0, s>>>(n, As, alpha, beta, r); break;
        default: k_resid<8><<<g, b, 0, s>>>(n, As, alpha, beta, r); break;
    }
    k_norms<<<nrhs, kNormThreads, 0, s>>>(n, r, beta, norms);
}

// Right-hand side of one refinement step in the factor's type: the residual
// divided by its norm (sqrt of scale[2k], if given) and, for a factor of
// D As D, multiplied by D (dscale, if given).
template <typename T>
__global__ void k_cast_in(int cnt, const double* __restrict__ src, T* __restrict__ dst, const double* __restrict__ scale,
                          int n, const float* __restrict__ dscale) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cnt) return;
    const double sc = scale ? scale[2 * (q / n)] : 0.0;
    const double inv = (sc > 0) ? 1.0 / sqrt(sc) : 1.0;
    const double dv = dscale ? (double)dscale[q % n] : 1.0;
    dst[q] = (T)(src[q] * inv * dv);
}

// x += D dx times the residual norm (the correction of one refinement step).
template <typename T>
__global__ void k_accum(int cnt, const T* __restrict__ dx, double* __restrict__ x, const double* __restrict__ scale,
                        int n, int first, const float* __restrict__ dscale) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cnt) return;
    const double sc = scale ? scale[2 * (q / n)] : 0.0;
    const double f = (sc > 0) ? sqrt(sc) : 1.0;
    const double dv = dscale ? (double)dscale[q % n] : 1.0;
    const double v = (double)dx[q] * f * dv;
    x[q] = first ? v : x[q] + v;
}

template <typename T>
static size_t panel_smem(int ns, bool fuse) {
    return (panel_rows(ns) * kPB + panel_rows(ns) * (kNB + 1) + (fuse ? panel_rows(ns) * (kNB + 16 / sizeof(T)) : 0)) *
           sizeof(T);
}
template <typename T>
static size_t syrk_smem() { return 2 * kST * syrk_ld<T>() * sizeof(T); }

// Issue the whole factorisation on stream s (used under stream capture).
// Trailing update on the 5th-generation tensor cores (MIXED tier).  Tile of
// 128 rows x 64 columns, K = 64 (the panel): D = sum_l F[i][k0+l] F[j][k0+l]
// accumulated in tensor memory by tcgen05.mma kind::tf32 in a 3-term split
// (x = hi + lo with hi = x rounded to TF32: hi.hi + hi.lo + lo.hi; the lo.lo term
// is below FP32 rounding), so the update keeps FP32-level accuracy.  Operands
// are staged in shared memory in the canonical K-major layout without swizzle
// (core matrices of 8 rows x 16 bytes; LBO = stride between core matrices
// along K, SBO = along M/N).  One thread issues the 24 MMAs and commits them to
// an mbarrier; every thread waits on it with a bounded number of polls (a miss
// sets bit 2 of *flag and skips the epilogue), then each warp reads its 32
// rows of the accumulator with tcgen05.ld and applies C -= D to the lower
// triangle.  Tiles align with the 64-wide panels, so `mode` splits the update
// as k_syrk does: 1 = the next panel's column block, 2 = the rest.
namespace tc {
constexpr uint32_t kM = 128, kN = 64, kK = 64;
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// D F32, A and B TF32, both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc() { return (1u << 4) | (2u << 7) | (2u << 10) | ((kN >> 3) << 17) | ((kM >> 4) << 24); }
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d), "l"(a), "l"(b), "r"(idesc()), "r"(accumulate));
}
__device__ __forceinline__ float tf32_hi(float x) {
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    return __uint_as_float(h);
}
constexpr size_t smem_bytes() { return (size_t)(2 * kM * kK + 2 * kN * kK) * 4 + 64; }
}  // namespace tc

__global__ void __launch_bounds__(256) k_syrk_tc(int n, float* __restrict__ F, int k0, int kb, int mode,
                                                 int* __restrict__ flag) {
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int base = k0 + kb;
    const int ti = blockIdx.y, tj = (mode == 1) ? 0 : blockIdx.x + 1;
    const int i0 = base + ti * (int)kM, j0 = base + tj * (int)kN;
    if (j0 > i0 + (int)kM - 1 || j0 >= n) return;              // no lower-triangle entry in this tile
    float* Ahi = (float*)smem_raw;
    float* Alo = Ahi + kM * kK;
    float* Bhi = Alo + kM * kK;
    float* Blo = Bhi + kN * kK;
    uint64_t* mbar = (uint64_t*)(Blo + kN * kK);
    uint32_t* s_taddr = (uint32_t*)(mbar + 1);
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(su32(s_taddr)), "r"(kN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // Staging: element (r, l) at float offset (((r/8)*(kK/4) + l/4)*8 + r%8)*4 + l%4.  A warp
    // covers 8 rows x 16 columns (512 contiguous bytes of shared memory).  Every thread
    // issues all its loads (8 float4 of A, 4 of B) before splitting and storing any.
    constexpr int kPA = (int)(kM * kK / 4) / 256, kPB = (int)(kN * kK / 4) / 256;
    float4 v[kPA + kPB];
#pragma unroll
    for (int q = 0; q < kPA + kPB; ++q) {
        const bool isA = q < kPA;
        const int idx = tid + (isA ? q : q - kPA) * 256;
        const int rr = idx % 8, c = (idx / 8) % (kK / 4), r = (idx / (8 * (kK / 4))) * 8 + rr;
        const int row = (isA ? i0 : j0) + r;
        v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < n) {
            const float* src = F + (size_t)row * n + k0 + 4 * c;
            if ((n & 3) == 0) v[q] = *(const float4*)src;
            else v[q] = make_float4(src[0], src[1], src[2], src[3]);
        }
    }
#pragma unroll
    for (int q = 0; q < kPA + kPB; ++q) {
        const bool isA = q < kPA;
        const int idx = tid + (isA ? q : q - kPA) * 256;
        const int rr = idx % 8, c = (idx / 8) % (kK / 4), g = idx / (8 * (kK / 4));
        float4 h, l;
        h.x = tf32_hi(v[q].x); l.x = v[q].x - h.x;
        h.y = tf32_hi(v[q].y); l.y = v[q].y - h.y;
        h.z = tf32_hi(v[q].z); l.z = v[q].z - h.z;
        h.w = tf32_hi(v[q].w); l.w = v[q].w - h.w;
        const size_t off = ((size_t)(g * (kK / 4) + c) * 8 + rr) * 4;
        *(float4*)((isA ? Ahi : Bhi) + off) = h;
        *(float4*)((isA ? Alo : Blo) + off) = l;
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = *s_taddr;
    if (tid == 0) {
        const uint32_t lbo = 128, sbo = (kK / 4) * 128;
        for (uint32_t ks = 0; ks < kK / 8; ++ks) {
            const uint32_t koff = ks * 256;                        // K = 8: two core matrices
            const uint64_t ah = sdesc(su32(Ahi) + koff, lbo, sbo), al = sdesc(su32(Alo) + koff, lbo, sbo);
            const uint64_t bh = sdesc(su32(Bhi) + koff, lbo, sbo), bl = sdesc(su32(Blo) + koff, lbo, sbo);
            mma(taddr, ah, bh, ks > 0 ? 1u : 0u);
            mma(taddr, ah, bl, 1u);
            mma(taddr, al, bh, 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(su32(mbar)));
    }
    bool done = false;
    for (long it = 0; it < (1L << 24) && !done; ++it) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok) : "r"(su32(mbar)), "r"(0));
        done = ok != 0;
    }
    if (!done && tid == 0) atomicOr(flag, 2);
    asm volatile("tcgen05.fence::after_thread_sync;");
    // accumulator -> shared (over the operand tiles, no longer read): warp w takes lanes
    // 32 (w % 4) .. +31 and columns 32 (w / 4) .. +31
    float (*D)[kN + 1] = (float (*)[kN + 1])smem_raw;
    if (done) {
        const int rbase = (warp % 4) * 32, cbase = (warp / 4) * 32;
#pragma unroll
        for (int c0 = 0; c0 < 32; c0 += 16) {
            uint32_t r[16];
            const uint32_t a = taddr + ((uint32_t)rbase << 16) + (uint32_t)(cbase + c0);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                           "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                         : "r"(a));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
            for (int q = 0; q < 16; ++q) D[rbase + lane][cbase + c0 + q] = __uint_as_float(r[q]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(kN));
    if (!done) return;
    // C -= D on the lower triangle, coalesced: warp w takes rows w, w+8, ..., a lane two
    // columns; every C value of the thread is loaded before any is written
    constexpr int kRows = (int)kM / 8;
    float cv[kRows][2];
#pragma unroll
    for (int t = 0; t < kRows; ++t) {
        const int i = i0 + warp + 8 * t;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = j0 + lane + 32 * h;
            cv[t][h] = (i < n && j <= i) ? F[(size_t)i * n + j] : 0.0f;
        }
    }
#pragma unroll
    for (int t = 0; t < kRows; ++t) {
        const int rl = warp + 8 * t, i = i0 + rl;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = lane + 32 * h, j = j0 + c;
            if (i < n && j <= i) F[(size_t)i * n + j] = cv[t][h] - D[rl][c];
        }
    }
}

// Outer-block operands for the tensor-core update, split once per outer block:
// rows base .. base + 64 G2 - 1 of columns K0 .. K0 + kbo - 1 of F (the factor
// of D As D, every entry at most 1 in magnitude), as FP16 high and low parts
// x = hi + lo + O(2^-22 |x| + 2^-25), in the shared-memory image the MMA
// descriptors read: K-major core matrices of 8 rows x 16 bytes, element (r, l)
// of a 64-row group and a chunk of kKC = 32 columns at half offset
// (((r/8)*4 + l/8)*8 + r%8)*8 + l%8.  img[(kc*2 + part)*G2 + g] is the 4 KB
// image of row group g, K chunk kc, part 0 = high, 1 = low; rows >= n and
// columns >= K0 + kbo are zero.  Grid (G2, chunks).
constexpr int kKC = 32;                     // factor columns per K chunk (64 bytes of FP16 per row)
constexpr int kImgHalves = 64 * kKC;        // one 64-row group of one chunk and part (4 KB)
__global__ void __launch_bounds__(256) k_split_panel(int n, const float* __restrict__ F, int K0, int kbo, int base,
                                                     int G2, __half* __restrict__ img) {
    const int g = blockIdx.x, kc = blockIdx.y;
    __half* hi = img + ((size_t)(kc * 2 + 0) * G2 + g) * kImgHalves;
    __half* lo = img + ((size_t)(kc * 2 + 1) * G2 + g) * kImgHalves;
    for (int idx = threadIdx.x; idx < kImgHalves / 8; idx += blockDim.x) {
        const int r8 = idx % 8, c = (idx / 8) % (kKC / 8), rg = idx / (8 * (kKC / 8));
        const int row = base + g * 64 + rg * 8 + r8, col = K0 + kc * kKC + 8 * c;
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = (row < n && col + q < K0 + kbo) ? F[(size_t)row * n + col + q] : 0.0f;
        __align__(16) __half h[8], l[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            h[q] = __float2half_rn(v[q]);
            l[q] = __float2half_rn(v[q] - __half2float(h[q]));
        }
        reinterpret_cast<uint4*>(hi)[idx] = *reinterpret_cast<const uint4*>(h);   // idx = ((rg*8 + c)*8 + r8)
        reinterpret_cast<uint4*>(lo)[idx] = *reinterpret_cast<const uint4*>(l);
    }
}


// Persistent, warp-specialised form of the outer-block update (MIXED tier,
// n >= 4096): one CTA per SM walks its share of the 128 x 256 lower-triangle
// tiles (column tiles tj_off .. ntc-1 of 256 columns; in column tile tj the
// 128-row tiles 2 tj .. ntr-1) in column order.  Warp 0 issues the bulk
// copies of the split operand images into kTcpStages 48 KB stages, warp 1
// issues the MMAs of the three-term FP16 split (hi.hi + hi.lo + lo.hi, FP32
// accumulation; kind::f16 runs at twice the TF32 rate on half the operand
// bytes; M = 128, N = 256: each operand byte serves 1.33x the flops of a
// 128 x 128 tile) into one of two TMEM accumulators (2 x 256 columns), warps
// 4-11 read the other accumulator back (one tile row per lane, one 128-column
// half per warp) and apply C -= D, so a tile's epilogue runs under the next
// tile's copies and MMAs.  Every wait is bounded: on a timeout (or after
// another role's timeout) the kernel sets *flag |= 2 and skips the rest.
constexpr int kTcpStages = 4;
constexpr uint32_t kTN = 256;                                  // tile columns (MMA N)
constexpr uint32_t kTcpPartA = tc::kM * kKC * 2;               // 128 rows x one chunk of FP16 (8 KB)
constexpr uint32_t kTcpPartB = kTN * kKC * 2;                  // 256 rows x one chunk of FP16 (16 KB)
constexpr uint32_t kTcpStageBytes = 2 * kTcpPartA + 2 * kTcpPartB;   // A hi, A lo, B hi, B lo (48 KB)
constexpr uint32_t kTcpBufBytes = 32 * 33 * 4;                // per epilogue warp: 32 x 32 block, padded rows
constexpr size_t tcp_smem_bytes() { return (size_t)kTcpStages * kTcpStageBytes + 8 * kTcpBufBytes + 128; }
// D F32, A and B F16, both K-major, N = kTN, M = 128
__host__ __device__ constexpr uint32_t tcp_idesc() {
    return (1u << 4) | (0u << 7) | (0u << 10) | ((kTN >> 3) << 17) | ((tc::kM >> 4) << 24);
}
__device__ __forceinline__ void tcp_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d), "l"(a), "l"(b), "r"(tcp_idesc()), "r"(accumulate));
}

// Tile t of the walk (t non-decreasing between calls); square tiles, so the
// first row tile of column tile tj is tj.
struct TcpIter {
    int tj, ti, t;
    __device__ void init(int tj_off) { tj = tj_off; ti = 2 * tj_off; t = 0; }
    __device__ void seek(int target, int ntr) {
        while (target - t >= ntr - ti) { t += ntr - ti; ++tj; ti = 2 * tj; }
        ti += target - t;
        t = target;
    }
};

// Bounded mbarrier wait: gives up after 2^24 polls or one second, or as soon
// as another role of the CTA has given up.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort) {
    const unsigned long long t0 = global_ns();
    for (long it = 0; it < (1L << 24); ++it) {
        uint32_t r;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(r) : "r"(bar), "r"(parity) : "memory");
        if (r) return true;
        if (*abort) return false;
        if ((it & 255) == 255 && global_ns() - t0 > kSpinNs) return false;
    }
    return false;
}

constexpr int kTcpThreads = 384;              // warp 0 copies, warp 1 MMAs, warps 4-11 epilogue
__global__ void __launch_bounds__(kTcpThreads, 1) k_syrk_tcp(int n, float* __restrict__ F, const __half* __restrict__ img,
                                                     int K0, int kbo, int G2, int tj_off, int ntc, int ntr, int ntiles,
                                                     int* __restrict__ flag) {
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* stages = smem_raw;
    uint64_t* bars = (uint64_t*)(stages + (size_t)kTcpStages * kTcpStageBytes + 8 * kTcpBufBytes);
    uint64_t* full = bars;                         // [kTcpStages]
    uint64_t* empty = bars + kTcpStages;           // [kTcpStages]
    uint64_t* accf = bars + 2 * kTcpStages;        // [2]
    uint64_t* acce = bars + 2 * kTcpStages + 2;    // [2]
    uint32_t* s_taddr = (uint32_t*)(bars + 2 * kTcpStages + 4);
    volatile int* s_abort = (volatile int*)(s_taddr + 1);
    const int base = K0 + kbo;
    const int nch = (kbo + kKC - 1) / kKC;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(su32(s_taddr)), "r"(2 * kTN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < kTcpStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(full + s)), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(empty + s)), "r"(1));
        }
        for (int a = 0; a < 2; ++a) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(accf + a)), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(acce + a)), "r"(8));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        *s_abort = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = *s_taddr;
    auto abort = [&]() {
        if (!*s_abort) atomicOr(flag, 2);
        *s_abort = 1;
    };

    if (warp == 0 && lane == 0) {
        // producer: bulk copies of each tile's K chunks into the stages
        TcpIter it;
        it.init(tj_off);
        long g = 0;
        for (int t = blockIdx.x; t < ntiles && !*s_abort; t += gridDim.x) {
            it.seek(t, ntr);
            for (int kc = 0; kc < nch; ++kc, ++g) {
                const int s = (int)(g % kTcpStages);
                const long use = g / kTcpStages;
                if (use >= 1 && !mbar_wait_or_abort(su32(empty + s), (uint32_t)((use - 1) & 1), s_abort)) { abort(); break; }
                unsigned char* sA = stages + (size_t)s * kTcpStageBytes;
                const uint32_t fb = su32(full + s);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(fb), "r"(kTcpStageBytes) : "memory");
                // A: two consecutive 64-row groups (4 KB each) per part, 8 KB contiguous;
                // B: four groups, 16 KB contiguous
                const __half* srcs[4] = {img + ((size_t)(kc * 2 + 0) * G2 + 2 * it.ti) * kImgHalves,
                                         img + ((size_t)(kc * 2 + 1) * G2 + 2 * it.ti) * kImgHalves,
                                         img + ((size_t)(kc * 2 + 0) * G2 + 4 * it.tj) * kImgHalves,
                                         img + ((size_t)(kc * 2 + 1) * G2 + 4 * it.tj) * kImgHalves};
                const uint32_t offs[4] = {0, kTcpPartA, 2 * kTcpPartA, 2 * kTcpPartA + kTcpPartB};
                const uint32_t sizes[4] = {kTcpPartA, kTcpPartA, kTcpPartB, kTcpPartB};
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                 :: "r"(su32(sA + offs[q])), "l"(srcs[q]), "r"(sizes[q]), "r"(fb) : "memory");
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: accumulator lt & 1 for the tile with local index lt
        const uint32_t lbo = 128, sbo = (kKC / 8) * 128;
        long g = 0;
        int lt = 0;
        for (int t = blockIdx.x; t < ntiles && !*s_abort; t += gridDim.x, ++lt) {
            const int a = lt & 1, use = lt / 2;
            if (use >= 1 && !mbar_wait_or_abort(su32(acce + a), (uint32_t)((use - 1) & 1), s_abort)) { abort(); break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t d = taddr + (uint32_t)(a * kTN);
            bool ok = true;
            for (int kc = 0; kc < nch; ++kc, ++g) {
                const int s = (int)(g % kTcpStages);
                if (!mbar_wait_or_abort(su32(full + s), (uint32_t)((g / kTcpStages) & 1), s_abort)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const unsigned char* sA = stages + (size_t)s * kTcpStageBytes;
                const uint32_t aH = su32(sA), aL = su32(sA + kTcpPartA), bH = su32(sA + 2 * kTcpPartA),
                               bL = su32(sA + 2 * kTcpPartA + kTcpPartB);
                for (uint32_t ks = 0; ks < kKC / 16; ++ks) {                  // K = 16 halves (32 bytes) per MMA
                    const uint32_t koff = ks * 256;
                    const uint64_t ah = sdesc(aH + koff, lbo, sbo), al = sdesc(aL + koff, lbo, sbo);
                    const uint64_t bh = sdesc(bH + koff, lbo, sbo), bl = sdesc(bL + koff, lbo, sbo);
                    tcp_mma(d, ah, bh, (kc > 0 || ks > 0) ? 1u : 0u);
                    tcp_mma(d, ah, bl, 1u);
                    tcp_mma(d, al, bh, 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(su32(empty + s)) : "memory");
            }
            if (!ok) { abort(); break; }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(su32(accf + a)) : "memory");
        }
    } else if (warp >= 4) {
        // epilogue: warp 4 + q + 4 h reads TMEM lane quadrant q (= warp % 4, the
        // quadrant a warp may access) and column half h: tile rows 32 q .. +31,
        // columns 128 h .. +127, in four passes of 32 columns.  A pass loads the
        // 32 x 32 block from TMEM (lane = row), transposes it through the warp's
        // padded shared-memory buffer and applies C -= D with lanes spread as 4
        // rows x 8 float4 per instruction (4 cache lines per access instead of
        // 32).  The first pass's C values are loaded before the accumulator wait.
        const int q4 = (warp - 4) % 4, h = (warp - 4) / 4;
        float (*buf)[33] = (float (*)[33])(stages + (size_t)kTcpStages * kTcpStageBytes + (size_t)(warp - 4) * kTcpBufBytes);
        const int rl = lane / 8, c4 = lane % 8;                 // row-in-quad, float4 column of a pass
        TcpIter it;
        it.init(tj_off);
        int lt = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
            const int a = lt & 1, use = lt / 2;
            it.seek(t, ntr);
            const int i0 = base + it.ti * (int)kM, j0 = base + it.tj * (int)kTN;
            const int ib = i0 + q4 * 32;                          // first row of this warp
            float4 cv[8];
            auto prefetch = [&](int ps) {
                const int jc = j0 + h * 128 + ps * 32 + 4 * c4;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int i = ib + 4 * q + rl;
                    if ((n & 3) == 0 && i < n && jc + 3 <= i) cv[q] = *(const float4*)(F + (size_t)i * n + jc);
                }
            };
            prefetch(0);
            bool ok = mbar_wait_or_abort(su32(accf + a), (uint32_t)(use & 1), s_abort);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) abort();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            for (int ps = 0; ps < 4; ++ps) {
                uint32_t r[32];
                const uint32_t addr = taddr + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(a * kTN + h * 128 + ps * 32);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                             "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                               "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                               "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                               "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                             : "r"(addr));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                if (ps == 3) {
                    // this warp's share of the accumulator is read: free it for the tile after next
                    asm volatile("tcgen05.fence::before_thread_sync;");
                    __syncwarp();
                    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(su32(acce + a)) : "memory");
                }
                __syncwarp();                                     // the previous pass's reads of buf are done
#pragma unroll
                for (int c = 0; c < 32; ++c) buf[lane][c] = __uint_as_float(r[c]);
                __syncwarp();
                const int jc = j0 + h * 128 + ps * 32 + 4 * c4;
                float4 w[8];
                bool whole[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int rr = 4 * q + rl, i = ib + rr;
                    whole[q] = (n & 3) == 0 && i < n && jc + 3 <= i;
                    w[q] = cv[q];
                    w[q].x -= buf[rr][4 * c4];
                    w[q].y -= buf[rr][4 * c4 + 1];
                    w[q].z -= buf[rr][4 * c4 + 2];
                    w[q].w -= buf[rr][4 * c4 + 3];
                }
                if (ps < 3) prefetch(ps + 1);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int rr = 4 * q + rl, i = ib + rr;
                    if (whole[q]) {
                        *(float4*)(F + (size_t)i * n + jc) = w[q];
                    } else if (i < n) {
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (jc + u <= i && jc + u < n) F[(size_t)i * n + jc + u] -= buf[rr][4 * c4 + u];
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(2 * kTN));
}

// The factorisation's critical chain (panels, the next column block's or outer
// block's update, the operand split) launches at the device's highest
// scheduling priority: when SM resources free up, its CTAs go before those of
// concurrent work (the right-hand side of igs_solve_data, the update of the
// columns beyond the next outer block), which has the default priority.
static int chain_priority() {
    static int prio = 1;
    if (prio == 1) {
        int least = 0, greatest = 0;
        IGS_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        prio = greatest;
    }
    return prio;
}

// Launch at the chain priority, with programmatic stream serialisation if pdl
// (see pdl_wait).
template <typename... KArgs, typename... Args>
static void launch_chain(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                         Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = chain_priority();
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 2 : 1;
    IGS_CUDA(cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...));
}
template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    launch_chain(true, kern, grid, block, smem, s, args...);
}

// Panel step at column k0: CTA 0 the diagonal block, the others the rows
// below, 64 per CTA or, where those CTAs would not all fit at once (FP32),
// 192 per CTA.  FP32 panels apply the update by the previous panel kp of
// their own column block first (kp < 0: none).
template <typename T, int NS, int PARTS, bool FUSE>
static void launch_panel_ns(igs_prob p, int n, T* F, int k0, int kb, int kp, int below, cudaStream_t s) {
    launch_pdl(k_panel<T, NS, PARTS, FUSE>, dim3(1 + (below + NS * kNB - 1) / (NS * kNB)),
               dim3(panel_threads(NS, PARTS)), panel_smem<T>(NS, FUSE), s, n, F, k0, kb, kp, (T*)p->d_diagL,
               p->d_flag);
}

template <typename T>
static void launch_panel(igs_prob p, int n, T* F, int k0, int kb, int kp, cudaStream_t s) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        IGS_CUDA(cudaGetDevice(&dev));
        IGS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const int below = std::max(0, n - k0 - kNB);
    if constexpr (std::is_same<T, float>::value) {
        if (1 + (below + kNB - 1) / kNB > sms) return launch_panel_ns<T, 3, 2, true>(p, n, F, k0, kb, kp, below, s);
        return launch_panel_ns<T, 1, 4, true>(p, n, F, k0, kb, kp, below, s);
    } else {
        launch_panel_ns<T, 1, 4, false>(p, n, F, k0, kb, -1, below, s);
    }
}

template <typename T>
static void launch_update(igs_prob p, int n, T* F, int k0, int kb, int mode, cudaStream_t s);
template <>
void launch_update<double>(igs_prob, int n, double* F, int k0, int kb, int mode, cudaStream_t s) {
    const int rem = n - k0 - kb, nt = (rem + kST - 1) / kST;
    if (mode == 1) launch_pdl(k_syrk<double>, dim3(nt), dim3(256), syrk_smem<double>(), s, n, F, k0, kb, 1);
    else k_syrk<double><<<(nt - 1) * nt / 2, 256, syrk_smem<double>(), s>>>(n, F, k0, kb, 2);
}
// MIXED tier: the next panel's column block (on the critical path, few tiles) by the
// SIMT kernel, whose 64 x 64 tiles have the shorter latency; the rest of the trailing
// matrix, which runs beside the next panel, on the tensor cores.
template <>
void launch_update<float>(igs_prob p, int n, float* F, int k0, int kb, int mode, cudaStream_t s) {
    const int rem = n - k0 - kb;
    const int ntr = (rem + (int)tc::kM - 1) / (int)tc::kM, ntc = (rem + (int)tc::kN - 1) / (int)tc::kN;
    if (mode == 1)
        launch_pdl(k_syrk<float>, dim3((rem + kST - 1) / kST), dim3(256), syrk_smem<float>(), s, n, F, k0, kb, 1);
    else k_syrk_tc<<<dim3(ntc - 1, ntr), 256, tc::smem_bytes(), s>>>(n, F, k0, kb, 2, p->d_flag);
}

// One factorisation as a two-stream launch sequence (captured into a graph):
// s0 carries panel k, the update of column block k+1 and panel k+1 (FP32: the
// panel k+1 applies that update itself); s1 the rest of the update of step k,
// concurrent with panel k+1.  Ordering: the first-column update of step k
// (FP32: panel k+1) waits for the rest-update of step k-1 (both touch column
// block k+1); the rest-update of step k waits for panel k.
template <typename T>
static void issue_factor(igs_prob p, cudaStream_t s0, cudaStream_t s1, cudaEvent_t evP, cudaEvent_t evB,
                         cudaEvent_t evJ) {
    const int n = p->plan.n;
    T* F = (T*)p->d_F;
    IGS_CUDA(cudaMemsetAsync(p->d_flag, 0, sizeof(int), s0));
    bool pending = false, forked = false;
    if constexpr (std::is_same<T, float>::value) {
        // FP32: panel j updates its own column block by panel j - 1; the rest of
        // step j's update (beyond column block j + 1) on s1, after panel j.  Panel
        // j waits for the rest-update of step j - 2 (which touched its columns):
        // the completion events alternate by the parity of j.
        cudaEvent_t evSide[2] = {evB, evJ};
        bool side[2] = {false, false};
        for (int k0 = 0; k0 < n; k0 += kNB) {
            const int kb = std::min(kNB, n - k0), j = k0 / kNB;
            if (side[j & 1]) {
                IGS_CUDA(cudaStreamWaitEvent(s0, evSide[j & 1], 0));
                side[j & 1] = false;
            }
            launch_panel<T>(p, n, F, k0, kb, k0 > 0 ? k0 - kNB : -1, s0);
            if (n - k0 - kb <= kST) continue;
            IGS_CUDA(cudaEventRecord(evP, s0));
            IGS_CUDA(cudaStreamWaitEvent(s1, evP, 0));
            forked = true;
            launch_update<T>(p, n, F, k0, kb, 2, s1);
            IGS_CUDA(cudaEventRecord(evSide[j & 1], s1));
            side[j & 1] = true;
        }
    }
    for (int k0 = 0; k0 < n && !std::is_same<T, float>::value; k0 += kNB) {
        const int kb = std::min(kNB, n - k0);
        launch_panel<T>(p, n, F, k0, kb, -1, s0);
        const int rem = n - k0 - kb;
        if (rem <= 0) continue;
        const int nt = (rem + kST - 1) / kST;
        if (nt > 1) IGS_CUDA(cudaEventRecord(evP, s0));
        if (pending) {
            IGS_CUDA(cudaStreamWaitEvent(s0, evB, 0));
            pending = false;
        }
        launch_update<T>(p, n, F, k0, kb, 1, s0);
        if (nt > 1) {
            IGS_CUDA(cudaStreamWaitEvent(s1, evP, 0));
            forked = true;
            launch_update<T>(p, n, F, k0, kb, 2, s1);
            IGS_CUDA(cudaEventRecord(evB, s1));
            pending = true;
        }
    }
    if (forked) {
        IGS_CUDA(cudaEventRecord(evJ, s1));
        IGS_CUDA(cudaStreamWaitEvent(s0, evJ, 0));
    }
    // the inverses of the diagonal blocks (from diagL and the strictly lower part
    // of F) on the second stream, beside the mirror (diagonal blocks and upper
    // triangle of F) on the first
    IGS_CUDA(cudaEventRecord(evP, s0));
    IGS_CUDA(cudaStreamWaitEvent(s1, evP, 0));
    k_diag_inverse<T><<<(n + kNB - 1) / kNB, 256, 0, s1>>>(n, (const T*)p->d_diagL, (T*)p->d_diagLinv);
    if (std::is_same<T, float>::value && p->d_diagLinv128)
        k_diag_inverse128<<<(n + 127) / 128, 256, kInv128Smem, s1>>>(n, (const float*)p->d_F,
                                                                   (const float*)p->d_diagLinv, p->d_diagLinv128);
    const int nft = (n + kTT - 1) / kTT;
    k_finalize<T><<<nft * (nft + 1) / 2, 256, 0, s0>>>(n, F, (const T*)p->d_diagL, 0, 0);
    IGS_CUDA(cudaEventRecord(evJ, s1));
    IGS_CUDA(cudaStreamWaitEvent(s0, evJ, 0));
    IGS_CUDA(cudaGetLastError());
}

// MIXED tier, large n: the same panels, with the trailing update blocked by
// outer column blocks of kOB = 8 panels.  Inside an outer block each panel
// updates only the remaining columns of that block: the next panel's columns
// in the next panel itself, the block's later columns (SIMT, mode 4) on a
// third stream s2 beside the next panel (the panel after next waits for it,
// both touching its columns); after the
// block's last panel the rest of the matrix is updated once with K = kOB on
// the tensor cores.  Look-ahead as in issue_factor, one level up: the next
// outer block's columns are updated first on s0; the rest of the outer update
// runs on s1 beside the next outer block's panels, and the next outer step's
// s0 update waits for it (both touch the columns after the next block).
constexpr int kOB = 8 * kNB;
constexpr int kBlockedMinN = 4096;

// The image buffers hold two outer blocks (alternating), so the split of
// block k+1 does not overwrite what the rest-update of block k still reads;
// the split of block k+2 comes after the s0 wait on that rest-update.
// 64-row groups of the split images: four per 256-column tile (which also
// covers the two per 128-row tile)
static int tcb_groups(int n) { return 4 * ((n + (int)kTN - 1) / (int)kTN); }
static size_t tcb_image_halves(int n) { return (size_t)(kOB / kKC) * 2 * tcb_groups(n) * kImgHalves; }

constexpr int kTcpReserveSMs = 80;
static void tcb_launch(int n, float* F, const __half* img, int K0, int kbo, int tj_off, int tcols, int* flag,
                       cudaStream_t s) {
    const int rem = n - K0 - kbo;
    const int ntr = (rem + (int)tc::kM - 1) / (int)tc::kM;
    if (tcols <= 0 || ntr <= 0) return;
    const int ntc = tj_off + tcols;
    const int G2 = tcb_groups(rem);
    int ntiles = 0;
    for (int tj = tj_off; tj < ntc; ++tj) ntiles += ntr - 2 * tj;     // row tiles 2 tj .. ntr - 1
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        IGS_CUDA(cudaGetDevice(&dev));
        IGS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    // a CTA of this kernel fills an SM's shared memory: the update of the columns
    // beyond the next outer block (tj_off > 0, on the second stream) leaves
    // kTcpReserveSMs SMs to the next outer block's panel chain, so the two overlap
    const int avail = tj_off > 0 ? std::max(1, sms - kTcpReserveSMs) : sms;
    const int grid = std::max(1, std::min(ntiles, avail));
    if (tj_off == 0)        // the next outer block's columns: on the chain
        launch_chain(false, k_syrk_tcp, dim3(grid), dim3(kTcpThreads), tcp_smem_bytes(), s, n, F, img, K0, kbo, G2,
                     tj_off, ntc, ntr, ntiles, flag);
    else
        k_syrk_tcp<<<grid, kTcpThreads, tcp_smem_bytes(), s>>>(n, F, img, K0, kbo, G2, tj_off, ntc, ntr, ntiles, flag);
}

static void issue_factor_blocked(igs_prob p, cudaStream_t s0, cudaStream_t s1, cudaStream_t s2, cudaEvent_t evP,
                                 cudaEvent_t evB, cudaEvent_t evJ, cudaEvent_t evQ, cudaEvent_t evS) {
    const int n = p->plan.n;
    float* F = (float*)p->d_F;
    IGS_CUDA(cudaMemsetAsync(p->d_flag, 0, sizeof(int), s0));
    bool pending = false, forked = false;
    int mirrored = 0;                        // columns below which U = L^T is written (outer-block mirrors)
    cudaEvent_t evSide[2] = {evS, evJ};      // in-block side updates by parity (evJ recorded again at the end)
    for (int K0 = 0; K0 < n; K0 += kOB) {
        const int kbo = std::min(kOB, n - K0);
        bool side[2] = {false, false};           // side updates of this block pending, by parity of the step
        for (int k0 = K0; k0 < K0 + kbo; k0 += kNB) {
            const int kb = std::min(kNB, n - k0), j = (k0 - K0) / kNB;
            // panel j updates its own columns by panel j - 1 of the block, after the
            // side update of step j - 2 (which touched them; events by parity of j)
            if (side[j & 1]) {
                IGS_CUDA(cudaStreamWaitEvent(s0, evSide[j & 1], 0));
                side[j & 1] = false;
            }
            launch_panel<float>(p, n, F, k0, kb, k0 > K0 ? k0 - kNB : -1, s0);
            const int inner = (K0 + kbo - (k0 + kb) + kST - 1) / kST;   // column tiles left in this block
            if (inner <= 1) continue;
            // the block's columns beyond the next panel's on the third stream
            const int nt = (n - k0 - kb + kST - 1) / kST;
            IGS_CUDA(cudaEventRecord(evQ, s0));
            IGS_CUDA(cudaStreamWaitEvent(s2, evQ, 0));
            k_syrk<float><<<dim3(nt, inner - 1), 256, syrk_smem<float>(), s2>>>(n, F, k0, kb, 4);
            IGS_CUDA(cudaEventRecord(evSide[j & 1], s2));
            side[j & 1] = true;
        }
        const int rem = n - K0 - kbo;
        if (rem <= 0) continue;
        const int ntc = (rem + (int)kTN - 1) / (int)kTN;             // 256-column tiles
        const int G2 = tcb_groups(rem);
        __half* img = reinterpret_cast<__half*>(p->d_timg) + (size_t)((K0 / kOB) & 1) * tcb_image_halves(n);
        launch_chain(false, k_split_panel, dim3(G2, (kbo + kKC - 1) / kKC), dim3(256), 0, s0, n, (const float*)F, K0, kbo,
                     K0 + kbo, G2, img);
        const int first = std::min(ntc, kOB / (int)kTN);             // the next outer block's column tiles
        if (ntc > first) IGS_CUDA(cudaEventRecord(evP, s0));
        if (pending) {
            IGS_CUDA(cudaStreamWaitEvent(s0, evB, 0));
            pending = false;
        }
        tcb_launch(n, F, img, K0, kbo, 0, first, p->d_flag, s0);
        if (ntc > first) {
            IGS_CUDA(cudaStreamWaitEvent(s1, evP, 0));
            forked = true;
            tcb_launch(n, F, img, K0, kbo, first, ntc - first, p->d_flag, s1);
            IGS_CUDA(cudaEventRecord(evB, s1));
            pending = true;
            // the mirror of this outer block (its rows are final: later updates touch
            // rows of later blocks only), on s1 after the update it must not delay
            const int nft = (n + kTT - 1) / kTT;
            k_finalize<float><<<dim3(nft - K0 / kTT, kbo / kTT), 256, 0, s1>>>(n, F, (const float*)p->d_diagL,
                                                                             K0 / kTT, kbo / kTT);
            mirrored = K0 + kbo;
        }
    }
    if (forked) {
        IGS_CUDA(cudaEventRecord(evJ, s1));
        IGS_CUDA(cudaStreamWaitEvent(s0, evJ, 0));
    }
    // inverses beside the mirror, as in the unblocked factorisation
    IGS_CUDA(cudaEventRecord(evP, s0));
    IGS_CUDA(cudaStreamWaitEvent(s1, evP, 0));
    k_diag_inverse<float><<<(n + kNB - 1) / kNB, 256, 0, s1>>>(n, (const float*)p->d_diagL, (float*)p->d_diagLinv);
    if (p->d_diagLinv128)
        k_diag_inverse128<<<(n + 127) / 128, 256, kInv128Smem, s1>>>(n, (const float*)p->d_F,
                                                                   (const float*)p->d_diagLinv, p->d_diagLinv128);
    const int nft = (n + kTT - 1) / kTT, m = nft - mirrored / kTT;   // tile columns not yet mirrored
    k_finalize<float><<<m * (m + 1) / 2, 256, 0, s0>>>(n, F, (const float*)p->d_diagL, mirrored / kTT, 0);
    IGS_CUDA(cudaEventRecord(evJ, s1));
    IGS_CUDA(cudaStreamWaitEvent(s0, evJ, 0));
    IGS_CUDA(cudaGetLastError());
}

static int factor_launches_blocked(int n) {
    int c = 2;
    for (int K0 = 0; K0 < n; K0 += kOB) {
        const int kbo = std::min(kOB, n - K0);
        for (int k0 = K0; k0 < K0 + kbo; k0 += kNB) c += 1 + (k0 + 2 * kNB < K0 + kbo ? 1 : 0);
        const int rem = n - K0 - kbo;
        if (rem > 0) c += (rem > kOB) ? 4 : 2;
    }
    return c;
}

static int factor_launches(int n, bool fused) {
    int c = 2;
    for (int k0 = 0; k0 < n; k0 += kNB) {
        ++c;
        const int rem = n - k0 - kNB;
        if (rem > 0) c += (rem > kST) ? 2 - fused : 1 - fused;
    }
    return c;
}

// Capture the factorisation's fixed launch sequence into p->factor_exec, on
// two private streams.
template <typename T>
static void capture_factor(igs_prob p, bool blocked) {
    // capture the fixed launch sequence once, on private streams
    cudaStream_t cs = nullptr, cs1 = nullptr, cs2 = nullptr;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    auto release = [&]() {
        for (cudaEvent_t& e : ev)
            if (e) cudaEventDestroy(e);
        if (cs1) cudaStreamDestroy(cs1);
        if (cs2) cudaStreamDestroy(cs2);
        if (cs) cudaStreamDestroy(cs);
    };
    cudaGraph_t graph = nullptr;
    try {
        IGS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        IGS_CUDA(cudaStreamCreateWithFlags(&cs1, cudaStreamNonBlocking));
        IGS_CUDA(cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking));
        for (cudaEvent_t& e : ev) IGS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        IGS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        try {
            if (blocked) issue_factor_blocked(p, cs, cs1, cs2, ev[0], ev[1], ev[2], ev[3], ev[4]);
            else issue_factor<T>(p, cs, cs1, ev[0], ev[1], ev[2]);
        } catch (...) {
            cudaStreamEndCapture(cs, &graph);
            if (graph) cudaGraphDestroy(graph);
            throw;
        }
        IGS_CUDA(cudaStreamEndCapture(cs, &graph));
    } catch (...) {
        release();
        throw;
    }
    cudaError_t e = cudaGraphInstantiate(&p->factor_exec, graph, 0);
    cudaGraphDestroy(graph);
    release();
    if (e != cudaSuccess) {
        p->factor_exec = nullptr;
        throw Error(IGS_E_CUDA, cuda_msg(e, "cudaGraphInstantiate", __FILE__, __LINE__));
    }
}

template <typename T>
static void factor(igs_prob p, cudaStream_t s) {
    const int n = p->plan.n;
    if constexpr (std::is_same<T, float>::value) {
        ensure_dyn_smem((const void*)k_panel<T, 1, 4, true>, panel_smem<T>(1, true));
        ensure_dyn_smem((const void*)k_panel<T, 3, 2, true>, panel_smem<T>(3, true));
    } else {
        ensure_dyn_smem((const void*)k_panel<T, 1, 4, false>, panel_smem<T>(1, false));
    }
    ensure_dyn_smem((const void*)k_syrk<T>, (size_t)syrk_smem<T>());
    ensure_dyn_smem((const void*)k_syrk_tc, tc::smem_bytes());
    ensure_dyn_smem((const void*)k_syrk_tcp, tcp_smem_bytes());
    ensure_dyn_smem((const void*)k_diag_inverse128, kInv128Smem);
    const bool blocked = std::is_same<T, float>::value && n >= kBlockedMinN;
    if (!p->factor_exec && p->factor_runs == 0) {
        // first factorisation of this problem: issue the launch sequence directly
        // (a problem factored once, such as a served request, does not pay for a
        // graph capture); the graph is captured when the problem is factored again
        cudaStream_t s1 = nullptr, s2 = nullptr;
        cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
        auto release = [&]() {
            for (cudaEvent_t& e : ev)
                if (e) cudaEventDestroy(e);
            if (s1) cudaStreamDestroy(s1);
            if (s2) cudaStreamDestroy(s2);
        };
        try {
            IGS_CUDA(cudaStreamCreateWithFlags(&s1, cudaStreamNonBlocking));
            IGS_CUDA(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
            for (cudaEvent_t& e : ev) IGS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            if (blocked) issue_factor_blocked(p, s, s1, s2, ev[0], ev[1], ev[2], ev[3], ev[4]);
            else issue_factor<T>(p, s, s1, ev[0], ev[1], ev[2]);
        } catch (...) {
            release();
            throw;
        }
        release();
    } else {
        if (!p->factor_exec) capture_factor<T>(p, blocked);
        IGS_CUDA(cudaGraphLaunch(p->factor_exec, s));
    }
    p->factor_runs++;
    p->launches += (blocked ? factor_launches_blocked(n) : factor_launches(n, std::is_same<T, float>::value)) + (p->d_diagLinv128 ? 1 : 0);
    int flag = 0;
    IGS_CUDA(cudaMemcpyAsync(&flag, p->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    IGS_CUDA(cudaStreamSynchronize(s));
    if (flag & 2) throw Error(IGS_E_TIMEOUT, "tensor-core update: MMA completion wait exceeded its budget");
    if (flag) throw Error(IGS_E_NOT_SPD, "Cholesky met a non-positive pivot");
}

template <typename T>
static void prepare_factor(igs_prob p, cudaStream_t s) {
    const int n = p->plan.n;
    if (!p->d_F) {
        p->d_F = dev_alloc(p, sizeof(T) * (size_t)n * n);
        p->d_diagL = dev_alloc(p, sizeof(T) * (size_t)n * kNB);
        p->d_diagLinv = dev_alloc(p, sizeof(T) * (size_t)n * kNB);
        p->d_tflags = (int*)dev_alloc(p, sizeof(int) * ((n + kNB - 1) / kNB));
        IGS_CUDA(cudaMemsetAsync(p->d_tflags, 0, sizeof(int) * ((n + kNB - 1) / kNB), s));
        if (std::is_same<T, float>::value && n >= kBlockedMinN)
            p->d_timg = (float*)dev_alloc(p, sizeof(__half) * 2 * tcb_image_halves(n));
        if (std::is_same<T, float>::value) {
            p->d_tpub = (unsigned long long*)dev_alloc(p, sizeof(unsigned long long) * 8 * (size_t)n);
            IGS_CUDA(cudaMemsetAsync(p->d_tpub, 0, sizeof(unsigned long long) * 8 * (size_t)n, s));
        }
        p->tepoch = 0;
        int dev = 0, coop = 0;
        IGS_CUDA(cudaGetDevice(&dev));
        IGS_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        p->coop_ok = coop != 0;
        if (std::is_same<T, float>::value && p->coop_ok && (n % 4) == 0 && n >= 256)
            p->d_diagLinv128 = (float*)dev_alloc(p, sizeof(float) * (size_t)n * 128);
        // the factor graph captures these pointers: allocate before capture, keep for the problem's life
        IGS_CUDA(cudaStreamSynchronize(s));
    }
    if (!p->at_ready) {
        if (!p->d_AT) p->d_AT = dev_alloc(p, sizeof(T) * (size_t)n * n);
        k_transpose<T><<<dim3((n + 31) / 32, (n + 31) / 32), 256, 0, s>>>(n, (const T*)p->d_A, (T*)p->d_AT);
        p->launches++;
        p->at_ready = 1;
    }
    if (std::is_same<T, float>::value) {
        // MIXED tier: factor D As D with unit diagonal (D = diag(As_ii^-1/2)), so that
        // every factor entry is at most 1 in magnitude (the tensor-core update's
        // FP16 split); the refinement residual reads A and A^T (no FP64 copy of As)
        if (!p->d_dscale) p->d_dscale = (float*)dev_alloc(p, sizeof(float) * (size_t)n);
        k_diag_scale<<<(n + 255) / 256, 256, 0, s>>>(n, (const float*)p->d_A, p->d_dscale);
        k_symmetrize_lower_f<<<dim3((n + 1023) / 1024, n), 256, 0, s>>>(n, (const float*)p->d_A, (const float*)p->d_AT,
                                                                         (float*)p->d_F, p->d_dscale);
        p->launches += 2;
    } else {
        if (!p->d_As64) p->d_As64 = (double*)dev_alloc(p, sizeof(double) * (size_t)n * n);
        constexpr int VN = Vec16<T>::N;
        k_symmetrize<T><<<dim3((n + 256 * VN - 1) / (256 * VN), n), 256, 0, s>>>(
            n, (const T*)p->d_A, (const T*)p->d_AT, (T*)p->d_F, p->d_As64);
        p->launches++;
    }
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
    float2* d_aff = std::is_same<T, float>::value ? (float2*)dev_alloc(p, sizeof(float2) * cnt) : nullptr;
    std::vector<double> hn(2 * nrhs);
    int it = 0;
    const double* src = d_beta;
    const double* scale = nullptr;
    IGS_CUDA(cudaMemsetAsync(p->d_flag, 0, sizeof(int), s));
    for (;;) {
        const float* dsc = std::is_same<T, float>::value ? p->d_dscale : nullptr;
        k_cast_in<T><<<(cnt + 255) / 256, 256, 0, s>>>(cnt, src, d_x, scale, n, dsc);
        if (std::is_same<T, float>::value && p->coop_ok) {
            launch_trsv_pk(n, (const float*)p->d_F, (const float*)p->d_diagLinv, p->d_diagLinv128, (float*)d_x, nrhs, 1,
                           p->d_tpub,
                           ++p->tepoch, p->d_flag, s);
            launch_trsv_pk(n, (const float*)p->d_F, (const float*)p->d_diagLinv, p->d_diagLinv128, (float*)d_x, nrhs, 0,
                           p->d_tpub,
                           ++p->tepoch, p->d_flag, s);
        } else if (p->coop_ok) {
            launch_trsv_coop<T>(n, (const T*)p->d_F, (const T*)p->d_diagLinv, d_x, nrhs, 1, p->d_tflags,
                                ++p->tepoch, p->d_flag, s);
            launch_trsv_coop<T>(n, (const T*)p->d_F, (const T*)p->d_diagLinv, d_x, nrhs, 0, p->d_tflags,
                                ++p->tepoch, p->d_flag, s);
        } else {
            launch_trsv<T>(n, (const T*)p->d_F, (const T*)p->d_diagLinv, d_x, nrhs, 1, s);
            launch_trsv<T>(n, (const T*)p->d_F, (const T*)p->d_diagLinv, d_x, nrhs, 0, s);
        }
        k_accum<T><<<(cnt + 255) / 256, 256, 0, s>>>(cnt, d_x, d_alpha, scale, n, it == 0, dsc);
        if (std::is_same<T, float>::value)
            launch_resid_ff(n, nrhs, (const float*)p->d_A, (const float*)p->d_AT, d_alpha, d_aff, d_beta, d_r, d_norm, s);
        else
            launch_resid(n, nrhs, p->d_As64, d_alpha, d_beta, d_r, d_norm, s);
        p->launches += std::is_same<T, float>::value ? 7 : 6;
        IGS_CUDA(cudaGetLastError());
        if (it == 0 && max_it > 1) {
            // an FP32 factor never meets the tolerance after one step: go on to the
            // second without a round trip to the host (the next step reads the
            // residual and its norm on the device)
            ++it;
            src = d_r;
            scale = d_norm;
            continue;
        }
        IGS_CUDA(cudaMemcpyAsync(hn.data(), d_norm, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, s));
        int tflag = 0;
        IGS_CUDA(cudaMemcpyAsync(&tflag, p->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        IGS_CUDA(cudaStreamSynchronize(s));
        if (tflag) {
            dev_free(p, d_x);
            dev_free(p, d_r);
            dev_free(p, d_norm);
            if (d_aff) dev_free(p, d_aff);
            throw Error(IGS_E_TIMEOUT, "triangular solve: a block waited past its budget");
        }
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
    if (d_aff) dev_free(p, d_aff);
    double worst = 0;
    for (int k = 0; k < nrhs; ++k) worst = std::max(worst, hn[2 * k + 1] > 0 ? std::sqrt(hn[2 * k] / hn[2 * k + 1]) : 0.0);
    if (worst > tol && max_it > 1) throw Error(IGS_E_NOT_CONVERGED, "iterative refinement did not reach 1e-10");
}

int wait_selftest(int device, double budget_s) {
    IGS_CUDA(cudaSetDevice(device));
    unsigned long long* d_w = nullptr;
    int* d_st = nullptr;
    IGS_CUDA(cudaMalloc(&d_w, sizeof(unsigned long long)));
    IGS_CUDA(cudaMalloc(&d_st, sizeof(int)));
    IGS_CUDA(cudaMemset(d_w, 0, sizeof(unsigned long long)));
    IGS_CUDA(cudaMemset(d_st, 0xff, sizeof(int)));
    k_wait_probe<<<1, 1>>>(d_w, (unsigned long long)(budget_s * 1e9), d_st);
    IGS_CUDA(cudaGetLastError());
    int st = -1;
    IGS_CUDA(cudaMemcpy(&st, d_st, sizeof(int), cudaMemcpyDeviceToHost));
    cudaFree(d_w);
    cudaFree(d_st);
    return st;
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

// Right-hand side and solve in one call: the right-hand side kernels run on
// the problem's auxiliary stream beside the factorisation on the context
// stream (the two are independent: the factor reads A, the right-hand side
// the rules, the node geometry and u_D), and the refinement waits for both.
// Buffers are allocated on the context stream before the fork; the scratch is
// freed on it after the join.
void solve_with_data(igs_prob p, const double* d_uD, int nrhs, double* d_alpha, double* resid) {
    cudaStream_t s = p->geom->ctx->stream;
    const Plan& P = p->plan;
    if (nrhs < 1 || nrhs > 8) throw Error(IGS_E_INVALID_ARG, "nrhs must be in [1, 8]");
    if (!p->aux_stream) IGS_CUDA(cudaStreamCreateWithFlags(&p->aux_stream, cudaStreamNonBlocking));
    cudaStream_t sr = p->aux_stream;
    if (!p->d_beta) p->d_beta = (double*)dev_alloc(p, sizeof(double) * (size_t)8 * P.n);
    p->rhs_n = nrhs;
    const int np = rhs_slots(p);
    double* scratch = np > 0 ? (double*)dev_alloc(p, sizeof(double) * (size_t)np * nrhs * P.Nq) : nullptr;
    cudaEvent_t ev[6] = {};
    bool forked = false;
    try {
        for (cudaEvent_t& e : ev) IGS_CUDA(cudaEventCreate(&e));
        IGS_CUDA(cudaEventRecord(ev[0], s));                 // fork: buffers and u_D are ready
        IGS_CUDA(cudaStreamWaitEvent(sr, ev[0], 0));
        forked = true;
        IGS_CUDA(cudaEventRecord(ev[1], sr));
        rhs_compute(p, d_uD, nrhs, p->d_beta, scratch, sr);
        IGS_CUDA(cudaEventRecord(ev[2], sr));                // join
        IGS_CUDA(cudaEventRecord(ev[3], s));
        const bool mixed = p->precision == IGS_MIXED;
        if (!p->factored) {
            if (mixed) prepare_factor<float>(p, s);
            else prepare_factor<double>(p, s);
        }
        IGS_CUDA(cudaEventRecord(ev[4], s));
        IGS_CUDA(cudaStreamWaitEvent(s, ev[2], 0));
        if (mixed) refine<float>(p, p->d_beta, nrhs, d_alpha, resid, s, 30, 1e-10);
        else refine<double>(p, p->d_beta, nrhs, d_alpha, resid, s, 1, 1e-10);
        IGS_CUDA(cudaEventRecord(ev[5], s));
        IGS_CUDA(cudaEventSynchronize(ev[5]));
        float r_ms = 0, f_ms = 0, s_ms = 0;
        cudaEventElapsedTime(&r_ms, ev[1], ev[2]);
        cudaEventElapsedTime(&f_ms, ev[3], ev[4]);
        cudaEventElapsedTime(&s_ms, ev[4], ev[5]);
        p->timing.rhs_ms = r_ms;
        p->timing.factor_ms = f_ms;
        p->timing.solve_ms = s_ms;
    } catch (...) {
        if (forked) cudaStreamSynchronize(sr);
        cudaStreamSynchronize(s);
        for (cudaEvent_t& e : ev)
            if (e) cudaEventDestroy(e);
        if (scratch) dev_free(p, scratch);
        throw;
    }
    for (cudaEvent_t& e : ev) cudaEventDestroy(e);
    if (scratch) dev_free(p, scratch);
}

}  // namespace igs
