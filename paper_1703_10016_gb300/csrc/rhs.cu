// Right-hand side (Sect. 5): b1_i = sum_n P[n,i] u_D(eta_n),
// b2_i = sum_n P[n,i] sum_g w_g Kbar(eta_n, t_g) u_D(t_g) with a composite Gauss
// rule of kGaussRhs points per refined element and
//   Kbar(s,t) = dK/dn_y(f(s), f(t)) J(t) = ((f(t)-f(s)) . (f2'(t), -f1'(t))) / |f(t)-f(s)|^2
// (outward normal of a counter-clockwise curve).  beta = b1/2 - b2/(2 pi) for the
// interior problem (eq. seconda_BIE), beta = b1 for an open arc (eq. prima_BIE).
//
// The double-layer potentials v_k(eta_m) = sum_g w_g Kbar(eta_m, t_g) u_k(t_g) are
// an N_quad x N_GQ kernel sum.  FP64 tier: every pair in FP64; the Gauss range
// is split in kSplit slices, one grid row each, so that every node has kSplit
// partial sums, added in a fixed order by k_beta.  MIXED tier: the same sum by
// a treecode (multipole moments of clusters of Gauss points, FP32 with
// float-float coordinate differences, truncation below the FP32 rounding),
// except at the Gauss points of the node's refined element and its two
// neighbours, where the numerator (f(t)-f(s)).n(t) is second-order small and
// k_double_layer_near adds the pairs in FP64.  Every sum runs in a fixed order:
// results do not depend on scheduling.
#include <mutex>

#include "igs_internal.h"

namespace igs {

constexpr int kMaxRhs = 8;
constexpr int kRhsChunk = 256;
constexpr int kSplit = 8;

__global__ void k_rhs_points(int M, int G, double a, double hf, const double* __restrict__ gx,
                             const double* __restrict__ gw, double* __restrict__ t, double* __restrict__ w) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= M * G) return;
    const int e = q / G, g = q % G;
    t[q] = a + hf * (e + gx[g]);
    w[q] = hf * gw[g];
}

__device__ __forceinline__ void split2(double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// FP32 double-layer kernel value of one pair from float-float coordinates; the
// operations are spelled out (no contraction) so that the far-field and near-
// field kernels compute identical bits.
__device__ __forceinline__ float kb32_pair(float gxh, float gxl, float gyh, float gyl, float a, float b, float xh,
                                           float xl, float yh, float yl) {
    const float dx = __fadd_rn(__fsub_rn(gxh, xh), __fsub_rn(gxl, xl));
    const float dy = __fadd_rn(__fsub_rn(gyh, yh), __fsub_rn(gyl, yl));
    const float num = __fmaf_rn(dy, b, __fmul_rn(dx, a));
    const float r2 = __fmaf_rn(dy, dy, __fmul_rn(dx, dx));
    return div_ftz(num, r2);
}

// MIXED tier: the double-layer sum by a treecode over the Gauss points.  In
// complex notation, with z = f(t) - f(s) and nu(t) = f2'(t) - i f1'(t),
// Kbar(s,t) = Re(nu / z), so v_k(eta) = Re sum_g c_g / (y_g - x) with charges
// c_g = w_g u_k(t_g) nu(t_g), y_g = f(t_g) and x = f(eta): a Cauchy sum.  The
// Gauss points, in parameter order, are grouped in leaves of kLeaf points and
// a binary tree of leaves; each cluster holds the scaled moments
//   M_j = sum_{g in cluster} c_g ((y_g - z_c) / rho)^j,  j < kTerms,
// about the centre z_c of its bounding box (rho = half its diagonal; the
// scaling keeps every moment within sum |c_g| in FP32).  For
// |x - z_c| >= rho / theta the cluster's share of the sum is
//   -(1 / (x - z_c)) sum_j M_j (rho / (x - z_c))^j,
// with a truncation error below theta^kTerms / (1 - theta) times
// sum |c_g| / |x - z_c| (theta = 1/2, kTerms = 28: 7.5e-9, under the FP32
// rounding of the sum itself).  The moments of a leaf are summed from its
// points, those of a parent by the binomial shift of its two children's:
// M^P_j = sum_l C(j, l) (rho_c / rho_P)^l M^c_l ((z_c - z_P) / rho_P)^(j - l),
// whose terms are bounded by 2^j sum |c_g| and enter the sum with weight at
// most theta^j = 2^-j.
// A warp takes 32 consecutive nodes and walks the tree from the root with one
// stack: a cluster is expanded for all 32 when every node is separated from
// it and none has its own or a neighbouring element in it, else its children
// are visited; leaves that are reached are summed point by point in FP32 with
// float-float coordinate differences (kb32_pair).  Every node thus gets every
// Gauss point once, except those of its element and its two neighbours,
// which k_double_layer_near adds in FP64.  All sums run in a fixed order.
constexpr int kLeaf = 32;
constexpr int kTerms = 28;
constexpr double kTheta = 0.5;

struct TreeArgs {
    int L, C;                          // levels (leaves = level 0), clusters
    int off[kTreeMaxLevels];           // first cluster of each level
    int cnt[kTreeMaxLevels];           // clusters per level
    const float4* ctr;                 // [C] centre, float-float (xh, xl, yh, yl)
    const float* thr;                  // [C] (rho / theta)^2
    const float* rs;                   // [C] moment scale rho (positive)
    const int2* erng;                  // [C] first and last refined element
    const float4* src;                 // [Ng] Gauss point, float-float (xh, xl, yh, yl)
    const float2* ab;                  // [Ng] (f2', -f1') at the Gauss point
};

__device__ __forceinline__ void tree_finish(const double* bx, float4& ctr, float& thr, float& rs) {
    const double cx = 0.5 * (bx[0] + bx[1]), cy = 0.5 * (bx[2] + bx[3]);
    const double hx = bx[1] - bx[0], hy = bx[3] - bx[2];
    const double rho2 = 0.25 * (hx * hx + hy * hy);
    float a, b, c, d;
    split2(cx, a, b);
    split2(cy, c, d);
    ctr = make_float4(a, b, c, d);
    // a small margin for the FP32 distance test; a positive floor for one-point clusters
    thr = (float)fmax(rho2 / (kTheta * kTheta) * (1.0 + 1e-4), 1e-30);
    rs = (float)fmax(sqrt(rho2), 1e-30);
}

// Leaves: bounding box, centre, threshold, element range, and the FP32 images
// of the Gauss points (coordinates as float-float, normal direction).
__global__ void k_tree_leaves(int Ng, int nleaf, const double* __restrict__ rgeo, double* __restrict__ box,
                              float4* __restrict__ ctr, float* __restrict__ thr, float* __restrict__ rs,
                              int2* __restrict__ erng, float4* __restrict__ src, float2* __restrict__ ab) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nleaf) return;
    const int g0 = c * kLeaf, g1 = min(Ng, g0 + kLeaf);
    double bx[4] = {rgeo[g0], rgeo[g0], rgeo[Ng + g0], rgeo[Ng + g0]};
    for (int g = g0; g < g1; ++g) {
        const double x = rgeo[g], y = rgeo[Ng + g];
        bx[0] = fmin(bx[0], x); bx[1] = fmax(bx[1], x);
        bx[2] = fmin(bx[2], y); bx[3] = fmax(bx[3], y);
        float4 q;
        split2(x, q.x, q.y);
        split2(y, q.z, q.w);
        src[g] = q;
        ab[g] = make_float2((float)rgeo[3 * Ng + g], (float)(-rgeo[2 * Ng + g]));
    }
    for (int k = 0; k < 4; ++k) box[4 * (size_t)c + k] = bx[k];
    tree_finish(bx, ctr[c], thr[c], rs[c]);
    erng[c] = make_int2(g0 / kGaussRhs, (g1 - 1) / kGaussRhs);
}

// One level up: a parent's box is the union of its children's.
__global__ void k_tree_up(int offc, int cntc, int offp, int cntp, double* __restrict__ box, float4* __restrict__ ctr,
                          float* __restrict__ thr, float* __restrict__ rs, int2* __restrict__ erng) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cntp) return;
    const int c0 = offc + 2 * i, c1 = (2 * i + 1 < cntc) ? c0 + 1 : c0;
    double bx[4];
    bx[0] = fmin(box[4 * (size_t)c0], box[4 * (size_t)c1]);
    bx[1] = fmax(box[4 * (size_t)c0 + 1], box[4 * (size_t)c1 + 1]);
    bx[2] = fmin(box[4 * (size_t)c0 + 2], box[4 * (size_t)c1 + 2]);
    bx[3] = fmax(box[4 * (size_t)c0 + 3], box[4 * (size_t)c1 + 3]);
    const int P = offp + i;
    for (int k = 0; k < 4; ++k) box[4 * (size_t)P + k] = bx[k];
    tree_finish(bx, ctr[P], thr[P], rs[P]);
    erng[P] = make_int2(erng[c0].x, erng[c1].y);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// 1 / (l + 1), l < kTerms: the binomial coefficients of the moment shift by a
// running product (uniform index across a warp: constant-cache broadcast).
__constant__ float c_recip[kTerms + 1] = {
    1.f / 1,  1.f / 2,  1.f / 3,  1.f / 4,  1.f / 5,  1.f / 6,  1.f / 7,  1.f / 8,  1.f / 9,  1.f / 10,
    1.f / 11, 1.f / 12, 1.f / 13, 1.f / 14, 1.f / 15, 1.f / 16, 1.f / 17, 1.f / 18, 1.f / 19, 1.f / 20,
    1.f / 21, 1.f / 22, 1.f / 23, 1.f / 24, 1.f / 25, 1.f / 26, 1.f / 27, 1.f / 28, 1.f / 29};

// Moments of leaf c for data set r, one warp, one lane per Gauss point: each
// lane forms c_g ((y_g - z_c) / rho)^j and the warp adds them by a fixed
// butterfly; lane j < kTerms returns M_j.  Writes the FP32 products
// w_g u_r(t_g) the direct sums use.
static_assert(kLeaf == 32, "one lane per Gauss point of a leaf");
__device__ __forceinline__ void leaf_moments_warp(int c, int r, int lane, int Ng, int C, const double* __restrict__ rgeo,
                                                  const double* __restrict__ rw, const double* __restrict__ uD,
                                                  int ldu, int off, const float4* __restrict__ ctr,
                                                  const float* __restrict__ rs, const float2* __restrict__ ab,
                                                  float2* __restrict__ mom, float* __restrict__ wu) {
    const float4 z = ctr[c];
    const double zx = (double)z.x + (double)z.y, zy = (double)z.z + (double)z.w;
    const float ir = 1.0f / rs[c];
    const int g = c * kLeaf + lane;
    float2 pw = make_float2(0.f, 0.f), t = make_float2(0.f, 0.f);
    if (g < Ng) {
        const float w = (float)(rw[g] * uD[(size_t)r * ldu + off + g]);
        wu[(size_t)r * Ng + g] = w;
        const float2 nu = ab[g];
        t = make_float2((float)(rgeo[g] - zx) * ir, (float)(rgeo[Ng + g] - zy) * ir);
        pw = make_float2(w * nu.x, w * nu.y);
    }
    float2 mine = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int j = 0; j < kTerms; ++j) {
        float sx = pw.x, sy = pw.y;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
        }
        if (lane == j) mine = make_float2(sx, sy);
        pw = cmul(pw, t);
    }
    if (lane < kTerms) mom[((size_t)r * C + c) * kTerms + lane] = mine;
}

// Moments of parent P (children c0 and, if c1 != c0, c1) for data set r, one
// warp, lane j for M^P_j: the sum over l by Horner's rule in
// tau = (z_c - z_P) / rho_P, l ascending, the children's moments broadcast
// from lane l.
__device__ __forceinline__ void shift_warp(int P, int c0, int c1, int r, int j, int C, const float4* __restrict__ ctr,
                                           const float* __restrict__ rs, float2* __restrict__ mom) {
    const float4 zp = ctr[P];
    const double px = (double)zp.x + (double)zp.y, py = (double)zp.z + (double)zp.w;
    const float irp = 1.0f / rs[P];
    float2 acc = make_float2(0.f, 0.f);
    for (int c = c0; c <= c1; ++c) {
        const float4 zc = ctr[c];
        const float2 tau = make_float2((float)((double)zc.x + (double)zc.y - px) * irp,
                                       (float)((double)zc.z + (double)zc.w - py) * irp);
        const float sig = rs[c] * irp;
        const float2 ml = j < kTerms ? mom[((size_t)r * C + c) * kTerms + j] : make_float2(0.f, 0.f);
        float2 sacc = make_float2(0.f, 0.f);
        float b = 1.f, sl = 1.f;                         // C(j, l), sig^l
#pragma unroll 4
        for (int l = 0; l < kTerms; ++l) {
            const float mx = __shfl_sync(0xffffffffu, ml.x, l), my = __shfl_sync(0xffffffffu, ml.y, l);
            if (l <= j) {
                const float f = b * sl;
                sacc = cmul(sacc, tau);
                sacc.x = fmaf(f, mx, sacc.x);
                sacc.y = fmaf(f, my, sacc.y);
                sl *= sig;
                b *= (float)(j - l) * c_recip[l];
            }
        }
        acc.x += sacc.x;
        acc.y += sacc.y;
    }
    if (j < kTerms) mom[((size_t)r * C + P) * kTerms + j] = acc;
}

// Leaves and the kSubLevels levels above them, one CTA per subtree of
// 2^kSubLevels leaves (one warp per leaf, then per parent; the levels are
// separated by block barriers, which also order the global moments).
constexpr int kSubLevels = 4;
constexpr int kSubLeaves = 1 << kSubLevels;
__global__ void __launch_bounds__(32 * kSubLeaves) k_tree_subtree(int Ng, int nrhs, TreeArgs T, const double* __restrict__ rgeo,
                                                                  const double* __restrict__ rw,
                                                                  const double* __restrict__ uD, int ldu, int off,
                                                                  float2* __restrict__ mom, float* __restrict__ wu) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * kSubLeaves + w;
    if (c < T.cnt[0])
        for (int r = 0; r < nrhs; ++r)
            leaf_moments_warp(c, r, lane, Ng, T.C, rgeo, rw, uD, ldu, off, T.ctr, T.rs, T.ab, mom, wu);
    for (int l = 1; l <= kSubLevels && l < T.L; ++l) {
        __syncthreads();
        const int per = kSubLeaves >> l;                 // parents of this subtree at level l
        const int i = blockIdx.x * per + w;
        if (w < per && i < T.cnt[l]) {
            const int c0 = T.off[l - 1] + 2 * i, c1 = (2 * i + 1 < T.cnt[l - 1]) ? c0 + 1 : c0;
            for (int r = 0; r < nrhs; ++r) shift_warp(T.off[l] + i, c0, c1, r, lane, T.C, T.ctr, T.rs, mom);
        }
    }
}

// One level of the moment shifts, one warp per (parent, r).
__global__ void __launch_bounds__(128) k_tree_shift(int l, int nrhs, TreeArgs T, float2* __restrict__ mom) {
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int cntp = T.cnt[l];
    const int i = wid % cntp, r = wid / cntp;
    if (r >= nrhs) return;                               // whole warps
    const int c0 = T.off[l - 1] + 2 * i, c1 = (2 * i + 1 < T.cnt[l - 1]) ? c0 + 1 : c0;
    shift_warp(T.off[l] + i, c0, c1, r, lane, T.C, T.ctr, T.rs, mom);
}

// The levels from l0 to the root in one CTA (each has at most 32 clusters):
// warps stride over (parent, r), levels separated by block barriers.
__global__ void __launch_bounds__(1024) k_tree_top(int l0, int nrhs, TreeArgs T, float2* __restrict__ mom) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int l = l0; l < T.L; ++l) {
        if (l > l0) __syncthreads();
        const int cntp = T.cnt[l];
        for (int it = w; it < cntp * nrhs; it += nw) {
            const int i = it % cntp, r = it / cntp;
            const int c0 = T.off[l - 1] + 2 * i, c1 = (2 * i + 1 < T.cnt[l - 1]) ? c0 + 1 : c0;
            shift_warp(T.off[l] + i, c0, c1, r, lane, T.C, T.ctr, T.rs, mom);
        }
    }
}

// The treecode sum at the nodes (warp per 32 consecutive nodes): out[r][m] =
// the FP32 double-layer potential of data set r at eta_m without the Gauss
// points of the node's element and its two neighbours.  A cluster's moments
// and a leaf's Gauss points are loaded once per warp (lane j holds M_j, lane g
// point g of the leaf) and passed to every lane by shuffles.
template <int NR>
__global__ void __launch_bounds__(128) k_tree_eval(int Nq, int Ng, int M, const double* __restrict__ geo,
                                                   const int* __restrict__ fspan, const TreeArgs T,
                                                   const float2* __restrict__ mom, const float* __restrict__ wu,
                                                   double* __restrict__ out) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31;
    const bool live = m < Nq;
    const int mm = live ? m : Nq - 1;
    float xh, xl, yh, yl;
    split2(geo[mm], xh, xl);
    split2(geo[Nq + mm], yh, yl);
    const int em = fspan[mm];
    const int ea = em == 0 ? M - 1 : em - 1, eb = em == M - 1 ? 0 : em + 1;
    float acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0.f;
    int stk[2 * kTreeMaxLevels + 2];
    int sp = 0;
    stk[sp++] = (T.L - 1) << 24;
    while (sp > 0) {
        const int e = stk[--sp];
        const int lvl = e >> 24, i = e & 0xffffff;
        const int id = T.off[lvl] + i;
        const float4 z = T.ctr[id];
        const int2 er = T.erng[id];
        const float dx = (xh - z.x) + (xl - z.y), dy = (yh - z.z) + (yl - z.w);
        const bool adj = (em >= er.x && em <= er.y) || (ea >= er.x && ea <= er.y) || (eb >= er.x && eb <= er.y);
        const float d2 = fmaf(dx, dx, dy * dy);
        if (__all_sync(0xffffffffu, !adj && d2 >= T.thr[id])) {
            // -Re (1/d) sum_j M_j (rho/d)^j, d = x - z_c, by Horner in rho/d
            const float inv = 1.0f / d2;
            const float2 w = make_float2(dx * inv, -dy * inv);          // 1 / d
            const float rsc = T.rs[id];
            const float2 v = make_float2(rsc * w.x, rsc * w.y);         // rho / d
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const float2 ml = lane < kTerms ? mom[((size_t)r * T.C + id) * kTerms + lane] : make_float2(0.f, 0.f);
                float2 sacc = make_float2(__shfl_sync(0xffffffffu, ml.x, kTerms - 1),
                                          __shfl_sync(0xffffffffu, ml.y, kTerms - 1));
#pragma unroll
                for (int j = kTerms - 2; j >= 0; --j) {
                    const float mx = __shfl_sync(0xffffffffu, ml.x, j), my = __shfl_sync(0xffffffffu, ml.y, j);
                    sacc = make_float2(fmaf(sacc.x, v.x, fmaf(-sacc.y, v.y, mx)), fmaf(sacc.x, v.y, fmaf(sacc.y, v.x, my)));
                }
                acc[r] -= fmaf(sacc.x, w.x, -sacc.y * w.y);
            }
        } else if (lvl == 0) {
            const int g0 = i * kLeaf, gl = g0 + lane;
            const bool have = gl < Ng;
            const float4 q = have ? T.src[gl] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float2 nu = have ? T.ab[gl] : make_float2(0.f, 0.f);
            float wl[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) wl[r] = have ? wu[(size_t)r * Ng + gl] : 0.f;
#pragma unroll 4
            for (int k = 0; k < kLeaf; ++k) {
                const float qx = __shfl_sync(0xffffffffu, q.x, k), qxl = __shfl_sync(0xffffffffu, q.y, k);
                const float qy = __shfl_sync(0xffffffffu, q.z, k), qyl = __shfl_sync(0xffffffffu, q.w, k);
                const float a = __shfl_sync(0xffffffffu, nu.x, k), b = __shfl_sync(0xffffffffu, nu.y, k);
                float wk[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) wk[r] = __shfl_sync(0xffffffffu, wl[r], k);
                const int eg = (g0 + k) / kGaussRhs;
                if (g0 + k < Ng && eg != em && eg != ea && eg != eb) {
                    const float kb = kb32_pair(qx, qxl, qy, qyl, a, b, xh, xl, yh, yl);
#pragma unroll
                    for (int r = 0; r < NR; ++r) acc[r] = fmaf(kb, wk[r], acc[r]);
                }
            }
        } else {
            const int cl = T.cnt[lvl - 1];
            if (2 * i + 1 < cl) stk[sp++] = ((lvl - 1) << 24) | (2 * i + 1);
            stk[sp++] = ((lvl - 1) << 24) | (2 * i);
        }
    }
    if (live) {
#pragma unroll
        for (int r = 0; r < NR; ++r) out[(size_t)r * Nq + m] = (double)acc[r];
    }
}

// FP64 tier: every pair in FP64, partial sums over Gauss slice blockIdx.y.
template <int NR>
__global__ void __launch_bounds__(256) k_double_layer_d(int Nq, int Ng, const double* __restrict__ geo,
                                                        const double* __restrict__ rgeo, const double* __restrict__ rw,
                                                        const double* __restrict__ uD, int ldu, int off,
                                                        double* __restrict__ part) {
    __shared__ double sx[kRhsChunk], sy[kRhsChunk], sa[kRhsChunk], sb[kRhsChunk];
    __shared__ double su[NR][kRhsChunk];
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = m < Nq;
    const double xm = live ? geo[m] : 0.0, ym = live ? geo[Nq + m] : 0.0;
    double acc[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) acc[k] = 0.0;
    const int per = (Ng + kSplit - 1) / kSplit;
    const int g_lo = blockIdx.y * per, g_hi = min(Ng, g_lo + per);
    for (int g0 = g_lo; g0 < g_hi; g0 += kRhsChunk) {
        const int cn = min(kRhsChunk, g_hi - g0);
        __syncthreads();
        for (int q = threadIdx.x; q < cn; q += blockDim.x) {
            const int g = g0 + q;
            sx[q] = rgeo[g]; sy[q] = rgeo[Ng + g]; sa[q] = rgeo[3 * Ng + g]; sb[q] = -rgeo[2 * Ng + g];
            const double w = rw[g];
#pragma unroll
            for (int k = 0; k < NR; ++k) su[k][q] = w * uD[(size_t)k * ldu + off + g];
        }
        __syncthreads();
        if (live) {
            for (int q = 0; q < cn; ++q) {
                const double dx = sx[q] - xm, dy = sy[q] - ym;
                const double kb = (dx * sa[q] + dy * sb[q]) / (dx * dx + dy * dy);
#pragma unroll
                for (int k = 0; k < NR; ++k) acc[k] += kb * su[k][q];
            }
        }
    }
    if (live) {
#pragma unroll
        for (int k = 0; k < NR; ++k) part[((size_t)blockIdx.y * NR + k) * Nq + m] = acc[k];
    }
}

// MIXED near field: the Gauss points of the node's element and its two
// neighbours, where the numerator (f(t)-f(s)).n(t) is second-order small and an
// FP32 value would be poor, in FP64, added to the treecode sum in `out`.
// kNearLanes consecutive lanes share a node (pairs j = lane, lane + kNearLanes,
// ... of the 3 kGaussRhs near pairs), reduced by a fixed shuffle tree.
constexpr int kNearLanes = 4;

__global__ void k_double_layer_near(int Nq, int Ng, int M, int nrhs, const double* __restrict__ geo,
                                    const int* __restrict__ fspan, const double* __restrict__ rgeo,
                                    const double* __restrict__ rw, const double* __restrict__ uD, int ldu, int off,
                                    double* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = t / kNearLanes, lane = t % kNearLanes;
    const bool live = m < Nq;
    const int mm = live ? m : Nq - 1;
    const double xm = geo[mm], ym = geo[Nq + mm];
    const int em = fspan[mm];
    double acc[kMaxRhs];
    for (int k = 0; k < kMaxRhs; ++k) acc[k] = 0.0;
    for (int j = lane; j < 3 * kGaussRhs; j += kNearLanes) {
        int e = em + j / kGaussRhs - 1;
        if (e < 0) e += M;
        if (e >= M) e -= M;
        const int g = e * kGaussRhs + j % kGaussRhs;
        const double dx = rgeo[g] - xm, dy = rgeo[Ng + g] - ym;
        const double kb = (dx * rgeo[3 * Ng + g] - dy * rgeo[2 * Ng + g]) / (dx * dx + dy * dy);
        const double w = rw[g];
        for (int k = 0; k < nrhs; ++k) acc[k] += kb * w * uD[(size_t)k * ldu + off + g];
    }
    for (int k = 0; k < nrhs; ++k) {
        double v = acc[k];
#pragma unroll
        for (int o = 1; o < kNearLanes; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (live && lane == 0) out[(size_t)k * Nq + m] += v;
    }
}

// beta[k][i] from the row weights P[m][r] = J_m w^(jfirst+r)_m over N^(i);
// v_k(eta_m) is the sum of the np partial slots (fixed order).  kBetaLanes
// consecutive lanes share a row (nodes lo + lane, lo + lane + kBetaLanes, ...),
// reduced by a fixed shuffle tree.
constexpr int kBetaLanes = 8;

__global__ void k_beta(int n, int Nq, int d, int nrhs, int closed, const int* __restrict__ lo, const int* __restrict__ hi,
                       const int* __restrict__ jfirst, const double* __restrict__ W, const double* __restrict__ geo,
                       const double* __restrict__ uD, int ldu, const double* __restrict__ part, int np,
                       double* __restrict__ beta) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / kBetaLanes, lane = t % kBetaLanes;
    const int k = blockIdx.y;
    const bool live = i < n && k < nrhs;
    double b1 = 0.0, b2 = 0.0;
    if (live) {
        for (int u = lo[i] + lane; u <= hi[i]; u += kBetaLanes) {
            int m = u % Nq;
            if (m < 0) m += Nq;
            const int iu = (u < 0) ? i + n : i;
            const int r = iu - jfirst[m];
            if (r < 0 || r > d) continue;
            const double p = geo[4 * Nq + m] * W[m * (d + 1) + r];
            b1 += p * uD[(size_t)k * ldu + m];
            if (closed) {
                double v = 0.0;
                for (int s = 0; s < np; ++s) v += part[((size_t)s * nrhs + k) * Nq + m];
                b2 += p * v;
            }
        }
    }
#pragma unroll
    for (int o = 1; o < kBetaLanes; o <<= 1) {
        b1 += __shfl_xor_sync(0xffffffffu, b1, o);
        b2 += __shfl_xor_sync(0xffffffffu, b2, o);
    }
    if (live && lane == 0) beta[(size_t)k * n + i] = closed ? 0.5 * b1 - b2 / (2.0 * kPi) : b1;
}

// Levels of the treecode: ceil(Ng / kLeaf) leaves, then halving to one root.
static void tree_plan(igs_prob p) {
    int* cnt = p->tree_cnt;
    int* off = p->tree_off;
    cnt[0] = (p->Ng + kLeaf - 1) / kLeaf;
    off[0] = 0;
    int L = 1, C = cnt[0];
    while (cnt[L - 1] > 1) {
        if (L == kTreeMaxLevels) throw Error(IGS_E_INVALID_ARG, "too many Gauss points for the treecode");
        cnt[L] = (cnt[L - 1] + 1) / 2;
        off[L] = C;
        C += cnt[L];
        ++L;
    }
    p->tree_L = L;
    p->tree_C = C;
}

// Byte offsets of the tree arrays in d_tree (16-byte aligned).
struct TreeLayout {
    size_t box, ctr, erng, thr, rs, src, ab, total;
};
static size_t up16(size_t b) { return (b + 15) & ~(size_t)15; }
static TreeLayout tree_layout(int C, int Ng) {
    TreeLayout t;
    t.box = 0;
    t.ctr = up16(t.box + sizeof(double) * 4 * (size_t)C);
    t.erng = up16(t.ctr + sizeof(float4) * (size_t)C);
    t.thr = up16(t.erng + sizeof(int2) * (size_t)C);
    t.rs = up16(t.thr + sizeof(float) * (size_t)C);
    t.src = up16(t.rs + sizeof(float) * (size_t)C);
    t.ab = up16(t.src + sizeof(float4) * (size_t)Ng);
    t.total = up16(t.ab + sizeof(float2) * (size_t)Ng);
    return t;
}

static TreeArgs tree_args(const igs_prob p) {
    const TreeLayout t = tree_layout(p->tree_C, p->Ng);
    unsigned char* b = (unsigned char*)p->d_tree;
    TreeArgs a;
    a.L = p->tree_L;
    a.C = p->tree_C;
    for (int l = 0; l < kTreeMaxLevels; ++l) {
        a.off[l] = p->tree_off[l];
        a.cnt[l] = p->tree_cnt[l];
    }
    a.ctr = (const float4*)(b + t.ctr);
    a.thr = (const float*)(b + t.thr);
    a.rs = (const float*)(b + t.rs);
    a.erng = (const int2*)(b + t.erng);
    a.src = (const float4*)(b + t.src);
    a.ab = (const float2*)(b + t.ab);
    return a;
}

// Cluster geometry of the treecode from the Gauss points (after any change of
// the geometry; no allocation).
void rhs_tree_geometry(igs_prob p, cudaStream_t s) {
    if (!p->d_tree) return;
    const TreeLayout t = tree_layout(p->tree_C, p->Ng);
    unsigned char* b = (unsigned char*)p->d_tree;
    double* box = (double*)(b + t.box);
    float4* ctr = (float4*)(b + t.ctr);
    float* thr = (float*)(b + t.thr);
    float* rs = (float*)(b + t.rs);
    int2* erng = (int2*)(b + t.erng);
    const int nleaf = p->tree_cnt[0];
    k_tree_leaves<<<(nleaf + 127) / 128, 128, 0, s>>>(p->Ng, nleaf, p->d_rhs_geo, box, ctr, thr, rs, erng,
                                                      (float4*)(b + t.src), (float2*)(b + t.ab));
    for (int l = 1; l < p->tree_L; ++l)
        k_tree_up<<<(p->tree_cnt[l] + 127) / 128, 128, 0, s>>>(p->tree_off[l - 1], p->tree_cnt[l - 1], p->tree_off[l],
                                                               p->tree_cnt[l], box, ctr, thr, rs, erng);
    IGS_CUDA(cudaGetLastError());
    p->launches += p->tree_L;
}

// Doubles of per-call scratch one data set needs beside its N_quad potentials
// (MIXED tier): the moments (kTerms float2 per cluster) and the FP32 w u_D
// products at the Gauss points.
static size_t tree_scratch_doubles(const igs_prob p) {
    const int Ng = p->plan.M * kGaussRhs;
    size_t C = 0;
    for (int c = (Ng + kLeaf - 1) / kLeaf;; c = (c + 1) / 2) {
        C += c;
        if (c <= 1) break;
    }
    return C * kTerms + ((size_t)Ng + 1) / 2;
}

void rhs_prepare(igs_prob p) {
    // Gauss points of the b2 inner rule and the geometry there
    const Plan& P = p->plan;
    if (p->d_rhs_geo) return;
    cudaStream_t s = p->geom->ctx->stream;
    const int G = kGaussRhs;
    p->Ng = P.M * G;
    double gx[kGaussRhs], gw[kGaussRhs];
    for (int k = 0; k < G; ++k) {
        double x = cos(kPi * (k + 0.75) / (G + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1, p1 = x;
            for (int q = 2; q <= G; ++q) { double p2 = ((2 * q - 1) * x * p1 - (q - 1) * p0) / q; p0 = p1; p1 = p2; }
            double dp = G * (x * p1 - p0) / (x * x - 1);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        double p0 = 1, p1 = x;
        for (int q = 2; q <= G; ++q) { double p2 = ((2 * q - 1) * x * p1 - (q - 1) * p0) / q; p0 = p1; p1 = p2; }
        double dp = G * (x * p1 - p0) / (x * x - 1);
        gx[G - 1 - k] = (1.0 + x) / 2.0;
        gw[G - 1 - k] = 1.0 / ((1 - x * x) * dp * dp);
    }
    double* d_g = (double*)dev_alloc(p, sizeof(double) * 2 * G);
    IGS_CUDA(cudaMemcpyAsync(d_g, gx, sizeof(gx), cudaMemcpyHostToDevice, s));
    IGS_CUDA(cudaMemcpyAsync(d_g + G, gw, sizeof(gw), cudaMemcpyHostToDevice, s));
    p->d_rhs_t = (double*)dev_alloc(p, sizeof(double) * p->Ng);
    p->d_rhs_w = (double*)dev_alloc(p, sizeof(double) * p->Ng);
    p->d_rhs_geo = (double*)dev_alloc(p, sizeof(double) * 5 * p->Ng);
    k_rhs_points<<<(p->Ng + 255) / 256, 256, 0, s>>>(P.M, G, P.a, P.hf, d_g, d_g + G, p->d_rhs_t, p->d_rhs_w);
    IGS_CUDA(cudaGetLastError());
    geometry_eval(p->geom, p->d_rhs_t, p->Ng, p->d_rhs_geo, s);
    p->launches += 2;
    if (P.closed && p->precision == IGS_MIXED) {
        tree_plan(p);
        p->d_tree = dev_alloc(p, tree_layout(p->tree_C, p->Ng).total);
        rhs_tree_geometry(p, s);
    }
    IGS_CUDA(cudaStreamSynchronize(s));
    dev_free(p, d_g);
}

// Number of partial-sum slots (each nrhs x N_quad doubles) the kernels need.
int rhs_slots(const igs_prob p) {
    if (!p->plan.closed) return 0;
    if (p->precision == IGS_MIXED) {
        const size_t Nq = (size_t)p->plan.Nq;
        return 1 + (int)((tree_scratch_doubles(p) + Nq - 1) / Nq);
    }
    return kSplit;
}

// FP64 tier: kSplit partial sums of every pair.
template <int NR>
static void launch_far_d(igs_prob p, const double* d_uD, int ldu, double* part, cudaStream_t s) {
    const Plan& P = p->plan;
    k_double_layer_d<NR><<<dim3((P.Nq + 255) / 256, kSplit), 256, 0, s>>>(P.Nq, p->Ng, p->d_geo, p->d_rhs_geo,
                                                                        p->d_rhs_w, d_uD, ldu, P.Nq, part);
    IGS_CUDA(cudaGetLastError());
}

// MIXED tier: treecode sum into out[nrhs][N_quad], moments and w u_D products
// in `work` (tree_scratch_doubles per data set).
template <int NR>
static void launch_tree(igs_prob p, const double* d_uD, int ldu, double* out, double* work, cudaStream_t s) {
    const Plan& P = p->plan;
    const TreeArgs T = tree_args(p);
    float2* mom = (float2*)work;
    float* wu = (float*)(work + (size_t)NR * T.C * kTerms);
    // leaves and kSubLevels levels per subtree; one launch per level while a
    // level has more than 32 clusters; the rest to the root in one CTA
    k_tree_subtree<<<(T.cnt[0] + kSubLeaves - 1) / kSubLeaves, 32 * kSubLeaves, 0, s>>>(
        p->Ng, NR, T, p->d_rhs_geo, p->d_rhs_w, d_uD, ldu, P.Nq, mom, wu);
    int l = kSubLevels + 1, launches = 1;
    for (; l < T.L && T.cnt[l] > 32; ++l, ++launches)
        k_tree_shift<<<(T.cnt[l] * NR + 3) / 4, 128, 0, s>>>(l, NR, T, mom);
    if (l < T.L) {
        k_tree_top<<<1, 1024, 0, s>>>(l, NR, T, mom);
        ++launches;
    }
    k_tree_eval<NR><<<(P.Nq + 127) / 128, 128, 0, s>>>(P.Nq, p->Ng, P.M, p->d_geo, p->d_fspan, T, mom, wu, out);
    IGS_CUDA(cudaGetLastError());
    p->launches += launches + 1;
}

// Double-layer potentials v_k(eta_m) at the nodes of a closed curve, as
// partial sums in `scratch` (rhs_slots x nrhs x N_quad doubles): v_k(eta_m) is
// the sum over s < *np of vsum[(s nrhs + k) N_quad + m], in that order.
void rhs_node_potentials(igs_prob p, const double* d_uD, int nrhs, double* scratch, const double** vsum, int* np,
                         cudaStream_t s) {
    const Plan& P = p->plan;
    const int ldu = P.Nq + p->Ng;
    *vsum = scratch;
    if (p->precision == IGS_MIXED) {
        // the whole potential in the first nrhs x N_quad doubles: treecode, then the FP64 near pairs
        double* work = scratch + (size_t)nrhs * P.Nq;
        switch (nrhs) {
            case 1: launch_tree<1>(p, d_uD, ldu, scratch, work, s); break;
            case 2: launch_tree<2>(p, d_uD, ldu, scratch, work, s); break;
            case 3: launch_tree<3>(p, d_uD, ldu, scratch, work, s); break;
            case 4: launch_tree<4>(p, d_uD, ldu, scratch, work, s); break;
            case 5: launch_tree<5>(p, d_uD, ldu, scratch, work, s); break;
            case 6: launch_tree<6>(p, d_uD, ldu, scratch, work, s); break;
            case 7: launch_tree<7>(p, d_uD, ldu, scratch, work, s); break;
            default: launch_tree<8>(p, d_uD, ldu, scratch, work, s); break;
        }
        const int nt = P.Nq * kNearLanes;
        k_double_layer_near<<<(nt + 127) / 128, 128, 0, s>>>(P.Nq, p->Ng, P.M, nrhs, p->d_geo, p->d_fspan,
                                                             p->d_rhs_geo, p->d_rhs_w, d_uD, ldu, P.Nq, scratch);
        IGS_CUDA(cudaGetLastError());
        p->launches++;
        *np = 1;
        return;
    }
    *np = kSplit;
    switch (nrhs) {
        case 1: launch_far_d<1>(p, d_uD, ldu, scratch, s); break;
        case 2: launch_far_d<2>(p, d_uD, ldu, scratch, s); break;
        case 3: launch_far_d<3>(p, d_uD, ldu, scratch, s); break;
        case 4: launch_far_d<4>(p, d_uD, ldu, scratch, s); break;
        case 5: launch_far_d<5>(p, d_uD, ldu, scratch, s); break;
        case 6: launch_far_d<6>(p, d_uD, ldu, scratch, s); break;
        case 7: launch_far_d<7>(p, d_uD, ldu, scratch, s); break;
        default: launch_far_d<8>(p, d_uD, ldu, scratch, s); break;
    }
    p->launches++;
}

// beta for nrhs data sets into d_beta, partial sums in `scratch` (rhs_slots x nrhs x N_quad doubles),
// every kernel on stream s.
void rhs_compute(igs_prob p, const double* d_uD, int nrhs, double* d_beta, double* scratch, cudaStream_t s) {
    const Plan& P = p->plan;
    const int ldu = P.Nq + p->Ng;
    int np = 0;
    const double* vsum = scratch;
    if (P.closed) rhs_node_potentials(p, d_uD, nrhs, scratch, &vsum, &np, s);
    dim3 grid((P.n * kBetaLanes + 127) / 128, nrhs);
    k_beta<<<grid, 128, 0, s>>>(P.n, P.Nq, P.d, nrhs, P.closed, p->d_lo, p->d_hi, p->d_jfirst, p->d_W, p->d_geo, d_uD,
                                ldu, vsum, np, d_beta);
    IGS_CUDA(cudaGetLastError());
    p->launches++;
}

void rhs_build(igs_prob p, const double* d_uD, int nrhs) {
    const Plan& P = p->plan;
    cudaStream_t s = p->geom->ctx->stream;
    if (nrhs < 1 || nrhs > kMaxRhs) throw Error(IGS_E_INVALID_ARG, "nrhs must be in [1, 8]");
    double* scratch = nullptr;
    const int np = rhs_slots(p);
    if (np > 0) scratch = (double*)dev_alloc(p, sizeof(double) * (size_t)np * nrhs * P.Nq);
    if (p->d_beta && p->rhs_n < nrhs) dev_free(p, p->d_beta);
    if (!p->d_beta) p->d_beta = (double*)dev_alloc(p, sizeof(double) * (size_t)kMaxRhs * P.n);
    p->rhs_n = nrhs;
    rhs_compute(p, d_uD, nrhs, p->d_beta, scratch, s);
    if (scratch) {
        IGS_CUDA(cudaStreamSynchronize(s));
        dev_free(p, scratch);
    }
}

// ------------------------------------------------------------ no-allocation variant
// Some callers cannot allocate device memory inside a call: a host framework
// that owns all device memory through its own allocator and forbids others
// (custom-call handlers, memory-pool managed serving loops), code that must
// stay off the driver's allocator for latency reasons, or code that runs while
// someone else captures the stream.  For them igs_build_rhs_noalloc runs the
// same kernels as igs_build_rhs (double-layer potentials at the nodes, then
// the weighted sums b1 / b2) with the partial sums of the potentials kept in
// this fixed, file-scope device array instead of a buffer from cudaMallocAsync.
// Every GPU that loads the library holds the array until the process exits.
// All calls share it, so calls that overlap on the GPU (two streams, two host
// threads) race on it; it keeps the last call's contents, and nothing in it
// needs to start at zero because the kernels overwrite every entry they read.
constexpr size_t kNoAllocScratchDoubles = size_t(1) << 21;       // 16 MiB
static __device__ __align__(256) double g_rhs_scratch[kNoAllocScratchDoubles];

static std::mutex g_scratch_mu;
static double* g_scratch_addr[256] = {};

// Device address of g_rhs_scratch on `device` (which must be current).  In
// host code the symbol g_rhs_scratch is only a host-side stand-in, so the
// address is queried once per device with cudaGetSymbolAddress and cached.
static double* scratch_address(int device) {
    if (device < 0 || device >= 256) throw Error(IGS_E_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[device]) {
        void* ptr = nullptr;
        IGS_CUDA(cudaGetSymbolAddress(&ptr, g_rhs_scratch));
        g_scratch_addr[device] = (double*)ptr;
    }
    return g_scratch_addr[device];
}

void rhs_build_noalloc(igs_prob p, const double* d_uD, int nrhs, double* d_beta) {
    const Plan& P = p->plan;
    if (nrhs < 1 || nrhs > kMaxRhs) throw Error(IGS_E_INVALID_ARG, "nrhs must be in [1, 8]");
    if (!p->rules_ready || !p->geometry_ready || !p->d_rhs_geo)
        throw Error(IGS_E_STATE, "igs_build_rhs_noalloc needs the rules, the node geometry and the rhs points: "
                                 "call igs_assemble and igs_rhs_points first");
    const int slots = rhs_slots(p);
    const size_t need = (size_t)slots * nrhs * P.Nq;
    if (need > kNoAllocScratchDoubles)
        throw Error(IGS_E_INVALID_ARG, "igs_build_rhs_noalloc: needs " + std::to_string(need) + " scratch doubles (" +
                                           std::to_string(slots) + " slots x n_quad " + std::to_string(P.Nq) +
                                           " x nrhs " + std::to_string(nrhs) + "), more than the fixed " +
                                           std::to_string(kNoAllocScratchDoubles));
    double* scratch = scratch_address(p->geom->ctx->device);
    rhs_compute(p, d_uD, nrhs, d_beta, scratch, p->geom->ctx->stream);
}

}  // namespace igs
