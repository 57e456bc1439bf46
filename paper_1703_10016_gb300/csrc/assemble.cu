// Fused assembly of A = -(I_K1 + I_K2)/(2 pi) (Sect. 5, eqs. IK1e2 and IK1e2_bis).
//
// With P = diag(J(eta)) W (regular rules, Algorithm 1), Q = diag(J(eta)) B_test and
// the singular rules W^s (Algorithm 2):
//     I_K1 = P^T C0 P,  C0[a,b] = K1(eta_a, eta_b)          (eq. IK1e2)
//     I_K2 = P^T W^s Q                                       (eq. IK1e2_bis)
// so A = -(1/2pi) P^T (C0 P + W^s Q).  One CTA owns a TILE x TILE block of A;
// the node ranges of its rows (A-range) and columns (B-range) follow from the
// index sets N^(i).  Stage 1 (sum factorisation, cf. Algorithm 3): each thread
// owns one A-range node a and walks the B-range in order, evaluating the kernel
// K1(eta_a, eta_b) on the fly and accumulating S1[a][j] = sum_b C0 P + W^s Q in a
// sliding register window of the d+1 columns j whose support holds b.  Stage 2
// contracts S1 with the row weights P.  C0 is never stored.
//
// K1 = ln|f(s)-f(t)| - K2(s,t) is evaluated as (1/2) ln(|f(s)-f(t)|^2 / D(t-s)^2)
// with D = exp(K2): D(x) = |x| (open arc) or |x| |x+L| |x-L| / L^2 (closed
// curve, three-image log).  The factors x+L and L-x are formed as
// eta_b + (L - eta_a) and (L - eta_b) + eta_a, sums of non-negative numbers, so
// the corner region keeps full relative accuracy.  In the FP32 tier the node
// coordinates are float-float pairs: the differences are taken hi-hi plus lo-lo,
// which keeps their relative error at FP32 rounding even for adjacent nodes.
// Limits (eq. F1_lim and the corner limit): K1(s,s) = ln J(s);
// K1(a,b) = K1(b,a) = ln J - ln 2 on a closed curve.
#include "bspline_dev.cuh"
#include "igs_internal.h"

namespace igs {

constexpr int kTile = 32;

struct NodeD { double x, y, e, eb, lnJ; };

template <typename T> struct NodeOf;
template <> struct NodeOf<double> { using type = NodeD; };
template <> struct NodeOf<float> { using type = NodeF; };

__global__ void k_prep_d(int Nq, int d, double L, const double* __restrict__ geo, const double* __restrict__ eta,
                         const double* __restrict__ W, const double* __restrict__ Bt, NodeD* __restrict__ nodes,
                         double* __restrict__ P, double* __restrict__ Q) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Nq) return;
    const double J = geo[4 * Nq + m];
    NodeD r;
    r.x = geo[m]; r.y = geo[Nq + m]; r.e = eta[m] - eta[0]; r.eb = L - r.e; r.lnJ = log(J);
    if (m == Nq - 1) { r.e = L; r.eb = 0.0; }
    if (m == 0) { r.e = 0.0; r.eb = L; }
    nodes[m] = r;
    for (int k = 0; k <= d; ++k) {
        P[m * (d + 1) + k] = J * W[m * (d + 1) + k];
        Q[m * (d + 1) + k] = J * Bt[m * (d + 1) + k];
    }
}

__device__ __forceinline__ void split(double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// FP32-tier node record and weights of node m (float-float coordinates and
// parameter offsets, both divided by the parameter length L, ln J, P = J W,
// Q = J B_test).  The common factor 1/L leaves |f(s) - f(t)| / D unchanged and
// turns the three-image factor's 1/L^2 into 1.
__device__ __forceinline__ void prep_f_node(int m, int Nq, int d, double L, const double* __restrict__ geo,
                                            const double* __restrict__ eta, const double* __restrict__ W,
                                            const double* __restrict__ Bt, NodeF* __restrict__ nodes,
                                            float* __restrict__ P, float* __restrict__ Q) {
    const double J = geo[4 * (size_t)Nq + m];
    double e = eta[m] - eta[0], eb = L - e;
    if (m == Nq - 1) { e = L; eb = 0.0; }
    if (m == 0) { e = 0.0; eb = L; }
    const double s = 1.0 / L;
    NodeF r;
    split(geo[m] * s, r.xh, r.xl);
    split(geo[Nq + m] * s, r.yh, r.yl);
    split(e * s, r.eh, r.el);
    split(eb * s, r.ebh, r.ebl);
    r.lnJ = (float)log(J);
    nodes[m] = r;
    for (int k = 0; k <= d; ++k) {
        P[m * (d + 1) + k] = (float)(J * W[m * (d + 1) + k]);
        Q[m * (d + 1) + k] = (float)(J * Bt[m * (d + 1) + k]);
    }
}

__global__ void k_prep_f(int Nq, int d, double L, const double* __restrict__ geo, const double* __restrict__ eta,
                         const double* __restrict__ W, const double* __restrict__ Bt, NodeF* __restrict__ nodes,
                         float* __restrict__ P, float* __restrict__ Q) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Nq) return;
    prep_f_node(m, Nq, d, L, geo, eta, W, Bt, nodes, P, Q);
}

// K1 between two distinct, non-corner nodes.
__device__ __forceinline__ double k1_pair(const NodeD& a, const NodeD& b, int closed, double invL2) {
    const double dx = b.x - a.x, dy = b.y - a.y;
    double D = fabs(b.e - a.e);
    if (closed) D *= (b.e + a.eb) * (b.eb + a.e) * invL2;
    return 0.5 * log((dx * dx + dy * dy) / (D * D));
}
__device__ __forceinline__ float k1_pair(const NodeF& a, const NodeF& b, int closed, float invL2) {
    const float dx = (b.xh - a.xh) + (b.xl - a.xl);
    const float dy = (b.yh - a.yh) + (b.yl - a.yl);
    float D = fabsf((b.eh - a.eh) + (b.el - a.el));
    if (closed) D *= ((b.eh + a.ebh) + (b.el + a.ebl)) * ((b.ebh + a.eh) + (b.ebl + a.el)) * invL2;
    return 0.5f * logf((dx * dx + dy * dy) / (D * D));
}

__device__ __forceinline__ int pmod(int u, int N) {
    int m = u % N;
    return m < 0 ? m + N : m;
}
__device__ __forceinline__ int pdiv(int u, int N) {   // floor(u / N)
    return (u >= 0) ? u / N : -((-u + N - 1) / N);
}

template <typename T, int D>
__global__ void __launch_bounds__(256) k_assemble_tile(
    int n, int Nq, int closed, T invL2, const int* __restrict__ lo, const int* __restrict__ hi,
    const int* __restrict__ jfirst, const typename NodeOf<T>::type* __restrict__ nodes, const T* __restrict__ P,
    const T* __restrict__ Q, const WsView<T> wsv, T* __restrict__ A, T* __restrict__ AT, int64_t ld, int maxr) {
    using Node = typename NodeOf<T>::type;
    constexpr int D1 = D + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    const int i0 = blockIdx.y * kTile, j0 = blockIdx.x * kTile;
    const int ni = min(kTile, n - i0), nj = min(kTile, n - j0);
    const int uA0 = lo[i0], Na = hi[i0 + ni - 1] - uA0 + 1;
    const int uB0 = lo[j0], Nb = hi[j0 + nj - 1] - uB0 + 1;
    // shared layout
    Node* sB = (Node*)smem;
    T* sPB = (T*)(sB + maxr);
    T* sQB = sPB + maxr * D1;
    T* sPA = sQB + maxr * D1;
    T* sS1 = sPA + maxr * D1;                         // [maxr][kTile + 1]
    int* sJB = (int*)(sS1 + maxr * (kTile + 1));
    int* sMB = sJB + maxr;
    int* sJA = sMB + maxr;

    for (int v = threadIdx.x; v < Nb; v += blockDim.x) {
        const int u = uB0 + v, m = pmod(u, Nq), per = pdiv(u, Nq);
        sB[v] = nodes[m];
        sMB[v] = m;
        sJB[v] = jfirst[m] + n * per - j0;
        for (int r = 0; r < D1; ++r) { sPB[v * D1 + r] = P[m * D1 + r]; sQB[v * D1 + r] = Q[m * D1 + r]; }
    }
    for (int v = threadIdx.x; v < Na; v += blockDim.x) {
        const int u = uA0 + v, m = pmod(u, Nq), per = pdiv(u, Nq);
        sJA[v] = jfirst[m] + n * per - i0;
        for (int r = 0; r < D1; ++r) sPA[v * D1 + r] = P[m * D1 + r];
    }
    __syncthreads();

    const T ln2 = (T)0.69314718055994530942;
    for (int a = threadIdx.x; a < Na; a += blockDim.x) {
        const int ma = pmod(uA0 + a, Nq);
        const Node na = nodes[ma];
        T acc[D1];
#pragma unroll
        for (int r = 0; r < D1; ++r) acc[r] = (T)0;
        int jcur = sJB[0];
        T* row = sS1 + a * (kTile + 1);
        for (int v = 0; v < Nb; ++v) {
            const int jf = sJB[v];
            while (jcur < jf) {
                if (jcur >= 0 && jcur < nj) row[jcur] = acc[0];
#pragma unroll
                for (int r = 0; r < D; ++r) acc[r] = acc[r + 1];
                acc[D] = (T)0;
                ++jcur;
            }
            const int mb = sMB[v];
            T c0;
            if (mb == ma) c0 = na.lnJ;
            else if (closed && (ma + mb == Nq - 1) && (ma == 0 || mb == 0)) c0 = na.lnJ - ln2;
            else c0 = k1_pair(na, sB[v], closed, invL2);
            const T ws = ws_at(wsv, ma, mb);
#pragma unroll
            for (int r = 0; r < D1; ++r) acc[r] += sPB[v * D1 + r] * c0 + sQB[v * D1 + r] * ws;
        }
#pragma unroll
        for (int r = 0; r < D1; ++r)
            if (jcur + r >= 0 && jcur + r < nj) row[jcur + r] = acc[r];
    }
    __syncthreads();

    const T scale = (T)(-1.0 / (2.0 * kPi));
    for (int idx = threadIdx.x; idx < ni * nj; idx += blockDim.x) {
        const int il = idx / nj, jl = idx % nj;
        const int i = i0 + il;
        const int a0 = lo[i] - uA0, a1 = hi[i] - uA0;
        T s = (T)0;
        for (int a = a0; a <= a1; ++a) {
            const int r = il - sJA[a];
            if (r >= 0 && r <= D) s += sPA[a * D1 + r] * sS1[a * (kTile + 1) + jl];
        }
        A[(size_t)i * ld + j0 + jl] = scale * s;
        if (AT) AT[(size_t)(j0 + jl) * ld + i] = scale * s;
    }
}

// FP32 tier, one thread per A-range node: the block is as wide as the largest
// node range (rounded up to a warp), so that no thread idles in stage 1.  Each
// B-range node is one shared-memory record of 3 + NW 16-byte words read by
// broadcast -- coordinates, parameter offsets, the P and Q weight rows and the
// indices (m, first column, Toeplitz offset) -- so one pointer addresses all of
// a node's data.  The nodes are walked in groups of equal first column, so
// that the window of d+1 running sums moves once per group, two nodes per step
// (interior groups hold 2 N_ref nodes).  The kernel value is formed in base-2
// units, c = log2(|f(s) - f(t)|^2 / D^2) = 2 K1 / ln 2, on node coordinates
// scaled by 1/L (which leaves the ratio unchanged and removes the 1/L^2 of the
// three-image factor); the factor ln 2 / 2 rides on the staged regular weights
// P.  The ratio is of order J^2 on these curves, and the hardware base-2
// logarithm (lg2.approx) measured on this GPU has an absolute error of at most
// 3.3e-7 for arguments in [1/16, 16] (2.1e-7 in [1/2, 2]).  Tiles whose nodes all
// lie where W^s is a Toeplitz sequence (interior columns and rows of the stored
// rules) stage the window of the two sequences they touch, so the singular
// weight is one shared-memory read at a per-node offset; the other tiles read
// the stored rules through ws_at, fetched a few steps ahead.  Only tiles whose
// A- and B-ranges share a node test for the diagonal limit.  Far tiles (the
// bounding boxes of the A- and B-range nodes at least twice the larger box
// diagonal apart, most tiles of a large problem) take the coordinate and
// parameter differences in plain FP32 from positions relative to the tile's
// first B node: every relative position is off by at most eps times its size,
// and the sizes are at most the difference plus one box diagonal, so the
// difference keeps a relative error below 3 eps (float-float keeps about 1 eps);
// three additions per pair instead of nine.
// 16-byte words of the P ln2/2 and Q rows of a node, packed back to back
template <int D> __host__ __device__ constexpr int wt_words() { return (2 * (D + 1) + 3) / 4; }
template <int D> __host__ __device__ constexpr int rec_words() { return 3 + wt_words<D>(); }

template <int D, bool CLOSED, bool TOE, bool DIAG, bool FAR>
__device__ __forceinline__ void tile_walk_f(const TileF& t, int ma, int a, int Nb, int nj,
                                            const float4* __restrict__ rec, const int* __restrict__ sGs,
                                            const float* __restrict__ sT, float* __restrict__ row, const NodeF& org) {
    constexpr int D1 = D + 1;
    constexpr int NW = wt_words<D>();
    constexpr int RW = rec_words<D>();
    const NodeF na = t.nodes[ma];
    // this node relative to the tile's first B node (far tiles)
    const float xr = (na.xh - org.xh) + (na.xl - org.xl), yr = (na.yh - org.yh) + (na.yl - org.yl);
    const float er = (na.eh - org.eh) + (na.el - org.el);
    const float cdiag = na.lnJ * 2.88539008177792681f;    // K1(s,s) = ln J in base-2 units (x 2 / ln 2)
    const float ccorner = cdiag - 2.0f;                    // ln J - ln 2 in the same units
    float acc[D1];
#pragma unroll
    for (int r = 0; r < D1; ++r) acc[r] = 0.0f;
    auto idx = [&](int v) { return *reinterpret_cast<const int4*>(&rec[v * RW + RW - 1]); };
    int jcur = idx(0).y;
    const int G = idx(Nb - 1).y - jcur + 1;
    constexpr int kPre = TOE ? 1 : 4;                      // singular weights in flight (general tiles)
    float wq[kPre];
    if (!TOE) {
#pragma unroll
        for (int q = 0; q < kPre; ++q) wq[q] = (q < Nb) ? ws_at(t.ws, ma, idx(q).x) : 0.0f;
    }
    auto node = [&](int v) {
        const float4* p = rec + v * RW;
        const int4 br = *reinterpret_cast<const int4*>(&p[RW - 1]);
        float ws;
        if (TOE) {
            ws = sT[br.z + a];
        } else {
            ws = wq[0];
#pragma unroll
            for (int q = 0; q < kPre - 1; ++q) wq[q] = wq[q + 1];
            wq[kPre - 1] = (v + kPre < Nb) ? ws_at(t.ws, ma, idx(v + kPre).x) : 0.0f;
        }
        float dx, dy, Dd, eb, ebb;                     // eb, ebb: high parts of x and L - x at node b
        if (FAR) {
            const float4 gr = p[0];
            dx = gr.x - xr;
            dy = gr.y - yr;
            Dd = gr.z - er;
            eb = gr.w;
            ebb = __int_as_float(br.w);
        } else {
            const float4 g0 = p[0], g1 = p[1];
            dx = (g0.x - na.xh) + (g0.y - na.xl);
            dy = (g0.z - na.yh) + (g0.w - na.yl);
            Dd = (g1.x - na.eh) + (g1.y - na.el);
            eb = g1.x;
            ebb = g1.z;
        }
        // x + L and L - x as sums of non-negative numbers: the high parts
        // alone keep FP32 relative accuracy
        if (CLOSED) Dd *= (eb + na.ebh) * (ebb + na.eh);
        float c0 = lg2_ftz(div_ftz(fmaf(dx, dx, dy * dy), Dd * Dd));
        if (DIAG) c0 = (br.x == ma) ? cdiag : c0;
        if (CLOSED && !TOE) c0 = (ma + br.x == t.Nq - 1 && (ma == 0 || br.x == 0)) ? ccorner : c0;
        float w[4 * NW];
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            const float4 t4 = p[2 + q];
            w[4 * q] = t4.x; w[4 * q + 1] = t4.y; w[4 * q + 2] = t4.z; w[4 * q + 3] = t4.w;
        }
#pragma unroll
        for (int r = 0; r < D1; ++r) acc[r] = fmaf(w[r], c0, fmaf(w[D1 + r], ws, acc[r]));
    };
    for (int k = 0; k < G; ++k) {
        if (k > 0) {
            if (jcur >= 0 && jcur < nj) row[jcur] = acc[0];
#pragma unroll
            for (int r = 0; r < D; ++r) acc[r] = acc[r + 1];
            acc[D] = 0.0f;
            ++jcur;
        }
        const int ve = sGs[k + 1];
        int v = sGs[k];
        for (; v + 1 < ve; v += 2) {
            node(v);
            node(v + 1);
        }
        if (v < ve) node(v);
    }
#pragma unroll
    for (int r = 0; r < D1; ++r)
        if (jcur + r >= 0 && jcur + r < nj) row[jcur + r] = acc[r];
}

template <int D, bool CLOSED, int TI>
__device__ __forceinline__ void tile_f(const TileF& t, int I, int J, unsigned char* smem) {
    static_assert(TI <= 32, "stage 2 maps one lane to one column of the tile");
    constexpr int D1 = D + 1;
    const int n = t.n, Nq = t.Nq, maxr = t.maxr;
    const int* __restrict__ lo = t.lo;
    const int* __restrict__ hi = t.hi;
    const int* __restrict__ jfirst = t.jfirst;
    const float* __restrict__ P = t.P;
    const float* __restrict__ Q = t.Q;
    const WsView<float> wsv = t.ws;
    const int i0 = I * TI, j0 = J * TI;
    const int ni = min(TI, n - i0), nj = min(TI, n - j0);
    const int uA0 = lo[i0], Na = hi[i0 + ni - 1] - uA0 + 1;
    const int uB0 = lo[j0], Nb = hi[j0 + nj - 1] - uB0 + 1;
    // block-uniform tile classes: every node where W^s is a Toeplitz
    // sequence; A- and B-ranges sharing a node (mod Nq)
    const bool toe = uB0 >= wsv.B && uB0 + Nb <= Nq - wsv.B && uA0 >= wsv.R && uA0 + Na <= Nq - wsv.R;
    bool diag = false;
    for (int k = -1; k <= 1; ++k)
        diag |= uA0 < uB0 + k * Nq + Nb && uB0 + k * Nq < uA0 + Na;
    const int tlen = Na + Nb - 1;
    // 16-byte records first, then 4-byte arrays: every offset stays aligned
    // for any maxr.  B-node record v: words 0-1 (xh, xl, yh, yl), (eh, el, ebh, ebl);
    // words 2 .. 2+NW-1 the P ln2/2 row and the Q row back to back (zero padded);
    // last word (m, first column - j0, Toeplitz offset, high part of L - x) as
    // integers.  Far tiles then replace word 0 by (x, y, e) relative to B node
    // 0 in plain FP32 and the high part of x.
    constexpr int RW = rec_words<D>();
    float4* sRec = (float4*)smem;                      // [maxr][RW]
    int* sJA = (int*)(sRec + (size_t)RW * maxr);       // [maxr]
    float* sPA = (float*)(sJA + maxr);                 // [maxr][D1]
    float* sT = sPA + maxr * D1;                       // [2][Na + Nb - 1] (Toeplitz tiles)
    int* sGs = (int*)(sT + 4 * maxr);                  // [TI + D + 2] first B node of each column group
    float* sS1 = (float*)(sGs + TI + D + 2);           // [maxr][TI + 1]
    float (*sBox)[8] = (float (*)[8])(sS1 + maxr * (TI + 1));   // [warps][8] node bounding boxes

    // bounding boxes of the A- and B-range nodes (high parts), for the far test
    const NodeF org = t.nodes[pmod(uB0, Nq)];
    float bx[8] = {3e38f, -3e38f, 3e38f, -3e38f, 3e38f, -3e38f, 3e38f, -3e38f};
    if ((int)threadIdx.x < Na) {
        const NodeF na = t.nodes[pmod(uA0 + (int)threadIdx.x, Nq)];
        bx[0] = bx[1] = na.xh;
        bx[2] = bx[3] = na.yh;
    }
    for (int v = threadIdx.x; v < Nb; v += blockDim.x) {
        const int u = uB0 + v, m = pmod(u, Nq), per = pdiv(u, Nq);
        const NodeF b = t.nodes[m];
        bx[4] = fminf(bx[4], b.xh); bx[5] = fmaxf(bx[5], b.xh);
        bx[6] = fminf(bx[6], b.yh); bx[7] = fmaxf(bx[7], b.yh);
        float4* rv = sRec + (size_t)v * RW;
        rv[0] = make_float4(b.xh, b.xl, b.yh, b.yl);
        rv[1] = make_float4(b.eh, b.el, b.ebh, b.ebl);
        constexpr int NW = wt_words<D>();
        float w[4 * NW];
#pragma unroll
        for (int r = 0; r < 4 * NW; ++r)
            w[r] = r < D1 ? P[m * D1 + r] * 0.346573590279972655f                 // x ln2 / 2
                          : (r < 2 * D1 ? Q[m * D1 + r - D1] : 0.0f);
#pragma unroll
        for (int q = 0; q < NW; ++q) rv[2 + q] = make_float4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        // W^s[ma][mb] = T[(mb - B) & 1][ma - mb + Nq - 1] = sT[offset + a]
        const int off = ((m - wsv.B) & 1) * tlen + (Nb - 1) - v;
        *reinterpret_cast<int4*>(&rv[RW - 1]) = make_int4(m, jfirst[m] + n * per - j0, off, __float_as_int(b.ebh));
    }
    for (int v = threadIdx.x; v < Na; v += blockDim.x) {
        const int u = uA0 + v, m = pmod(u, Nq), per = pdiv(u, Nq);
        sJA[v] = jfirst[m] + n * per - i0;
        for (int r = 0; r < D1; ++r) sPA[v * D1 + r] = P[m * D1 + r];
    }
#pragma unroll
    for (int k = 0; k < 8; k += 2)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            bx[k] = fminf(bx[k], __shfl_xor_sync(0xffffffffu, bx[k], o));
            bx[k + 1] = fmaxf(bx[k + 1], __shfl_xor_sync(0xffffffffu, bx[k + 1], o));
        }
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < 8; ++k) sBox[threadIdx.x >> 5][k] = bx[k];
    if (toe) {
        const int tbase = (uA0 - uB0) - (Nb - 1) + Nq - 1;      // sequence index of window entry 0
        const size_t slen = 2 * (size_t)Nq - 1;
        for (int k = threadIdx.x; k < 2 * tlen; k += blockDim.x) {
            const int p = k >= tlen, kk = k - p * tlen;
            sT[k] = wsv.toe[p * slen + tbase + kk];
        }
    }
    __syncthreads();
    // far tile: box gap at least twice the larger box diagonal (block-uniform)
    bool far = false;
    if (toe && !diag) {
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
            bx[k] = sBox[0][k];
            bx[k + 1] = sBox[0][k + 1];
        }
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
#pragma unroll
            for (int k = 0; k < 8; k += 2) {
                bx[k] = fminf(bx[k], sBox[w][k]);
                bx[k + 1] = fmaxf(bx[k + 1], sBox[w][k + 1]);
            }
        const float gx = fmaxf(0.0f, fmaxf(bx[0] - bx[5], bx[4] - bx[1]));
        const float gy = fmaxf(0.0f, fmaxf(bx[2] - bx[7], bx[6] - bx[3]));
        const float da = (bx[1] - bx[0]) * (bx[1] - bx[0]) + (bx[3] - bx[2]) * (bx[3] - bx[2]);
        const float db = (bx[5] - bx[4]) * (bx[5] - bx[4]) + (bx[7] - bx[6]) * (bx[7] - bx[6]);
        far = gx * gx + gy * gy >= 4.0f * fmaxf(da, db);
    }
    if (far)
        for (int v = threadIdx.x; v < Nb; v += blockDim.x) {
            float4* rv = sRec + (size_t)v * RW;
            const float4 g0 = rv[0], g1 = rv[1];
            rv[0] = make_float4((g0.x - org.xh) + (g0.y - org.xl), (g0.z - org.yh) + (g0.w - org.yl),
                                (g1.x - org.eh) + (g1.y - org.el), g1.x);
        }
    // column groups: the B nodes whose first column is jrel_0 + k start at
    // sGs[k] (empty groups repeat the next start); sGs[G] = Nb
    for (int v = threadIdx.x; v < Nb; v += blockDim.x) {
        auto jrel = [&](int q) { return reinterpret_cast<const int4*>(&sRec[(size_t)q * RW + RW - 1])->y; };
        const int j0r = jrel(0);
        const int k1 = jrel(v) - j0r, k0 = (v == 0) ? -1 : jrel(v - 1) - j0r;
        for (int k = k0 + 1; k <= k1; ++k) sGs[k] = v;
        if (v == Nb - 1) sGs[k1 + 1] = Nb;
    }
    __syncthreads();

    for (int a = threadIdx.x; a < Na; a += blockDim.x) {
        const int ma = pmod(uA0 + a, Nq);
        float* row = sS1 + a * (TI + 1);
        if (toe) {
            if (diag) tile_walk_f<D, CLOSED, true, true, false>(t, ma, a, Nb, nj, sRec, sGs, sT, row, org);
            else if (far) tile_walk_f<D, CLOSED, true, false, true>(t, ma, a, Nb, nj, sRec, sGs, sT, row, org);
            else tile_walk_f<D, CLOSED, true, false, false>(t, ma, a, Nb, nj, sRec, sGs, sT, row, org);
        } else {
            tile_walk_f<D, CLOSED, false, true, false>(t, ma, a, Nb, nj, sRec, sGs, sT, row, org);
        }
    }
    __syncthreads();

    // stage 2: A[i][j] = -(1/2pi) sum_a P[a][i - jA(a)] S1[a][j].  Each warp
    // owns a run of rows and one column per lane, and walks the A nodes of
    // those rows once with a window of d+1 row sums (rows jA(a)..jA(a)+d).
    const float scale = (float)(-1.0 / (2.0 * kPi));
    const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int RPW = (ni + nw - 1) / nw;                // rows per warp
    const int r0 = w * RPW, r1 = min(ni, r0 + RPW);
    if (r0 < r1) {
        const int bs = lo[i0 + r0] - uA0, be = hi[i0 + r1 - 1] - uA0;
        float acc[D1];
#pragma unroll
        for (int r = 0; r < D1; ++r) acc[r] = 0.0f;
        int jc = sJA[bs];
        float* Arow = t.A + (size_t)i0 * t.ld + j0 + lane;
        // A^T[j][i]: lane j's row of A^T, consecutive i from this warp (the partial
        // stores of a 32-byte sector come from one warp and merge in L2)
        float* ATcol = t.AT ? t.AT + (size_t)(j0 + lane) * t.ld + i0 : nullptr;
        const bool col = lane < nj;
        for (int b = bs; b <= be; ++b) {
            const int jb = sJA[b];
            while (jc < jb) {
                if (col && jc >= r0 && jc < r1) {
                    Arow[(size_t)jc * t.ld] = scale * acc[0];
                    if (ATcol) ATcol[jc] = scale * acc[0];
                }
#pragma unroll
                for (int r = 0; r < D; ++r) acc[r] = acc[r + 1];
                acc[D] = 0.0f;
                ++jc;
            }
            const float s1 = col ? sS1[b * (TI + 1) + lane] : 0.0f;
#pragma unroll
            for (int r = 0; r < D1; ++r) acc[r] = fmaf(sPA[b * D1 + r], s1, acc[r]);
        }
#pragma unroll
        for (int r = 0; r < D1; ++r)
            if (col && jc + r >= r0 && jc + r < r1) {
                Arow[(size_t)(jc + r) * t.ld] = scale * acc[r];
                if (ATcol) ATcol[jc + r] = scale * acc[r];
            }
    }
}

template <int D, bool CLOSED>
__global__ void __launch_bounds__(1024) k_assemble_f(const TileF t) {
    extern __shared__ __align__(16) unsigned char smem[];
    tile_f<D, CLOSED, kTile>(t, blockIdx.y, blockIdx.x, smem);
}

size_t tile_smem_f(int maxr, int d, int TI) {
    const int NW = (2 * (d + 1) + 3) / 4;
    return (size_t)maxr * (2 + NW) * 16 + (size_t)maxr * 16 + (size_t)maxr * 4 + (size_t)maxr * (d + 1) * 4 +
           (size_t)maxr * 4 * 4 + (size_t)(TI + d + 2) * 4 + (size_t)maxr * (TI + 1) * 4 +
           (size_t)((maxr + 31) / 32) * 8 * 4 + 64;
}

TileF tile_args_f(igs_prob p, int maxr) {
    const Plan& P = p->plan;
    return TileF{P.n, P.Nq, p->d_lo, p->d_hi, p->d_jfirst, (const NodeF*)p->d_nodes,
                 (const float*)p->d_P, (const float*)p->d_Q,
                 WsView<float>{p->d_WsT32, p->d_WsRow32, p->d_WsToe32, P.Nq, p->ws_B, p->ws_R}, (float*)p->d_A,
                 (float*)p->d_AT, (int64_t)P.n, maxr};
}

template <int D, bool CLOSED>
static void launch_tile_f(igs_prob p, int maxr, cudaStream_t s) {
    const Plan& P = p->plan;
    const size_t sm = tile_smem_f(maxr, D, kTile);
    auto kern = k_assemble_f<D, CLOSED>;
    ensure_dyn_smem((const void*)kern, (size_t)sm);
    const int nt = (P.n + kTile - 1) / kTile;
    const int threads = std::min(1024, (maxr + 31) / 32 * 32);
    kern<<<dim3(nt, nt), threads, sm, s>>>(tile_args_f(p, maxr));
    IGS_CUDA(cudaGetLastError());
}

template <int D>
static void launch_tile_f(igs_prob p, int maxr, cudaStream_t s) {
    if (p->plan.closed) launch_tile_f<D, true>(p, maxr, s);
    else launch_tile_f<D, false>(p, maxr, s);
}

template <typename T>
static size_t tile_smem(int maxr, int d) {
    using Node = typename NodeOf<T>::type;
    return maxr * sizeof(Node) + (size_t)maxr * (d + 1) * 3 * sizeof(T) + (size_t)maxr * (kTile + 1) * sizeof(T) +
           3 * sizeof(int) * maxr + 64;
}

template <typename T, int D>
static void launch_tile(igs_prob p, int maxr, cudaStream_t s) {
    const Plan& P = p->plan;
    const size_t sm = tile_smem<T>(maxr, D);
    auto kern = k_assemble_tile<T, D>;
    ensure_dyn_smem((const void*)kern, (size_t)sm);
    const int nt = (P.n + kTile - 1) / kTile;
    dim3 grid(nt, nt);
    const bool f32 = std::is_same<T, float>::value;
    const WsView<T> ws{f32 ? (const T*)p->d_WsT32 : (const T*)p->d_WsT, f32 ? (const T*)p->d_WsRow32 : (const T*)p->d_WsRow,
                       f32 ? (const T*)p->d_WsToe32 : (const T*)p->d_WsToe, P.Nq, p->ws_B, p->ws_R};
    kern<<<grid, 256, sm, s>>>(P.n, P.Nq, P.closed, (T)(f32 ? 1.0 : 1.0 / (P.L * P.L)), p->d_lo, p->d_hi, p->d_jfirst,
                               (const typename NodeOf<T>::type*)p->d_nodes, (const T*)p->d_P, (const T*)p->d_Q, ws,
                               (T*)p->d_A, (T*)p->d_AT, (int64_t)P.n, maxr);
    IGS_CUDA(cudaGetLastError());
}

template <typename T>
static void launch_tile_deg(igs_prob p, int maxr, cudaStream_t s) {
    if (std::is_same<T, float>::value && maxr <= 1024) {
        switch (p->plan.d) {
            case 2: launch_tile_f<2>(p, maxr, s); return;
            case 3: launch_tile_f<3>(p, maxr, s); return;
            case 4: launch_tile_f<4>(p, maxr, s); return;
            case 5: launch_tile_f<5>(p, maxr, s); return;
            default: throw Error(IGS_E_INVALID_ARG, "unsupported degree");
        }
    }
    switch (p->plan.d) {
        case 2: launch_tile<T, 2>(p, maxr, s); break;
        case 3: launch_tile<T, 3>(p, maxr, s); break;
        case 4: launch_tile<T, 4>(p, maxr, s); break;
        case 5: launch_tile<T, 5>(p, maxr, s); break;
        default: throw Error(IGS_E_INVALID_ARG, "unsupported degree");
    }
}

int max_tile_range(const Plan& P, int TI) {
    int mx = 0;
    for (int i0 = 0; i0 < P.n; i0 += TI) {
        int i1 = std::min(P.n, i0 + TI) - 1;
        mx = std::max(mx, P.hi[i1] - P.lo[i0] + 1);
    }
    return mx;
}

void geometry_nodes(igs_prob p) {
    const Plan& P = p->plan;
    cudaStream_t s = p->geom->ctx->stream;
    const int Nq = P.Nq, D1 = P.d + 1;
    if (!p->d_geo) p->d_geo = (double*)dev_alloc(p, sizeof(double) * 5 * Nq);
    geometry_eval(p->geom, p->d_eta, Nq, p->d_geo, s);
    p->launches++;
    const bool mixed = p->precision == IGS_MIXED;
    if (!p->d_nodes) {
        p->d_nodes = dev_alloc(p, (mixed ? sizeof(NodeF) : sizeof(NodeD)) * Nq);
        p->d_P = dev_alloc(p, (mixed ? sizeof(float) : sizeof(double)) * Nq * D1);
        p->d_Q = dev_alloc(p, (mixed ? sizeof(float) : sizeof(double)) * Nq * D1);
    }
    if (mixed)
        k_prep_f<<<(Nq + 127) / 128, 128, 0, s>>>(Nq, P.d, P.L, p->d_geo, p->d_eta, p->d_W, p->d_Bt,
                                                  (NodeF*)p->d_nodes, (float*)p->d_P, (float*)p->d_Q);
    else
        k_prep_d<<<(Nq + 127) / 128, 128, 0, s>>>(Nq, P.d, P.L, p->d_geo, p->d_eta, p->d_W, p->d_Bt,
                                                  (NodeD*)p->d_nodes, (double*)p->d_P, (double*)p->d_Q);
    p->launches++;
    IGS_CUDA(cudaGetLastError());
    p->geometry_ready = 1;
}

void assemble_matrix(igs_prob p) {
    const Plan& P = p->plan;
    cudaStream_t s = p->geom->ctx->stream;
    const bool mixed = p->precision == IGS_MIXED;
    const size_t esz = mixed ? sizeof(float) : sizeof(double);
    if (!p->d_A) p->d_A = dev_alloc(p, esz * (size_t)P.n * P.n);
    if (!p->d_AT) p->d_AT = dev_alloc(p, esz * (size_t)P.n * P.n);
    const int maxr = max_tile_range(P, kTile);
    if (mixed) launch_tile_deg<float>(p, maxr, s);
    else launch_tile_deg<double>(p, maxr, s);
    p->at_ready = 1;
    p->launches++;
}

// ------------------------------------------------------------------ batched form
constexpr int kBatchMaxThreads = 512;
// Geometry and FP32 node records of many problems in one launch: one thread
// per node over the concatenated node lists (items sorted by node0).
__global__ void k_batch_geom_f(const BatchGeomF* __restrict__ items, int nitems, int total) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= total) return;
    int lo = 0, hi = nitems - 1;                       // last item with node0 <= q
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (items[mid].node0 <= q) lo = mid;
        else hi = mid - 1;
    }
    const BatchGeomF& g = items[lo];
    const int m = q - g.node0;
    double v[5];
    curve_point_any(g.gdeg, g.nb, g.knots, g.ctrl, g.w, g.eta[m], v);
#pragma unroll
    for (int c = 0; c < 5; ++c) g.geo[(size_t)c * g.Nq + m] = v[c];
    prep_f_node(m, g.Nq, g.d, g.L, g.geo, g.eta, g.W, g.Bt, g.nodes, g.P, g.Q);
}

// Persistent assembly of many problems: each CTA takes (problem, tile) units
// from `units` in order through an atomic counter until none are left.  The
// unit order and the grid size come from the caller (the batch autotuner).
template <int TI>
__global__ void __launch_bounds__(kBatchMaxThreads, 1) k_batch_assemble_f(const BatchItemF* __restrict__ items,
                                                           const int2* __restrict__ units, int nunits,
                                                           int* __restrict__ counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_u;
    for (;;) {
        if (threadIdx.x == 0) s_u = atomicAdd(counter, 1);
        __syncthreads();
        const int u = s_u;
        if (u >= nunits) return;
        const int2 w = units[u];
        const BatchItemF& it = items[w.x];
        const int I = w.y / it.nt, J = w.y % it.nt;
        const TileF t = it.t;
        switch (it.d * 2 + it.closed) {
            case 4: tile_f<2, false, TI>(t, I, J, smem); break;
            case 5: tile_f<2, true, TI>(t, I, J, smem); break;
            case 6: tile_f<3, false, TI>(t, I, J, smem); break;
            case 7: tile_f<3, true, TI>(t, I, J, smem); break;
            case 8: tile_f<4, false, TI>(t, I, J, smem); break;
            case 9: tile_f<4, true, TI>(t, I, J, smem); break;
            case 10: tile_f<5, false, TI>(t, I, J, smem); break;
            default: tile_f<5, true, TI>(t, I, J, smem); break;
        }
        __syncthreads();
    }
}

void batch_geom_f(const BatchGeomF* d_items, int nitems, int total, cudaStream_t s) {
    k_batch_geom_f<<<(total + 127) / 128, 128, 0, s>>>(d_items, nitems, total);
    IGS_CUDA(cudaGetLastError());
}

template <int TI>
static void* batch_kernel() { return (void*)k_batch_assemble_f<TI>; }

int batch_blocks_per_sm(int TI, int threads, size_t smem) {
    void* k = TI == 16 ? batch_kernel<16>() : batch_kernel<32>();
    ensure_dyn_smem((const void*)k, (size_t)smem);
    int per = 0;
    IGS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, threads, smem));
    return per;
}

void batch_assemble_f(int TI, const BatchItemF* d_items, const int2* d_units, int nunits, int* d_counter, int grid,
                      int threads, size_t smem, cudaStream_t s) {
    if (TI == 16) {
        ensure_dyn_smem((const void*)k_batch_assemble_f<16>, (size_t)smem);
        k_batch_assemble_f<16><<<grid, threads, smem, s>>>(d_items, d_units, nunits, d_counter);
    } else {
        ensure_dyn_smem((const void*)k_batch_assemble_f<32>, (size_t)smem);
        k_batch_assemble_f<32><<<grid, threads, smem, s>>>(d_items, d_units, nunits, d_counter);
    }
    IGS_CUDA(cudaGetLastError());
}

}  // namespace igs
