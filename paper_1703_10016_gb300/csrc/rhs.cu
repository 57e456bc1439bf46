// Right-hand side (Sect. 5): b1_i = sum_n P[n,i] u_D(eta_n),
// b2_i = sum_n P[n,i] sum_g w_g Kbar(eta_n, t_g) u_D(t_g) with a composite Gauss
// rule of kGaussRhs points per refined element and
//   Kbar(s,t) = dK/dn_y(f(s), f(t)) J(t) = ((f(t)-f(s)) . (f2'(t), -f1'(t))) / |f(t)-f(s)|^2
// (outward normal of a counter-clockwise curve).  beta = b1/2 - b2/(2 pi) for the
// interior problem (eq. seconda_BIE), beta = b1 for an open arc (eq. prima_BIE).
//
// The double-layer potentials v_k(eta_m) = sum_g w_g Kbar(eta_m, t_g) u_k(t_g) are
// an N_quad x N_GQ kernel sum.  The Gauss range is split in kSplit slices, one
// grid row each, so that every node has kSplit partial sums (reduced in a fixed
// order, by k_double_layer_near in the MIXED tier and by k_beta in the FP64
// tier: results do not depend on scheduling).  MIXED tier: FP32 with
// float-float coordinate differences for every pair.  At the Gauss points of
// the node's refined element and its two neighbours the numerator
// (f(t)-f(s)).n(t) is second-order small and the FP32 value is poor, so
// k_double_layer_near recomputes those pairs in FP64 and, in one more partial
// slot, replaces their FP32 contributions (reproduced bit for bit by the same
// FP32 operations, kb32_pair) by the FP64 ones.  FP64 tier: every pair in FP64.
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

// MIXED far field: partial sums over Gauss slice blockIdx.y, FP32, every pair
// (the near pairs are replaced by k_double_layer_near).  Gauss data in shared
// memory as 16-byte coordinate records and 8-byte (a, b) records.  A block
// holds 32 NN nodes: thread (j, p), j < kFarLanes, p < kFarParts, keeps
// the float-float coordinates of the NN nodes j + kFarLanes k in
// registers and sums the chunk's Gauss points q = p (mod kFarParts) for all of
// them, so one shared-memory read of a Gauss point serves NN pairs (one
// warp = 32 node groups of one part: every read is a broadcast).  The parts
// are added in a fixed order at the end.
// (NN = 4; small problems take NN = 2, which doubles the grid: a node block of
// 64 instead of 128 nodes keeps every SM busy when N_quad is a few thousand)
constexpr int kFarLanes = 32, kFarParts = 8;

template <int NR, int kFarNN>
__global__ void __launch_bounds__(kFarLanes * kFarParts) k_double_layer_f(int Nq, int Ng, const double* __restrict__ geo,
                                                                          const double* __restrict__ rgeo,
                                                                          const double* __restrict__ rw,
                                                                          const double* __restrict__ uD, int ldu, int off,
                                                                          double* __restrict__ part) {
    __shared__ float4 sg[kRhsChunk];
    __shared__ float2 sab[kRhsChunk];
    __shared__ float su[NR][kRhsChunk];
    constexpr int kFarNodes = kFarLanes * kFarNN;
    __shared__ float red[kFarParts][NR][kFarNodes];
    const int lane = threadIdx.x % kFarLanes, prt = threadIdx.x / kFarLanes;
    const int m0 = blockIdx.x * kFarNodes + lane;
    float xh[kFarNN], xl[kFarNN], yh[kFarNN], yl[kFarNN];
#pragma unroll
    for (int k = 0; k < kFarNN; ++k) {
        const int m = min(m0 + kFarLanes * k, Nq - 1);
        split2(geo[m], xh[k], xl[k]);
        split2(geo[Nq + m], yh[k], yl[k]);
    }
    float acc[kFarNN][NR];
#pragma unroll
    for (int k = 0; k < kFarNN; ++k)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[k][r] = 0.f;
    const int per = (Ng + kSplit - 1) / kSplit;
    const int g_lo = blockIdx.y * per, g_hi = min(Ng, g_lo + per);
    for (int g0 = g_lo; g0 < g_hi; g0 += kRhsChunk) {
        const int cn = min(kRhsChunk, g_hi - g0);
        __syncthreads();
        for (int q = threadIdx.x; q < cn; q += blockDim.x) {
            const int g = g0 + q;
            float4 c;
            split2(rgeo[g], c.x, c.y);
            split2(rgeo[Ng + g], c.z, c.w);
            sg[q] = c;
            sab[q] = make_float2((float)rgeo[3 * Ng + g], (float)(-rgeo[2 * Ng + g]));   // f2'(t), -f1'(t)
            const double w = rw[g];
#pragma unroll
            for (int r = 0; r < NR; ++r) su[r][q] = (float)(w * uD[(size_t)r * ldu + off + g]);
        }
        __syncthreads();
#pragma unroll 2
        for (int q = prt; q < cn; q += kFarParts) {
            const float4 c = sg[q];
            const float2 ab = sab[q];
            float u[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) u[r] = su[r][q];
#pragma unroll
            for (int k = 0; k < kFarNN; ++k) {
                const float kb = kb32_pair(c.x, c.y, c.z, c.w, ab.x, ab.y, xh[k], xl[k], yh[k], yl[k]);
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[k][r] = fmaf(kb, u[r], acc[k][r]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kFarNN; ++k)
#pragma unroll
        for (int r = 0; r < NR; ++r) red[prt][r][lane + kFarLanes * k] = acc[k][r];
    __syncthreads();
    for (int idx = threadIdx.x; idx < NR * kFarNodes; idx += blockDim.x) {
        const int r = idx / kFarNodes, j = idx % kFarNodes;
        const int m = blockIdx.x * kFarNodes + j;
        if (m >= Nq) continue;
        float v = red[0][r][j];
#pragma unroll
        for (int q = 1; q < kFarParts; ++q) v += red[q][r][j];
        part[((size_t)blockIdx.y * NR + r) * Nq + m] = (double)v;
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

// MIXED near field: Gauss points of the node's element and its two neighbours.
// Adds their FP64 contributions and removes the FP32 ones the far-field kernel
// summed (same bits from kb32_pair; the product of two floats is exact in FP64).
// kNearLanes consecutive lanes share a node (pairs j = lane, lane + kNearLanes,
// ... of the 3 kGaussRhs near pairs), reduced by a fixed shuffle tree; the
// first lane adds the kSplit far-field partial sums (in slice order) and
// writes the node's whole potential v_k(eta_m) into `out`.
constexpr int kNearLanes = 4;

__global__ void k_double_layer_near(int Nq, int Ng, int M, int nrhs, const double* __restrict__ geo,
                                    const int* __restrict__ fspan, const double* __restrict__ rgeo,
                                    const double* __restrict__ rw, const double* __restrict__ uD, int ldu, int off,
                                    const double* __restrict__ far, double* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = t / kNearLanes, lane = t % kNearLanes;
    const bool live = m < Nq;
    const int mm = live ? m : Nq - 1;
    const double xm = geo[mm], ym = geo[Nq + mm];
    float xh, xl, yh, yl;
    split2(xm, xh, xl);
    split2(ym, yh, yl);
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
        float gxh, gxl, gyh, gyl;
        split2(rgeo[g], gxh, gxl);
        split2(rgeo[Ng + g], gyh, gyl);
        const float kb32 = kb32_pair(gxh, gxl, gyh, gyl, (float)rgeo[3 * Ng + g], (float)(-rgeo[2 * Ng + g]), xh,
                                     xl, yh, yl);
        const double w = rw[g];
        for (int k = 0; k < nrhs; ++k) {
            const double u = uD[(size_t)k * ldu + off + g];
            acc[k] += kb * w * u - (double)kb32 * (double)(float)(w * u);
        }
    }
    for (int k = 0; k < nrhs; ++k) {
        double v = acc[k];
#pragma unroll
        for (int o = 1; o < kNearLanes; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (live && lane == 0) {
            double tot = 0.0;
            for (int sl = 0; sl < kSplit; ++sl) tot += far[((size_t)sl * nrhs + k) * Nq + m];
            out[(size_t)k * Nq + m] = tot + v;
        }
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
    IGS_CUDA(cudaStreamSynchronize(s));
    dev_free(p, d_g);
}

// Number of partial-sum slots (each nrhs x N_quad doubles) the kernels need.
int rhs_slots(const igs_prob p) {
    if (!p->plan.closed) return 0;
    return kSplit + (p->precision == IGS_MIXED ? 1 : 0);
}

template <int NR>
static void launch_far(igs_prob p, const double* d_uD, int ldu, double* part, cudaStream_t s) {
    const Plan& P = p->plan;
    if (p->precision == IGS_MIXED) {
        // four nodes per thread, or two when that would leave SMs without a block
        if ((P.Nq + 127) / 128 * kSplit >= 4 * 152)
            k_double_layer_f<NR, 4><<<dim3((P.Nq + 127) / 128, kSplit), kFarLanes * kFarParts, 0, s>>>(
                P.Nq, p->Ng, p->d_geo, p->d_rhs_geo, p->d_rhs_w, d_uD, ldu, P.Nq, part);
        else
            k_double_layer_f<NR, 2><<<dim3((P.Nq + 63) / 64, kSplit), kFarLanes * kFarParts, 0, s>>>(
                P.Nq, p->Ng, p->d_geo, p->d_rhs_geo, p->d_rhs_w, d_uD, ldu, P.Nq, part);
    }
    else
        k_double_layer_d<NR><<<dim3((P.Nq + 255) / 256, kSplit), 256, 0, s>>>(P.Nq, p->Ng, p->d_geo, p->d_rhs_geo,
                                                                            p->d_rhs_w, d_uD, ldu, P.Nq, part);
    IGS_CUDA(cudaGetLastError());
}

// Double-layer potentials v_k(eta_m) at the nodes of a closed curve, as
// partial sums in `scratch` (rhs_slots x nrhs x N_quad doubles): v_k(eta_m) is
// the sum over s < *np of vsum[(s nrhs + k) N_quad + m], in that order.
void rhs_node_potentials(igs_prob p, const double* d_uD, int nrhs, double* scratch, const double** vsum, int* np,
                         cudaStream_t s) {
    const Plan& P = p->plan;
    const int ldu = P.Nq + p->Ng;
    *np = rhs_slots(p);
    *vsum = scratch;
    switch (nrhs) {
        case 1: launch_far<1>(p, d_uD, ldu, scratch, s); break;
        case 2: launch_far<2>(p, d_uD, ldu, scratch, s); break;
        case 3: launch_far<3>(p, d_uD, ldu, scratch, s); break;
        case 4: launch_far<4>(p, d_uD, ldu, scratch, s); break;
        case 5: launch_far<5>(p, d_uD, ldu, scratch, s); break;
        case 6: launch_far<6>(p, d_uD, ldu, scratch, s); break;
        case 7: launch_far<7>(p, d_uD, ldu, scratch, s); break;
        default: launch_far<8>(p, d_uD, ldu, scratch, s); break;
    }
    p->launches++;
    if (p->precision == IGS_MIXED) {
        // the near kernel writes the whole potential (far slices + near correction) into the last slot
        double* whole = scratch + (size_t)kSplit * nrhs * P.Nq;
        const int nt = P.Nq * kNearLanes;
        k_double_layer_near<<<(nt + 127) / 128, 128, 0, s>>>(P.Nq, p->Ng, P.M, nrhs, p->d_geo, p->d_fspan,
                                                             p->d_rhs_geo, p->d_rhs_w, d_uD, ldu, P.Nq, scratch,
                                                             whole);
        IGS_CUDA(cudaGetLastError());
        p->launches++;
        *vsum = whole;
        *np = 1;
    }
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
