// Right-hand side (Sect. 5): b1_i = sum_n P[n,i] u_D(eta_n),
// b2_i = sum_n P[n,i] sum_g w_g Kbar(eta_n, t_g) u_D(t_g) with a composite Gauss
// rule of kGaussRhs points per refined element and
//   Kbar(s,t) = dK/dn_y(f(s), f(t)) J(t) = ((f(t)-f(s)) . (f2'(t), -f1'(t))) / |f(t)-f(s)|^2
// (outward normal of a counter-clockwise curve).  beta = b1/2 - b2/(2 pi) for the
// interior problem (eq. seconda_BIE), beta = b1 for an open arc (eq. prima_BIE).
#include <mutex>

#include "igs_internal.h"

namespace igs {

constexpr int kMaxRhs = 8;
constexpr int kRhsChunk = 256;

__global__ void k_rhs_points(int M, int G, double a, double hf, const double* __restrict__ gx,
                             const double* __restrict__ gw, double* __restrict__ t, double* __restrict__ w) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= M * G) return;
    const int e = q / G, g = q % G;
    t[q] = a + hf * (e + gx[g]);
    w[q] = hf * gw[g];
}

// v[k][m] = sum_g w_g Kbar(eta_m, t_g) u_D^k(t_g)   (FP64)
__global__ void __launch_bounds__(256) k_double_layer(int Nq, int Ng, int nrhs, const double* __restrict__ geo,
                                                      const double* __restrict__ rgeo, const double* __restrict__ rw,
                                                      const double* __restrict__ uD, int ldu, int off,
                                                      double* __restrict__ v) {
    __shared__ double sx[kRhsChunk], sy[kRhsChunk], sx1[kRhsChunk], sy1[kRhsChunk];
    __shared__ double su[kMaxRhs][kRhsChunk];
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = m < Nq;
    const double xm = live ? geo[m] : 0.0, ym = live ? geo[Nq + m] : 0.0;
    double acc[kMaxRhs];
    for (int k = 0; k < kMaxRhs; ++k) acc[k] = 0.0;
    for (int g0 = 0; g0 < Ng; g0 += kRhsChunk) {
        const int cn = min(kRhsChunk, Ng - g0);
        __syncthreads();
        for (int q = threadIdx.x; q < cn; q += blockDim.x) {
            const int g = g0 + q;
            sx[q] = rgeo[g]; sy[q] = rgeo[Ng + g]; sx1[q] = rgeo[2 * Ng + g]; sy1[q] = rgeo[3 * Ng + g];
            for (int k = 0; k < nrhs; ++k) su[k][q] = rw[g] * uD[(size_t)k * ldu + off + g];
        }
        __syncthreads();
        if (live) {
            for (int q = 0; q < cn; ++q) {
                const double dx = sx[q] - xm, dy = sy[q] - ym;
                const double kb = (dx * sy1[q] - dy * sx1[q]) / (dx * dx + dy * dy);
                for (int k = 0; k < nrhs; ++k) acc[k] += kb * su[k][q];
            }
        }
    }
    if (live)
        for (int k = 0; k < nrhs; ++k) v[(size_t)k * Nq + m] = acc[k];
}

// beta[k][i] from the row weights P[m][r] = J_m w^(jfirst+r)_m over N^(i).
__global__ void k_beta(int n, int Nq, int d, int nrhs, int closed, const int* __restrict__ lo, const int* __restrict__ hi,
                       const int* __restrict__ jfirst, const double* __restrict__ W, const double* __restrict__ geo,
                       const double* __restrict__ uD, int ldu, const double* __restrict__ v, double* __restrict__ beta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= n || k >= nrhs) return;
    double b1 = 0.0, b2 = 0.0;
    for (int u = lo[i]; u <= hi[i]; ++u) {
        int m = u % Nq;
        if (m < 0) m += Nq;
        const int iu = (u < 0) ? i + n : i;
        const int r = iu - jfirst[m];
        if (r < 0 || r > d) continue;
        const double p = geo[4 * Nq + m] * W[m * (d + 1) + r];
        b1 += p * uD[(size_t)k * ldu + m];
        if (closed) b2 += p * v[(size_t)k * Nq + m];
    }
    beta[(size_t)k * n + i] = closed ? 0.5 * b1 - b2 / (2.0 * kPi) : b1;
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

void rhs_build(igs_prob p, const double* d_uD, int nrhs) {
    const Plan& P = p->plan;
    cudaStream_t s = p->geom->ctx->stream;
    if (nrhs < 1 || nrhs > kMaxRhs) throw Error(IGS_E_INVALID_ARG, "nrhs must be in [1, 8]");
    const int ldu = P.Nq + p->Ng;
    double* d_v = nullptr;
    if (P.closed) {
        d_v = (double*)dev_alloc(p, sizeof(double) * (size_t)nrhs * P.Nq);
        k_double_layer<<<(P.Nq + 255) / 256, 256, 0, s>>>(P.Nq, p->Ng, nrhs, p->d_geo, p->d_rhs_geo, p->d_rhs_w,
                                                          d_uD, ldu, P.Nq, d_v);
        p->launches++;
    }
    if (p->d_beta && p->rhs_n < nrhs) dev_free(p, p->d_beta);
    if (!p->d_beta) p->d_beta = (double*)dev_alloc(p, sizeof(double) * (size_t)kMaxRhs * P.n);
    p->rhs_n = nrhs;
    dim3 grid((P.n + 127) / 128, nrhs);
    k_beta<<<grid, 128, 0, s>>>(P.n, P.Nq, P.d, nrhs, P.closed, p->d_lo, p->d_hi, p->d_jfirst, p->d_W, p->d_geo, d_uD,
                                ldu, d_v, p->d_beta);
    p->launches++;
    IGS_CUDA(cudaGetLastError());
    if (d_v) {
        IGS_CUDA(cudaStreamSynchronize(s));
        dev_free(p, d_v);
    }
}

// ------------------------------------------------------------ no-allocation variant
// Some callers cannot allocate device memory inside a call: a host framework
// that owns all device memory through its own allocator and forbids others
// (custom-call handlers, memory-pool managed serving loops), code that must
// stay off the driver's allocator for latency reasons, or code that runs while
// someone else captures the stream.  For them igs_build_rhs_noalloc runs the
// same two kernels as igs_build_rhs (double-layer potential at the nodes, then
// the weighted sums b1 / b2) with the node potentials v kept in this fixed,
// file-scope device array instead of a buffer from cudaMallocAsync.  Every GPU
// that loads the library holds the array until the process exits.  All calls
// share it, so calls that overlap on the GPU (two streams, two host threads)
// race on it; it keeps the last call's contents, and nothing in it needs to
// start at zero because the first kernel overwrites every entry it uses.
constexpr size_t kNoAllocScratchDoubles = size_t(1) << 20;       // 8 MiB: n_quad * nrhs <= 1048576
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
    cudaStream_t s = p->geom->ctx->stream;
    if (nrhs < 1 || nrhs > kMaxRhs) throw Error(IGS_E_INVALID_ARG, "nrhs must be in [1, 8]");
    if (!p->rules_ready || !p->geometry_ready || !p->d_rhs_geo)
        throw Error(IGS_E_STATE, "igs_build_rhs_noalloc needs the rules, the node geometry and the rhs points: "
                                 "call igs_assemble and igs_rhs_points first");
    if ((size_t)P.Nq * nrhs > kNoAllocScratchDoubles)
        throw Error(IGS_E_INVALID_ARG, "igs_build_rhs_noalloc: n_quad * nrhs = " + std::to_string((size_t)P.Nq * nrhs) +
                                           " exceeds the fixed scratch of " + std::to_string(kNoAllocScratchDoubles) +
                                           " doubles");
    double* v = scratch_address(p->geom->ctx->device);
    const int ldu = P.Nq + p->Ng;
    if (P.closed) {
        k_double_layer<<<(P.Nq + 255) / 256, 256, 0, s>>>(P.Nq, p->Ng, nrhs, p->d_geo, p->d_rhs_geo, p->d_rhs_w,
                                                          d_uD, ldu, P.Nq, v);
        IGS_CUDA(cudaGetLastError());
        p->launches++;
    }
    dim3 grid((P.n + 127) / 128, nrhs);
    k_beta<<<grid, 128, 0, s>>>(P.n, P.Nq, P.d, nrhs, P.closed, p->d_lo, p->d_hi, p->d_jfirst, p->d_W, p->d_geo, d_uD,
                                ldu, v, d_beta);
    IGS_CUDA(cudaGetLastError());
    p->launches++;
}

}  // namespace igs

