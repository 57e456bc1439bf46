// Representation formula (Sect. 2), post-processing of a solved density:
//   u(x) = -(1/2 pi) int_Gamma ln|x - y| q(y) dgamma_y
//          + (1/2 pi) int_Gamma d/dn_y ln|x - y| u_D(y) dgamma_y,   x in Omega,
// for a closed curve (direct method, q = sum_j alpha_j B_j), and only the first
// term for an open arc (indirect method, density phi = sum_j alpha_j B_j).
// Both integrals use the composite Gauss rule of the right-hand side (kGaussRhs
// points per refined element), so u_D is taken at the same points as for
// igs_build_rhs.  FP64 in every tier.
//
// k_pot_density forms w_g J(t_g) q_k(t_g) once per Gauss point; k_potential
// sums the kernel over a slice of the Gauss points for one evaluation point per
// thread (the Gauss data staged in shared memory), and k_pot_reduce adds the
// slices in a fixed order (results do not depend on scheduling).
#include "bspline_dev.cuh"
#include "igs_internal.h"

namespace igs {

constexpr int kPotChunk = 256;                     // Gauss points staged per pass
constexpr int kPotThreads = 128;
constexpr int kPotMaxSlices = 64;
constexpr int kPotMinSlice = 64;                   // Gauss points per slice at least
constexpr int64_t kPotTargetThreads = int64_t(1) << 19;

// wq[k][g] = w_g J(t_g) q_k(t_g) with q_k = sum_j alpha_k[j] B_j (cyclic test
// basis for a closed curve: unrolled index c + r taken modulo N_h; clamped
// basis for an open arc, Cox-de Boor on the local knots).
__global__ void k_pot_density(int Ng, int G, int d, int Nref, int Nh, int n, int closed, double a, double b,
                              double h, double hf, const double* __restrict__ piece, const double* __restrict__ rt,
                              const double* __restrict__ rgeo, const double* __restrict__ rw,
                              const double* __restrict__ alpha, int nrhs, double* __restrict__ wq) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Ng) return;
    const int e = g / G;                     // refined element
    const int c = e / Nref;                  // coarse element: test functions c .. c + d
    const double t = rt[g];
    double B[kMaxDegree + 1];
    if (closed) {
        const double uf = (t - a) / hf - e;
        const double uc = ((e - c * Nref) + uf) / Nref;
        for (int r = 0; r <= d; ++r) B[r] = piece_eval(piece, d, d - r, uc);
    } else {
        // clamped knots a (d times), a + h k (k = 0..N_h, the last exactly b), b (d times):
        // U[k'] = knot c + k', and the span of coarse element c is local index d
        double U[2 * kMaxDegree + 2];
        for (int k = 0; k <= 2 * d + 1; ++k) {
            const int kk = c + k - d;
            U[k] = kk <= 0 ? a : (kk >= Nh ? b : a + h * kk);
        }
        basis_funs(U, d, d, t, B);
    }
    const double wj = rw[g] * rgeo[4 * (size_t)Ng + g];
    for (int k = 0; k < nrhs; ++k) {
        double q = 0.0;
        for (int r = 0; r <= d; ++r) {
            int j = c + r;
            if (closed && j >= Nh) j -= Nh;
            q += alpha[(size_t)k * n + j] * B[r];
        }
        wq[(size_t)k * Ng + g] = wj * q;
    }
}

// Partial sums over Gauss slice blockIdx.y for evaluation point i:
//   sum_g [ Kbar(x_i, t_g) w_g u_k(t_g) - (1/2) ln|x_i - f(t_g)|^2 w_g J_g q_k(t_g) ]
// with Kbar(x, t) = (f(t) - x) . (f2'(t), -f1'(t)) / |f(t) - x|^2 (DL: closed curve).
template <int NR, bool DL>
__global__ void __launch_bounds__(kPotThreads) k_potential(int64_t count, int Ng, int per,
                                                           const double* __restrict__ xy,
                                                           const double* __restrict__ rgeo,
                                                           const double* __restrict__ rw,
                                                           const double* __restrict__ wq,
                                                           const double* __restrict__ uD, int ldu, int off,
                                                           double* __restrict__ part) {
    __shared__ double sx[kPotChunk], sy[kPotChunk], sa[kPotChunk], sb[kPotChunk];
    __shared__ double sq[NR][kPotChunk];
    __shared__ double su[DL ? NR : 1][kPotChunk];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < count;
    const double x = live ? xy[2 * i] : 0.0, y = live ? xy[2 * i + 1] : 0.0;
    double acc[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) acc[k] = 0.0;
    const int g_lo = blockIdx.y * per, g_hi = min(Ng, g_lo + per);
    for (int g0 = g_lo; g0 < g_hi; g0 += kPotChunk) {
        const int cn = min(kPotChunk, g_hi - g0);
        __syncthreads();
        for (int q = threadIdx.x; q < cn; q += blockDim.x) {
            const int g = g0 + q;
            sx[q] = rgeo[g];
            sy[q] = rgeo[Ng + g];
#pragma unroll
            for (int k = 0; k < NR; ++k) sq[k][q] = -0.5 * wq[(size_t)k * Ng + g];
            if (DL) {
                sa[q] = rgeo[3 * (size_t)Ng + g];
                sb[q] = -rgeo[2 * (size_t)Ng + g];
                const double w = rw[g];
#pragma unroll
                for (int k = 0; k < NR; ++k) su[k][q] = w * uD[(size_t)k * ldu + off + g];
            }
        }
        __syncthreads();
        if (live) {
            for (int q = 0; q < cn; ++q) {
                const double dx = sx[q] - x, dy = sy[q] - y;
                const double r2 = dx * dx + dy * dy;
                const double lr = log(r2);
                if (DL) {
                    const double kb = (dx * sa[q] + dy * sb[q]) / r2;
#pragma unroll
                    for (int k = 0; k < NR; ++k) acc[k] += kb * su[k][q] + lr * sq[k][q];
                } else {
#pragma unroll
                    for (int k = 0; k < NR; ++k) acc[k] += lr * sq[k][q];
                }
            }
        }
    }
    if (live) {
#pragma unroll
        for (int k = 0; k < NR; ++k) part[((size_t)blockIdx.y * NR + k) * count + i] = acc[k];
    }
}

__global__ void k_pot_reduce(int64_t count, int nrhs, int S, const double* __restrict__ part, double* __restrict__ u) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= count) return;
    double s = 0.0;
    for (int sl = 0; sl < S; ++sl) s += part[((size_t)sl * nrhs + k) * count + i];
    u[(size_t)k * count + i] = s * (1.0 / (2.0 * kPi));
}

// Number of Gauss slices for `count` points: enough threads to fill the GPU,
// at least kPotMinSlice Gauss points per slice.  Depends on the sizes only.
static void pot_slices(int64_t count, int Ng, int& S, int& per) {
    int64_t want = kPotTargetThreads / (count > 0 ? count : 1);
    const int64_t cap = (Ng + kPotMinSlice - 1) / kPotMinSlice;
    if (want > kPotMaxSlices) want = kPotMaxSlices;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    per = (int)((Ng + want - 1) / want);
    S = (Ng + per - 1) / per;
}

template <int NR>
static void launch_pot(bool closed, dim3 grid, cudaStream_t s, int64_t count, int Ng, int per, const double* xy,
                       const double* rgeo, const double* rw, const double* wq, const double* uD, int ldu, int off,
                       double* part) {
    if (closed)
        k_potential<NR, true><<<grid, kPotThreads, 0, s>>>(count, Ng, per, xy, rgeo, rw, wq, uD, ldu, off, part);
    else
        k_potential<NR, false><<<grid, kPotThreads, 0, s>>>(count, Ng, per, xy, rgeo, rw, wq, uD, ldu, off, part);
}

void potential_eval(igs_prob p, const double* d_alpha, const double* d_uD, int nrhs, const double* d_xy,
                    int64_t count, double* d_u) {
    const Plan& P = p->plan;
    cudaStream_t s = p->geom->ctx->stream;
    if (nrhs < 1 || nrhs > 8) throw Error(IGS_E_INVALID_ARG, "nrhs must be in [1, 8]");
    if (count <= 0) return;
    if ((count + kPotThreads - 1) / kPotThreads > 0x7fffffffLL) throw Error(IGS_E_INVALID_ARG, "too many points");
    rhs_prepare(p);
    const int Ng = p->Ng;
    double* wq = (double*)dev_alloc(p, sizeof(double) * (size_t)nrhs * Ng);
    k_pot_density<<<(Ng + 127) / 128, 128, 0, s>>>(Ng, kGaussRhs, P.d, P.Nref, P.Nh, P.n, P.closed, P.a, P.b, P.h,
                                                  P.hf, p->d_piece, p->d_rhs_t, p->d_rhs_geo, p->d_rhs_w, d_alpha,
                                                  nrhs, wq);
    IGS_CUDA(cudaGetLastError());
    int S = 1, per = Ng;
    pot_slices(count, Ng, S, per);
    double* part = (double*)dev_alloc(p, sizeof(double) * (size_t)S * nrhs * count);
    const dim3 grid((unsigned)((count + kPotThreads - 1) / kPotThreads), S);
    const int ldu = P.Nq + Ng;
    const bool closed = P.closed != 0;
    switch (nrhs) {
        case 1: launch_pot<1>(closed, grid, s, count, Ng, per, d_xy, p->d_rhs_geo, p->d_rhs_w, wq, d_uD, ldu, P.Nq, part); break;
        case 2: launch_pot<2>(closed, grid, s, count, Ng, per, d_xy, p->d_rhs_geo, p->d_rhs_w, wq, d_uD, ldu, P.Nq, part); break;
        case 3: launch_pot<3>(closed, grid, s, count, Ng, per, d_xy, p->d_rhs_geo, p->d_rhs_w, wq, d_uD, ldu, P.Nq, part); break;
        case 4: launch_pot<4>(closed, grid, s, count, Ng, per, d_xy, p->d_rhs_geo, p->d_rhs_w, wq, d_uD, ldu, P.Nq, part); break;
        case 5: launch_pot<5>(closed, grid, s, count, Ng, per, d_xy, p->d_rhs_geo, p->d_rhs_w, wq, d_uD, ldu, P.Nq, part); break;
        case 6: launch_pot<6>(closed, grid, s, count, Ng, per, d_xy, p->d_rhs_geo, p->d_rhs_w, wq, d_uD, ldu, P.Nq, part); break;
        case 7: launch_pot<7>(closed, grid, s, count, Ng, per, d_xy, p->d_rhs_geo, p->d_rhs_w, wq, d_uD, ldu, P.Nq, part); break;
        default: launch_pot<8>(closed, grid, s, count, Ng, per, d_xy, p->d_rhs_geo, p->d_rhs_w, wq, d_uD, ldu, P.Nq, part); break;
    }
    IGS_CUDA(cudaGetLastError());
    k_pot_reduce<<<dim3((unsigned)((count + 255) / 256), nrhs), 256, 0, s>>>(count, nrhs, S, part, d_u);
    IGS_CUDA(cudaGetLastError());
    p->launches += 3;
    IGS_CUDA(cudaStreamSynchronize(s));
    dev_free(p, part);
    dev_free(p, wq);
}

}  // namespace igs
