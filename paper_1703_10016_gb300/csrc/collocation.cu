// Collocation form of the single-layer equation (the remark of Sect. 7: the
// quadrature rules serve collocation BEM as they are).  On a closed curve the
// pointwise form of eq. seconda_BIE at x = f(eta_m),
//   -(1/2 pi) int ln|x - y| q dgamma = u_D(x)/2 - (1/2 pi) int d/dn_y ln|x - y| u_D dgamma,
// is imposed at one node m_i per unknown, with the inner integrals by the same
// rules as the Galerkin form:
//   Ac[i][j] = -(1/2 pi) sum_{u in N^(j)} [ K1(eta_m, eta_u) J_u w^(j)_u + W^s[m][u] J_u B_j(eta_u) ],
//   beta_c[k][i] = u_D,k(eta_m)/2 - v_k(eta_m)/(2 pi),   m = m_i,
// with v_k the double-layer potential at the nodes (the b2 inner rule of Sect. 5).
// m_i is the node nearest the centre of the support of B_i (the Greville
// abscissa of the uniform cyclic basis), measured periodically in the plan's
// integer node units, ties to the smaller index.  Ac is not symmetric: LU with
// partial pivoting.  Matrix, LU and substitutions in FP64 in every tier; the
// node potentials follow the problem's tier (FP32 far field in the MIXED tier).
//
// The LU is unblocked (one pivot launch and one rank-1 update launch per
// column, 2 n launches) and the substitutions run in one block per data set:
// a post-processing path sized for n up to a few thousand, not a hot path.
#include <float.h>

#include <algorithm>
#include <vector>

#include "igs_internal.h"

namespace igs {

constexpr int kMaxCollocN = 16384;

// Row i of Ac: one thread per column j.
__global__ void k_colloc_matrix(int n, int Nq, int d, double L, const int* __restrict__ cnode,
                                const int* __restrict__ lo, const int* __restrict__ hi, const int* __restrict__ jfirst,
                                const double* __restrict__ geo, const double* __restrict__ eta,
                                const double* __restrict__ W, const double* __restrict__ Bt, WsView<double> ws,
                                double* __restrict__ Ac) {
    const int i = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int ma = cnode[i];
    const double xa = geo[ma], ya = geo[Nq + ma];
    double ea = eta[ma] - eta[0], eba = L - ea;
    if (ma == Nq - 1) { ea = L; eba = 0.0; }
    if (ma == 0) { ea = 0.0; eba = L; }
    const double lnJa = log(geo[4 * (size_t)Nq + ma]);
    const double invL2 = 1.0 / (L * L);
    double s = 0.0;
    for (int u = lo[j]; u <= hi[j]; ++u) {
        int mb = u % Nq;
        if (mb < 0) mb += Nq;
        const int ju = (u < 0) ? j + n : j;
        const int r = ju - jfirst[mb];
        if (r < 0 || r > d) continue;
        double c0;
        if (mb == ma) {
            c0 = lnJa;                                              // K1(s, s) = ln J(s)
        } else if (ma + mb == Nq - 1 && (ma == 0 || mb == 0)) {
            c0 = lnJa - 0.69314718055994530942;                     // corners (a, b), (b, a)
        } else {
            double eb = eta[mb] - eta[0], ebb = L - eb;
            if (mb == Nq - 1) { eb = L; ebb = 0.0; }
            if (mb == 0) { eb = 0.0; ebb = L; }
            const double dx = geo[mb] - xa, dy = geo[Nq + mb] - ya;
            const double D = fabs(eb - ea) * (eb + eba) * (ebb + ea) * invL2;   // three-image K2 = ln D
            c0 = 0.5 * log((dx * dx + dy * dy) / (D * D));
        }
        const double Jb = geo[4 * (size_t)Nq + mb];
        s += Jb * W[mb * (d + 1) + r] * c0 + Jb * Bt[mb * (d + 1) + r] * ws_at(ws, ma, mb);
    }
    Ac[(size_t)i * n + j] = s * (-1.0 / (2.0 * kPi));
}

// beta_c[k][i] = u_D,k(eta_m)/2 - v_k(eta_m)/(2 pi), v_k the sum of the np slots in order.
__global__ void k_colloc_rhs(int n, int Nq, int nrhs, const int* __restrict__ cnode, const double* __restrict__ uD,
                             int ldu, const double* __restrict__ vsum, int np, double* __restrict__ beta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= n) return;
    const int m = cnode[i];
    double v = 0.0;
    for (int sl = 0; sl < np; ++sl) v += vsum[((size_t)sl * nrhs + k) * Nq + m];
    beta[(size_t)k * n + i] = 0.5 * uD[(size_t)k * ldu + m] - v / (2.0 * kPi);
}

// Column k of the LU: pivot = largest |A[r][k]|, r >= k (ties to the smaller
// row, a fixed reduction tree), row swap, multipliers.  A zero or non-finite
// pivot sets *flag |= 1 and leaves the column as it is.
__global__ void __launch_bounds__(1024) k_lu_pivot(int n, int k, double* __restrict__ A, int* __restrict__ piv,
                                                   int* __restrict__ flag) {
    __shared__ double sv[1024];
    __shared__ int si[1024];
    const int tid = threadIdx.x;
    double best = -1.0;
    int bi = n;
    for (int r = k + tid; r < n; r += blockDim.x) {
        const double v = fabs(A[(size_t)r * n + k]);
        if (v > best) { best = v; bi = r; }
    }
    sv[tid] = best;
    si[tid] = bi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (tid < o) {
            const double v2 = sv[tid + o];
            const int i2 = si[tid + o];
            if (v2 > sv[tid] || (v2 == sv[tid] && i2 < si[tid])) { sv[tid] = v2; si[tid] = i2; }
        }
        __syncthreads();
    }
    const int pr = si[0];
    const double pv = sv[0];
    if (!(pv > 0.0) || !(pv <= DBL_MAX) || pr >= n) {
        if (tid == 0) { atomicOr(flag, 1); piv[k] = k; }
        return;
    }
    if (tid == 0) piv[k] = pr;
    if (pr != k) {
        for (int c = tid; c < n; c += blockDim.x) {
            const double t = A[(size_t)k * n + c];
            A[(size_t)k * n + c] = A[(size_t)pr * n + c];
            A[(size_t)pr * n + c] = t;
        }
    }
    __syncthreads();
    const double inv = 1.0 / A[(size_t)k * n + k];
    for (int r = k + 1 + tid; r < n; r += blockDim.x) A[(size_t)r * n + k] *= inv;
}

// Rank-1 update of the trailing block after column k: row k + 1 + blockIdx.y.
__global__ void k_lu_update(int n, int k, double* __restrict__ A) {
    const int r = k + 1 + blockIdx.y;
    const int c = k + 1 + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    A[(size_t)r * n + c] -= A[(size_t)r * n + k] * A[(size_t)k * n + c];
}

// P A = L U: x = U^{-1} L^{-1} P b for data set blockIdx.x, x staged in shared memory.
__global__ void __launch_bounds__(1024) k_lu_solve(int n, const double* __restrict__ A, const int* __restrict__ piv,
                                                   const double* __restrict__ b, double* __restrict__ x_out) {
    extern __shared__ double x[];
    const int tid = threadIdx.x, k = blockIdx.x;
    for (int r = tid; r < n; r += blockDim.x) x[r] = b[(size_t)k * n + r];
    __syncthreads();
    if (tid == 0) {
        for (int q = 0; q < n; ++q) {
            const int pq = piv[q];
            if (pq != q) { const double t = x[q]; x[q] = x[pq]; x[pq] = t; }
        }
    }
    __syncthreads();
    for (int q = 0; q < n; ++q) {                 // unit lower triangle
        const double xq = x[q];
        for (int r = q + 1 + tid; r < n; r += blockDim.x) x[r] -= A[(size_t)r * n + q] * xq;
        __syncthreads();
    }
    for (int q = n - 1; q >= 0; --q) {            // upper triangle
        if (tid == 0) x[q] /= A[(size_t)q * n + q];
        __syncthreads();
        const double xq = x[q];
        for (int r = tid; r < q; r += blockDim.x) x[r] -= A[(size_t)r * n + q] * xq;
        __syncthreads();
    }
    for (int r = tid; r < n; r += blockDim.x) x_out[(size_t)k * n + r] = x[r];
}

void collocation_solve(igs_prob p, const double* d_uD, int nrhs, double* d_alpha, double* Ac_out, int ac_mem,
                       int* nodes_out) {
    const Plan& P = p->plan;
    cudaStream_t s = p->geom->ctx->stream;
    if (!P.closed) throw Error(IGS_E_INVALID_ARG, "collocation is implemented for closed curves only");
    if (nrhs < 1 || nrhs > 8) throw Error(IGS_E_INVALID_ARG, "nrhs must be in [1, 8]");
    if (P.n > kMaxCollocN) throw Error(IGS_E_INVALID_ARG, "collocation supports n <= 16384");
    const int n = P.n, Nq = P.Nq;
    rhs_prepare(p);
    std::vector<int> cn;
    std::string err;
    if (collocation_nodes(P, cn, err) != IGS_OK) throw Error(IGS_E_INVALID_ARG, err);
    if (nodes_out) std::copy(cn.begin(), cn.end(), nodes_out);

    const size_t nn = (size_t)n * n;
    const int np_slots = rhs_slots(p);
    const size_t bytes = sizeof(double) * (nn + (size_t)nrhs * n + (size_t)np_slots * nrhs * Nq) +
                         sizeof(int) * (2 * (size_t)n + 1);
    unsigned char* buf = (unsigned char*)dev_alloc(p, bytes);
    double* A = (double*)buf;
    double* beta = A + nn;
    double* scratch = beta + (size_t)nrhs * n;
    int* d_cn = (int*)(scratch + (size_t)np_slots * nrhs * Nq);
    int* piv = d_cn + n;
    int* flag = piv + n;
    try {
        IGS_CUDA(cudaMemcpyAsync(d_cn, cn.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
        IGS_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
        const WsView<double> ws{p->d_WsT, p->d_WsRow, p->d_WsToe, Nq, p->ws_B, p->ws_R};
        k_colloc_matrix<<<dim3((n + 127) / 128, n), 128, 0, s>>>(n, Nq, P.d, P.L, d_cn, p->d_lo, p->d_hi,
                                                                 p->d_jfirst, p->d_geo, p->d_eta, p->d_W, p->d_Bt,
                                                                 ws, A);
        IGS_CUDA(cudaGetLastError());
        if (Ac_out)
            IGS_CUDA(cudaMemcpyAsync(Ac_out, A, sizeof(double) * nn,
                                     ac_mem == IGS_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
        const double* vsum = nullptr;
        int np = 0;
        rhs_node_potentials(p, d_uD, nrhs, scratch, &vsum, &np, s);
        k_colloc_rhs<<<dim3((n + 127) / 128, nrhs), 128, 0, s>>>(n, Nq, nrhs, d_cn, d_uD, Nq + p->Ng, vsum, np, beta);
        IGS_CUDA(cudaGetLastError());
        for (int k = 0; k < n; ++k) {
            k_lu_pivot<<<1, 1024, 0, s>>>(n, k, A, piv, flag);
            if (k + 1 < n) k_lu_update<<<dim3((n - k - 1 + 255) / 256, n - k - 1), 256, 0, s>>>(n, k, A);
        }
        IGS_CUDA(cudaGetLastError());
        const size_t smem = sizeof(double) * (size_t)n;
        if (smem > 48 * 1024)
            IGS_CUDA(cudaFuncSetAttribute(k_lu_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_lu_solve<<<nrhs, 1024, smem, s>>>(n, A, piv, beta, d_alpha);
        IGS_CUDA(cudaGetLastError());
        p->launches += 3 + 2 * n;
        int h_flag = 0;
        IGS_CUDA(cudaMemcpyAsync(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        IGS_CUDA(cudaStreamSynchronize(s));
        if (h_flag) throw Error(IGS_E_SINGULAR, "collocation matrix is singular (zero or non-finite pivot)");
    } catch (...) {
        cudaStreamSynchronize(s);
        dev_free_raw(p, buf);
        throw;
    }
    dev_free_raw(p, buf);
}

}  // namespace igs
