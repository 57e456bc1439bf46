// Boundary curve evaluation (Sect. 3): f, f' and the parametric speed J = |f'| (eq. J).
#include "bspline_dev.cuh"
#include "igs_internal.h"

namespace igs {

// NURBS f = N/W with N = sum w_i Q_i B_i, W = sum w_i B_i; f' = (N' - W' f)/W.
// out is SoA [5][count]: x, y, x', y', J.
template <int DEG>
__global__ void k_geom(int nb, const double* __restrict__ knots, const double* __restrict__ ctrl,
                       const double* __restrict__ w, const double* __restrict__ t, int count, double* __restrict__ out) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= count) return;
    const double s = t[q];
    const int span = find_span(knots, nb, DEG, s);
    double N[DEG + 1], dN[DEG + 1];
    basis_fixed_d1<DEG>(knots, span, s, N, dN);
    double nx = 0, ny = 0, W = 0, dnx = 0, dny = 0, dW = 0;
#pragma unroll
    for (int r = 0; r <= DEG; ++r) {
        const int i = span - DEG + r;
        const double wi = w[i];
        const double px = ctrl[2 * i], py = ctrl[2 * i + 1];
        nx += wi * px * N[r]; ny += wi * py * N[r]; W += wi * N[r];
        dnx += wi * px * dN[r]; dny += wi * py * dN[r]; dW += wi * dN[r];
    }
    const double fx = nx / W, fy = ny / W;
    const double fx1 = (dnx - dW * fx) / W, fy1 = (dny - dW * fy) / W;
    out[q] = fx;
    out[count + q] = fy;
    out[2 * count + q] = fx1;
    out[3 * count + q] = fy1;
    out[4 * count + q] = sqrt(fx1 * fx1 + fy1 * fy1);
}

void geometry_eval(igs_geom g, const double* d_t, int count, double* d_out, cudaStream_t s) {
    if (count <= 0) return;
    const dim3 grid((count + 127) / 128), block(128);
    switch (g->degree) {
        case 1: k_geom<1><<<grid, block, 0, s>>>(g->n_ctrl, g->d_knots, g->d_ctrl, g->d_w, d_t, count, d_out); break;
        case 2: k_geom<2><<<grid, block, 0, s>>>(g->n_ctrl, g->d_knots, g->d_ctrl, g->d_w, d_t, count, d_out); break;
        case 3: k_geom<3><<<grid, block, 0, s>>>(g->n_ctrl, g->d_knots, g->d_ctrl, g->d_w, d_t, count, d_out); break;
        case 4: k_geom<4><<<grid, block, 0, s>>>(g->n_ctrl, g->d_knots, g->d_ctrl, g->d_w, d_t, count, d_out); break;
        case 5: k_geom<5><<<grid, block, 0, s>>>(g->n_ctrl, g->d_knots, g->d_ctrl, g->d_w, d_t, count, d_out); break;
        case 6: k_geom<6><<<grid, block, 0, s>>>(g->n_ctrl, g->d_knots, g->d_ctrl, g->d_w, d_t, count, d_out); break;
        default: k_geom<7><<<grid, block, 0, s>>>(g->n_ctrl, g->d_knots, g->d_ctrl, g->d_w, d_t, count, d_out); break;
    }
    IGS_CUDA(cudaGetLastError());
}

}  // namespace igs
