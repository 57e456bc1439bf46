// Boundary curve evaluation (Sect. 3): f, f' and the parametric speed J = |f'| (eq. J).
#include "bspline_dev.cuh"
#include "igs_internal.h"

namespace igs {

// Curve evaluation at `count` parameters; out is SoA [5][count]: x, y, x', y', J.
template <int DEG>
__global__ void k_geom(int nb, const double* __restrict__ knots, const double* __restrict__ ctrl,
                       const double* __restrict__ w, const double* __restrict__ t, int count, double* __restrict__ out) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= count) return;
    double v[5];
    curve_point<DEG>(nb, knots, ctrl, w, t[q], v);
#pragma unroll
    for (int c = 0; c < 5; ++c) out[(size_t)c * count + q] = v[c];
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
