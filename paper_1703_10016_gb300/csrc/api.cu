#include <map>
// C ABI entry points (include/igs.h): handles, validation, allocation, copies.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "igs_internal.h"

namespace igs {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

void ensure_dyn_smem(const void* func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> limit;   // per device and kernel
    int dev = 0;
    IGS_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    size_t& cur = limit[{dev, func}];
    if (bytes <= cur) return;
    IGS_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cur = bytes;
}

std::string cuda_msg(cudaError_t e, const char* what, const char* file, int line) {
    return std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" + std::to_string(line) + ")";
}

struct AllocTable {
    std::mutex mu;
    std::unordered_map<void*, size_t> sizes;
};
static AllocTable& table() {
    static AllocTable t;
    return t;
}

void* dev_alloc(igs_prob p, size_t bytes) {
    void* ptr = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(&ptr, bytes, p->geom->ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(IGS_E_NO_MEMORY, "device allocation of " + std::to_string(bytes) + " bytes failed: " +
                                         cudaGetErrorString(e));
    }
    {
        std::lock_guard<std::mutex> lk(table().mu);
        table().sizes[ptr] = bytes;
    }
    p->bytes += (int64_t)bytes;
    return ptr;
}

void dev_free_raw(igs_prob p, void* ptr) {
    if (!ptr) return;
    size_t bytes = 0;
    {
        std::lock_guard<std::mutex> lk(table().mu);
        auto it = table().sizes.find(ptr);
        if (it != table().sizes.end()) { bytes = it->second; table().sizes.erase(it); }
    }
    cudaFreeAsync(ptr, p->geom->ctx->stream);
    p->bytes -= (int64_t)bytes;
}

void rhs_prepare(igs_prob p);

template <typename Tin, typename Tout>
__global__ void k_copy_convert(int n, const Tin* __restrict__ src, Tout* __restrict__ dst, int64_t ld) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
    if (j < n) dst[(size_t)i * ld + j] = (Tout)src[(size_t)i * n + j];
}

template <typename T>
static void upload(igs_prob p, T*& d, const std::vector<T>& h) {
    d = (T*)dev_alloc(p, sizeof(T) * std::max<size_t>(h.size(), 1));
    if (!h.empty())
        IGS_CUDA(cudaMemcpyAsync(d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, p->geom->ctx->stream));
}

void ensure_rules(igs_prob p) {
    if (!p->rules_ready) rules_build(p);
}

void ensure_geometry(igs_prob p) {
    ensure_rules(p);
    if (!p->geometry_ready) geometry_nodes(p);
}

}  // namespace igs

using namespace igs;

namespace igs {
// Copy the assembled A (tier type) to a caller buffer of the requested type.
static void copy_matrix(igs_prob p, void* A_out, int64_t ld, int mem, int dtype) {
    const Plan& P = p->plan;
    cudaStream_t s = p->geom->ctx->stream;
    const bool mixed = p->precision == IGS_MIXED;
    const size_t osz = dtype == IGS_F64 ? 8 : 4;
    void* dst = A_out;
    void* tmp = nullptr;
    if (mem == IGS_MEM_HOST) { tmp = dev_alloc(p, osz * (size_t)P.n * P.n); dst = tmp; }
    const int64_t dld = (mem == IGS_MEM_HOST) ? P.n : ld;
    dim3 grid((P.n + 255) / 256, P.n);
    if (mixed && dtype == IGS_F32) k_copy_convert<float, float><<<grid, 256, 0, s>>>(P.n, (const float*)p->d_A, (float*)dst, dld);
    else if (mixed) k_copy_convert<float, double><<<grid, 256, 0, s>>>(P.n, (const float*)p->d_A, (double*)dst, dld);
    else if (dtype == IGS_F32) k_copy_convert<double, float><<<grid, 256, 0, s>>>(P.n, (const double*)p->d_A, (float*)dst, dld);
    else k_copy_convert<double, double><<<grid, 256, 0, s>>>(P.n, (const double*)p->d_A, (double*)dst, dld);
    p->launches++;
    IGS_CUDA(cudaGetLastError());
    if (mem == IGS_MEM_HOST) {
        IGS_CUDA(cudaMemcpy2DAsync(A_out, ld * osz, tmp, P.n * osz, P.n * osz, P.n, cudaMemcpyDeviceToHost, s));
        IGS_CUDA(cudaStreamSynchronize(s));
        dev_free(p, tmp);
    }
}

}  // namespace igs

extern "C" {

const char* igs_last_error(void) { return g_last_error.c_str(); }

int igs_create(igs_ctx* out, int device, void* cuda_stream) {
    API_BEGIN
    REQUIRE(out, IGS_E_INVALID_ARG, "out is NULL");
    int count = 0;
    IGS_CUDA(cudaGetDeviceCount(&count));
    REQUIRE(device >= 0 && device < count, IGS_E_INVALID_ARG, "no such CUDA device");
    IGS_CUDA(cudaSetDevice(device));
    auto* c = new igs_ctx_s();
    c->device = device;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete c; throw Error(IGS_E_CUDA, cuda_msg(e, "cudaStreamCreate", __FILE__, __LINE__)); }
        c->own_stream = true;
    }
    *out = c;
    API_END
}

int igs_destroy(igs_ctx ctx) {
    API_BEGIN
    REQUIRE(ctx, IGS_E_INVALID_ARG, "ctx is NULL");
    REQUIRE(ctx->live_geoms == 0 && ctx->live_probs == 0 && ctx->live_batches == 0, IGS_E_STATE,
            "destroy batches, geometries and problems first");
    IGS_CUDA(cudaSetDevice(ctx->device));
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    API_END
}

int igs_selftest_wait(igs_ctx ctx, double budget_s, int* gave_up) {
    API_BEGIN
    REQUIRE(ctx && gave_up, IGS_E_INVALID_ARG, "ctx or gave_up is NULL");
    REQUIRE(budget_s == budget_s, IGS_E_INVALID_ARG, "budget is NaN");
    const int st = wait_selftest(ctx->device, std::min(2.0, std::max(1e-4, budget_s)));
    REQUIRE(st == 0 || st == 1, IGS_E_CUDA, "wait self-test kernel did not report");
    *gave_up = st;
    API_END
}

int igs_measure_peak(igs_ctx ctx, int kind, double* rate, double* ms) {
    API_BEGIN
    REQUIRE(ctx && rate, IGS_E_INVALID_ARG, "ctx or rate is NULL");
    REQUIRE(kind >= IGS_PEAK_FP32_FMA && kind <= IGS_PEAK_FP64_FMA, IGS_E_INVALID_ARG, "unknown peak kind");
    *rate = measure_peak(ctx->device, kind, ms);
    API_END
}

int igs_create_geometry(igs_ctx ctx, igs_geom* out, int degree, const double* knots, int n_knots,
                        const double* ctrl_xy, const double* weights, int n_ctrl, int closed) {
    API_BEGIN
    REQUIRE(ctx && out && knots && ctrl_xy, IGS_E_INVALID_ARG, "NULL argument");
    REQUIRE(degree >= 1 && degree <= kMaxGeomDegree, IGS_E_INVALID_ARG, "geometry degree must be in [1, 7]");
    REQUIRE(n_ctrl >= degree + 1, IGS_E_INVALID_ARG, "need n_ctrl >= degree + 1");
    REQUIRE(n_knots == n_ctrl + degree + 1, IGS_E_INVALID_ARG, "n_knots must equal n_ctrl + degree + 1");
    for (int k = 1; k < n_knots; ++k)
        REQUIRE(knots[k] >= knots[k - 1] && std::isfinite(knots[k]), IGS_E_INVALID_ARG, "knots must be non-decreasing");
    REQUIRE(knots[n_ctrl] > knots[degree], IGS_E_INVALID_ARG, "empty parameter interval");
    for (int k = 0; k < 2 * n_ctrl; ++k) REQUIRE(std::isfinite(ctrl_xy[k]), IGS_E_INVALID_ARG, "non-finite control point");
    if (weights)
        for (int k = 0; k < n_ctrl; ++k) REQUIRE(weights[k] > 0 && std::isfinite(weights[k]), IGS_E_INVALID_ARG, "weights must be positive");
    IGS_CUDA(cudaSetDevice(ctx->device));
    auto* g = new igs_geom_s();
    g->ctx = ctx; g->degree = degree; g->n_ctrl = n_ctrl; g->n_knots = n_knots; g->closed = closed ? 1 : 0;
    g->rational = weights ? 1 : 0;
    g->a = knots[degree]; g->b = knots[n_ctrl];
    std::vector<double> w(n_ctrl, 1.0);
    if (weights) std::copy(weights, weights + n_ctrl, w.begin());
    cudaStream_t s = ctx->stream;
    cudaError_t e1 = cudaMallocAsync((void**)&g->d_knots, sizeof(double) * n_knots, s);
    cudaError_t e2 = cudaMallocAsync((void**)&g->d_ctrl, sizeof(double) * 2 * n_ctrl, s);
    cudaError_t e3 = cudaMallocAsync((void**)&g->d_w, sizeof(double) * n_ctrl, s);
    if (e1 || e2 || e3) { delete g; throw Error(IGS_E_NO_MEMORY, "geometry allocation failed"); }
    IGS_CUDA(cudaMemcpyAsync(g->d_knots, knots, sizeof(double) * n_knots, cudaMemcpyHostToDevice, s));
    IGS_CUDA(cudaMemcpyAsync(g->d_ctrl, ctrl_xy, sizeof(double) * 2 * n_ctrl, cudaMemcpyHostToDevice, s));
    IGS_CUDA(cudaMemcpyAsync(g->d_w, w.data(), sizeof(double) * n_ctrl, cudaMemcpyHostToDevice, s));
    IGS_CUDA(cudaStreamSynchronize(s));
    ctx->live_geoms++;
    *out = g;
    API_END
}

int igs_destroy_geometry(igs_geom g) {
    API_BEGIN
    REQUIRE(g, IGS_E_INVALID_ARG, "geom is NULL");
    REQUIRE(g->live_probs == 0, IGS_E_STATE, "destroy the problems of this geometry first");
    IGS_CUDA(cudaSetDevice(g->ctx->device));
    cudaStream_t s = g->ctx->stream;
    cudaFreeAsync(g->d_knots, s); cudaFreeAsync(g->d_ctrl, s); cudaFreeAsync(g->d_w, s);
    cudaStreamSynchronize(s);
    g->ctx->live_geoms--;
    delete g;
    API_END
}

int igs_create_problem(igs_geom g, igs_prob* out, int degree, int n_elems, int n_ref, int precision) {
    API_BEGIN
    REQUIRE(g && out, IGS_E_INVALID_ARG, "NULL argument");
    REQUIRE(precision == IGS_FP64 || precision == IGS_MIXED, IGS_E_INVALID_ARG, "precision must be IGS_FP64 or IGS_MIXED");
    IGS_CUDA(cudaSetDevice(g->ctx->device));
    auto* p = new igs_prob_s();
    p->geom = g;
    p->precision = precision;
    std::string err;
    int rc = build_plan(p->plan, g->a, g->b, n_elems, degree, n_ref, g->closed, err);
    if (rc != IGS_OK) { delete p; throw Error(rc, err); }
    const Plan& P = p->plan;
    if (P.max_nodes_i > 64 || P.max_fine_i > 40) { delete p; throw Error(IGS_E_INVALID_ARG, "local rule system too large"); }
    if (P.n > 65535) { delete p; throw Error(IGS_E_INVALID_ARG, "n > 65535 is not supported"); }
    try {
        upload(p, p->d_pos, P.pos_num);
        upload(p, p->d_jfirst, P.jfirst);
        upload(p, p->d_member, P.member);
        upload(p, p->d_fspan, P.fspan);
        upload(p, p->d_lo, P.lo);
        upload(p, p->d_hi, P.hi);
        std::vector<int> jr(8 * (size_t)P.n);
        for (int i = 0; i < P.n; ++i) {
            int* r = &jr[8 * (size_t)i];
            r[0] = P.jlo1[i]; r[1] = P.jhi1[i]; r[2] = P.jlo2[i]; r[3] = P.jhi2[i];
            r[4] = P.elo1[i]; r[5] = P.ehi1[i]; r[6] = P.elo2[i]; r[7] = P.ehi2[i];
        }
        upload(p, p->d_jr, jr);
        upload(p, p->d_gfirst, P.gfirst);
        upload(p, p->d_glast, P.glast);
        upload(p, p->d_piece, P.piece);
        upload(p, p->d_series, P.series);
        p->d_flag = (int*)dev_alloc(p, sizeof(int));
        IGS_CUDA(cudaStreamSynchronize(g->ctx->stream));
    } catch (...) {
        delete p;
        throw;
    }
    g->live_probs++;
    g->ctx->live_probs++;
    *out = p;
    API_END
}

int igs_destroy_problem(igs_prob p) {
    API_BEGIN
    REQUIRE(p, IGS_E_INVALID_ARG, "prob is NULL");
    REQUIRE(p->live_batches == 0, IGS_E_STATE, "destroy the batches that hold this problem first");
    IGS_CUDA(cudaSetDevice(p->geom->ctx->device));
    void* ptrs[] = {p->d_pos, p->d_jfirst, p->d_member, p->d_fspan,
                     p->d_lo, p->d_hi, p->d_jr, p->d_gfirst, p->d_glast,
                     p->d_piece, p->d_series, p->d_eta, p->d_Bf,
                     p->d_Bt, p->d_W, p->d_G, p->d_Z, p->d_WsT,
                     p->d_WsT32, p->d_WsRow, p->d_WsRow32, p->d_WsToe, p->d_WsToe32,
                     p->d_flag, p->d_geo, p->d_nodes,
                     p->d_P, p->d_Q, p->d_A, p->d_AT, p->d_F, p->d_As64, p->d_dscale, p->d_diagL, p->d_diagLinv, p->d_diagLinv128, p->d_tflags, p->d_tpub, p->d_timg,
                     p->d_beta, p->d_rhs_geo, p->d_rhs_w, p->d_rhs_t, p->d_tree};
    if (p->aux_stream) {
        cudaStreamSynchronize(p->aux_stream);
        cudaStreamDestroy(p->aux_stream);
        p->aux_stream = nullptr;
    }
    for (void* q : ptrs) dev_free_raw(p, q);
    for (cudaEvent_t e : p->asm_ev)
        if (e) cudaEventDestroy(e);
    if (p->factor_exec) cudaGraphExecDestroy(p->factor_exec);
    cudaStreamSynchronize(p->geom->ctx->stream);
    p->geom->live_probs--;
    p->geom->ctx->live_probs--;
    delete p;
    API_END
}

int igs_set_geometry(igs_prob p, igs_geom g) {
    API_BEGIN
    REQUIRE(p && g, IGS_E_INVALID_ARG, "NULL argument");
    REQUIRE(g->ctx == p->geom->ctx, IGS_E_INVALID_ARG, "geometry belongs to another context");
    REQUIRE(g->closed == p->plan.closed, IGS_E_INVALID_ARG, "closed/open mismatch");
    REQUIRE(g->a == p->plan.a && g->b == p->plan.b, IGS_E_INVALID_ARG, "parameter interval differs");
    if (g != p->geom) {
        p->geom->live_probs--;
        g->live_probs++;
        p->geom = g;
        p->geometry_ready = 0;
        p->assembled = 0;
        p->factored = 0;
        p->rhs_n = 0;
        if (p->d_rhs_geo) {
            geometry_eval(g, p->d_rhs_t, p->Ng, p->d_rhs_geo, g->ctx->stream);
            rhs_tree_geometry(p, g->ctx->stream);
        }
    }
    API_END
}

int igs_problem_info(igs_prob p, igs_info* out) {
    API_BEGIN
    REQUIRE(p && out, IGS_E_INVALID_ARG, "NULL argument");
    const Plan& P = p->plan;
    std::memset(out, 0, sizeof(*out));
    out->n = P.n; out->degree = P.d; out->n_elems = P.Nh; out->n_ref = P.Nref; out->n_quad = P.Nq;
    out->n_exact = P.NE; out->n_rhs_pts = P.Nq + P.M * kGaussRhs; out->closed = P.closed;
    out->precision = p->precision; out->rules_ready = p->rules_ready; out->assembled = p->assembled;
    out->factored = p->factored; out->rhs_slots = rhs_slots(p); out->device_bytes = p->bytes;
    API_END
}

// Read the geometry and assembly times of the last igs_assemble once its
// kernels have finished (igs_assemble without a copy does not wait for them).
static void finish_assemble_timing(igs_prob p) {
    if (!p->asm_pending) return;
    p->asm_pending = false;
    IGS_CUDA(cudaEventSynchronize(p->asm_ev[2]));
    float g_ms = 0, a_ms = 0;
    IGS_CUDA(cudaEventElapsedTime(&g_ms, p->asm_ev[0], p->asm_ev[1]));
    IGS_CUDA(cudaEventElapsedTime(&a_ms, p->asm_ev[1], p->asm_ev[2]));
    p->timing.geometry_ms = g_ms;
    p->timing.assemble_ms = a_ms;
}

int igs_problem_timing(igs_prob p, igs_timing* out) {
    API_BEGIN
    REQUIRE(p && out, IGS_E_INVALID_ARG, "NULL argument");
    finish_assemble_timing(p);
    *out = p->timing;
    API_END
}

int igs_build_weighted_rules(igs_prob p) {
    API_BEGIN
    REQUIRE(p, IGS_E_INVALID_ARG, "prob is NULL");
    IGS_CUDA(cudaSetDevice(p->geom->ctx->device));
    p->launches = 0;
    ensure_rules(p);
    p->timing.kernel_launches = p->launches;
    API_END
}

int igs_assemble(igs_prob p, void* A_out, int64_t ld, int mem, int dtype) {
    API_BEGIN
    REQUIRE(p, IGS_E_INVALID_ARG, "prob is NULL");
    const Plan& P = p->plan;
    if (A_out) {
        REQUIRE(ld >= P.n, IGS_E_INVALID_ARG, "ld < n");
        REQUIRE(mem == IGS_MEM_HOST || mem == IGS_MEM_DEVICE, IGS_E_INVALID_ARG, "bad mem kind");
        REQUIRE(dtype == IGS_F64 || dtype == IGS_F32, IGS_E_INVALID_ARG, "bad dtype");
    }
    IGS_CUDA(cudaSetDevice(p->geom->ctx->device));
    cudaStream_t s = p->geom->ctx->stream;
    finish_assemble_timing(p);
    p->launches = 0;
    ensure_rules(p);
    for (cudaEvent_t& e : p->asm_ev)
        if (!e) IGS_CUDA(cudaEventCreate(&e));
    IGS_CUDA(cudaEventRecord(p->asm_ev[0], s));
    geometry_nodes(p);
    IGS_CUDA(cudaEventRecord(p->asm_ev[1], s));
    assemble_matrix(p);
    IGS_CUDA(cudaEventRecord(p->asm_ev[2], s));
    p->assembled = 1;
    p->factored = 0;
    p->asm_pending = true;
    if (A_out) {
        copy_matrix(p, A_out, ld, mem, dtype);
        finish_assemble_timing(p);
    }
    p->timing.kernel_launches = p->launches;
    API_END
}

int igs_get_matrix(igs_prob p, void* A_out, int64_t ld, int mem, int dtype) {
    API_BEGIN
    REQUIRE(p && A_out, IGS_E_INVALID_ARG, "prob and A_out must be set");
    REQUIRE(p->assembled, IGS_E_STATE, "not assembled");
    REQUIRE(ld >= p->plan.n, IGS_E_INVALID_ARG, "ld < n");
    REQUIRE(mem == IGS_MEM_HOST || mem == IGS_MEM_DEVICE, IGS_E_INVALID_ARG, "bad mem kind");
    REQUIRE(dtype == IGS_F64 || dtype == IGS_F32, IGS_E_INVALID_ARG, "bad dtype");
    IGS_CUDA(cudaSetDevice(p->geom->ctx->device));
    copy_matrix(p, A_out, ld, mem, dtype);
    IGS_CUDA(cudaStreamSynchronize(p->geom->ctx->stream));
    API_END
}

int igs_rhs_points(igs_prob p, double* xy_out, int64_t capacity, int64_t* count) {
    API_BEGIN
    REQUIRE(p && count, IGS_E_INVALID_ARG, "NULL argument");
    IGS_CUDA(cudaSetDevice(p->geom->ctx->device));
    const Plan& P = p->plan;
    *count = (int64_t)P.Nq + (int64_t)P.M * kGaussRhs;
    if (!xy_out) return IGS_OK;
    REQUIRE(capacity >= *count, IGS_E_INVALID_ARG, "capacity too small");
    p->launches = 0;
    ensure_geometry(p);
    rhs_prepare(p);
    cudaStream_t s = p->geom->ctx->stream;
    std::vector<double> g1(2 * (size_t)P.Nq), g2(2 * (size_t)p->Ng);
    IGS_CUDA(cudaMemcpyAsync(g1.data(), p->d_geo, sizeof(double) * 2 * P.Nq, cudaMemcpyDeviceToHost, s));
    IGS_CUDA(cudaMemcpyAsync(g2.data(), p->d_rhs_geo, sizeof(double) * 2 * p->Ng, cudaMemcpyDeviceToHost, s));
    IGS_CUDA(cudaStreamSynchronize(s));
    for (int m = 0; m < P.Nq; ++m) { xy_out[2 * m] = g1[m]; xy_out[2 * m + 1] = g1[P.Nq + m]; }
    for (int q = 0; q < p->Ng; ++q) {
        xy_out[2 * (P.Nq + q)] = g2[q];
        xy_out[2 * (P.Nq + q) + 1] = g2[p->Ng + q];
    }
    API_END
}

int igs_build_rhs(igs_prob p, const double* uD, int nrhs, double* beta_out, int mem) {
    API_BEGIN
    REQUIRE(p && uD, IGS_E_INVALID_ARG, "NULL argument");
    REQUIRE(nrhs >= 1 && nrhs <= 8, IGS_E_INVALID_ARG, "nrhs must be in [1, 8]");
    REQUIRE(mem == IGS_MEM_HOST || mem == IGS_MEM_DEVICE, IGS_E_INVALID_ARG, "bad mem kind");
    IGS_CUDA(cudaSetDevice(p->geom->ctx->device));
    cudaStream_t s = p->geom->ctx->stream;
    p->launches = 0;
    ensure_geometry(p);
    rhs_prepare(p);
    const Plan& P = p->plan;
    const size_t cnt = (size_t)(P.Nq + p->Ng) * nrhs;
    cudaEvent_t e0, e1;
    IGS_CUDA(cudaEventCreate(&e0)); IGS_CUDA(cudaEventCreate(&e1));
    IGS_CUDA(cudaEventRecord(e0, s));
    double* d_u = nullptr;
    if (mem == IGS_MEM_HOST) {
        d_u = (double*)dev_alloc(p, sizeof(double) * cnt);
        IGS_CUDA(cudaMemcpyAsync(d_u, uD, sizeof(double) * cnt, cudaMemcpyHostToDevice, s));
    }
    rhs_build(p, d_u ? d_u : uD, nrhs);
    if (beta_out)
        IGS_CUDA(cudaMemcpyAsync(beta_out, p->d_beta, sizeof(double) * (size_t)P.n * nrhs,
                                 mem == IGS_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    IGS_CUDA(cudaEventRecord(e1, s));
    IGS_CUDA(cudaStreamSynchronize(s));
    if (d_u) dev_free(p, d_u);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    p->timing.rhs_ms = ms;
    cudaEventDestroy(e0); cudaEventDestroy(e1);
    p->timing.kernel_launches = p->launches;
    API_END
}

int igs_eval_potential(igs_prob p, const double* alpha, const double* uD, int nrhs, const double* xy, int64_t count,
                       double* u_out, int mem) {
    API_BEGIN
    REQUIRE(p && alpha && (count == 0 || (xy && u_out)), IGS_E_INVALID_ARG, "NULL argument");
    REQUIRE(nrhs >= 1 && nrhs <= 8, IGS_E_INVALID_ARG, "nrhs must be in [1, 8]");
    REQUIRE(count >= 0, IGS_E_INVALID_ARG, "count must be >= 0");
    REQUIRE(mem == IGS_MEM_HOST || mem == IGS_MEM_DEVICE, IGS_E_INVALID_ARG, "bad mem kind");
    REQUIRE(!p->plan.closed || uD, IGS_E_INVALID_ARG, "a closed curve needs u_D at the right-hand side points");
    if (count == 0) return IGS_OK;
    IGS_CUDA(cudaSetDevice(p->geom->ctx->device));
    cudaStream_t s = p->geom->ctx->stream;
    p->launches = 0;
    rhs_prepare(p);
    const Plan& P = p->plan;
    const size_t na = (size_t)nrhs * P.n, nu = p->plan.closed ? (size_t)nrhs * (P.Nq + p->Ng) : 0;
    const double *d_alpha = alpha, *d_uD = p->plan.closed ? uD : nullptr, *d_xy = xy;
    double* d_u = u_out;
    double* tmp = nullptr;
    if (mem == IGS_MEM_HOST) {
        const size_t tot = na + nu + 2 * (size_t)count + (size_t)nrhs * count;
        tmp = (double*)dev_alloc(p, sizeof(double) * tot);
        double* t_alpha = tmp;
        double* t_uD = t_alpha + na;
        double* t_xy = t_uD + nu;
        d_u = t_xy + 2 * (size_t)count;
        IGS_CUDA(cudaMemcpyAsync(t_alpha, alpha, sizeof(double) * na, cudaMemcpyHostToDevice, s));
        if (nu) IGS_CUDA(cudaMemcpyAsync(t_uD, uD, sizeof(double) * nu, cudaMemcpyHostToDevice, s));
        IGS_CUDA(cudaMemcpyAsync(t_xy, xy, sizeof(double) * 2 * (size_t)count, cudaMemcpyHostToDevice, s));
        d_alpha = t_alpha;
        d_uD = nu ? t_uD : nullptr;
        d_xy = t_xy;
    }
    try {
        potential_eval(p, d_alpha, d_uD, nrhs, d_xy, count, d_u);
        if (tmp) {
            IGS_CUDA(cudaMemcpyAsync(u_out, d_u, sizeof(double) * (size_t)nrhs * count, cudaMemcpyDeviceToHost, s));
            IGS_CUDA(cudaStreamSynchronize(s));
        }
    } catch (...) {
        if (tmp) { cudaStreamSynchronize(s); dev_free(p, tmp); }
        throw;
    }
    if (tmp) dev_free(p, tmp);
    p->timing.kernel_launches = p->launches;
    API_END
}

int igs_collocation(igs_prob p, const double* uD, int nrhs, double* alpha_out, double* Ac_out, int32_t* nodes_out,
                    int mem) {
    API_BEGIN
    REQUIRE(p && uD && alpha_out, IGS_E_INVALID_ARG, "NULL argument");
    REQUIRE(nrhs >= 1 && nrhs <= 8, IGS_E_INVALID_ARG, "nrhs must be in [1, 8]");
    REQUIRE(mem == IGS_MEM_HOST || mem == IGS_MEM_DEVICE, IGS_E_INVALID_ARG, "bad mem kind");
    REQUIRE(p->plan.closed, IGS_E_INVALID_ARG, "collocation is implemented for closed curves only");
    IGS_CUDA(cudaSetDevice(p->geom->ctx->device));
    cudaStream_t s = p->geom->ctx->stream;
    p->launches = 0;
    ensure_geometry(p);
    rhs_prepare(p);
    const Plan& P = p->plan;
    const size_t nu = (size_t)nrhs * (P.Nq + p->Ng), na = (size_t)nrhs * P.n;
    const double* d_uD = uD;
    double* d_alpha = alpha_out;
    double* tmp = nullptr;
    if (mem == IGS_MEM_HOST) {
        tmp = (double*)dev_alloc(p, sizeof(double) * (nu + na));
        IGS_CUDA(cudaMemcpyAsync(tmp, uD, sizeof(double) * nu, cudaMemcpyHostToDevice, s));
        d_uD = tmp;
        d_alpha = tmp + nu;
    }
    try {
        collocation_solve(p, d_uD, nrhs, d_alpha, Ac_out, mem, nodes_out);
        if (tmp) {
            IGS_CUDA(cudaMemcpyAsync(alpha_out, d_alpha, sizeof(double) * na, cudaMemcpyDeviceToHost, s));
            IGS_CUDA(cudaStreamSynchronize(s));
        }
    } catch (...) {
        if (tmp) { cudaStreamSynchronize(s); dev_free(p, tmp); }
        throw;
    }
    if (tmp) dev_free(p, tmp);
    p->timing.kernel_launches = p->launches;
    API_END
}

int igs_solve_data(igs_prob p, const double* uD, int nrhs, double* alpha_out, double* resid_out, int mem) {
    API_BEGIN
    REQUIRE(p && uD && alpha_out, IGS_E_INVALID_ARG, "NULL argument");
    REQUIRE(nrhs >= 1 && nrhs <= 8, IGS_E_INVALID_ARG, "nrhs must be in [1, 8]");
    REQUIRE(mem == IGS_MEM_HOST || mem == IGS_MEM_DEVICE, IGS_E_INVALID_ARG, "bad mem kind");
    REQUIRE(p->assembled, IGS_E_STATE, "assemble before solve");
    IGS_CUDA(cudaSetDevice(p->geom->ctx->device));
    cudaStream_t s = p->geom->ctx->stream;
    p->launches = 0;
    rhs_prepare(p);
    const Plan& P = p->plan;
    const size_t nu = (size_t)nrhs * (P.Nq + p->Ng), na = (size_t)nrhs * P.n;
    const double* d_uD = uD;
    double* d_alpha = alpha_out;
    double* tmp = nullptr;
    if (mem == IGS_MEM_HOST) {
        tmp = (double*)dev_alloc(p, sizeof(double) * (nu + na));
        IGS_CUDA(cudaMemcpyAsync(tmp, uD, sizeof(double) * nu, cudaMemcpyHostToDevice, s));
        d_uD = tmp;
        d_alpha = tmp + nu;
    }
    std::vector<double> res(nrhs, 0.0);
    try {
        solve_with_data(p, d_uD, nrhs, d_alpha, res.data());
        if (tmp) {
            IGS_CUDA(cudaMemcpyAsync(alpha_out, d_alpha, sizeof(double) * na, cudaMemcpyDeviceToHost, s));
            IGS_CUDA(cudaStreamSynchronize(s));
        }
    } catch (...) {
        if (tmp) { cudaStreamSynchronize(s); dev_free(p, tmp); }
        throw;
    }
    if (tmp) dev_free(p, tmp);
    if (resid_out) std::copy(res.begin(), res.end(), resid_out);
    p->timing.kernel_launches = p->launches;
    API_END
}

int igs_build_rhs_noalloc(igs_prob p, const double* uD, int nrhs, double* beta_out) {
    API_BEGIN
    REQUIRE(p && uD && beta_out, IGS_E_INVALID_ARG, "NULL argument");
    IGS_CUDA(cudaSetDevice(p->geom->ctx->device));
    p->launches = 0;
    rhs_build_noalloc(p, uD, nrhs, beta_out);
    p->timing.kernel_launches = p->launches;
    API_END
}

int igs_solve(igs_prob p, const double* beta, int nrhs, double* alpha_out, double* resid_out, int mem) {
    API_BEGIN
    REQUIRE(p && alpha_out, IGS_E_INVALID_ARG, "NULL argument");
    REQUIRE(mem == IGS_MEM_HOST || mem == IGS_MEM_DEVICE, IGS_E_INVALID_ARG, "bad mem kind");
    REQUIRE(p->assembled, IGS_E_STATE, "assemble before solve");
    IGS_CUDA(cudaSetDevice(p->geom->ctx->device));
    cudaStream_t s = p->geom->ctx->stream;
    const Plan& P = p->plan;
    p->launches = 0;
    double* d_beta = nullptr;
    double* own_beta = nullptr;
    if (!beta) {
        REQUIRE(p->d_beta && p->rhs_n > 0, IGS_E_STATE, "no right-hand side: call igs_build_rhs or pass beta");
        REQUIRE(nrhs <= p->rhs_n, IGS_E_INVALID_ARG, "nrhs exceeds the built right-hand sides");
        d_beta = p->d_beta;
    } else if (mem == IGS_MEM_DEVICE) {
        d_beta = (double*)beta;
    } else {
        own_beta = (double*)dev_alloc(p, sizeof(double) * (size_t)P.n * nrhs);
        IGS_CUDA(cudaMemcpyAsync(own_beta, beta, sizeof(double) * (size_t)P.n * nrhs, cudaMemcpyHostToDevice, s));
        d_beta = own_beta;
    }
    double* d_alpha = (mem == IGS_MEM_DEVICE) ? alpha_out : (double*)dev_alloc(p, sizeof(double) * (size_t)P.n * nrhs);
    std::vector<double> res(nrhs, 0.0);
    try {
        solve_system(p, d_beta, nrhs, d_alpha, res.data());
    } catch (...) {
        if (own_beta) dev_free(p, own_beta);
        if (mem != IGS_MEM_DEVICE) dev_free(p, d_alpha);
        throw;
    }
    if (mem == IGS_MEM_HOST) {
        IGS_CUDA(cudaMemcpyAsync(alpha_out, d_alpha, sizeof(double) * (size_t)P.n * nrhs, cudaMemcpyDeviceToHost, s));
        IGS_CUDA(cudaStreamSynchronize(s));
        dev_free(p, d_alpha);
    }
    if (own_beta) dev_free(p, own_beta);
    if (resid_out) std::copy(res.begin(), res.end(), resid_out);
    p->timing.kernel_launches = p->launches;
    API_END
}

int igs_get_rules(igs_prob p, double* eta, double* W_band, int32_t* first, double* Ws) {
    API_BEGIN
    REQUIRE(p, IGS_E_INVALID_ARG, "prob is NULL");
    IGS_CUDA(cudaSetDevice(p->geom->ctx->device));
    ensure_rules(p);
    const Plan& P = p->plan;
    cudaStream_t s = p->geom->ctx->stream;
    if (eta) IGS_CUDA(cudaMemcpyAsync(eta, p->d_eta, sizeof(double) * P.Nq, cudaMemcpyDeviceToHost, s));
    if (W_band) IGS_CUDA(cudaMemcpyAsync(W_band, p->d_W, sizeof(double) * P.Nq * (P.d + 1), cudaMemcpyDeviceToHost, s));
    if (first) std::copy(P.jfirst.begin(), P.jfirst.end(), first);
    if (Ws) {
        REQUIRE(P.Nq <= 65535, IGS_E_INVALID_ARG, "dense W^s download is limited to n_quad <= 65535");
        double* d_ws = (double*)dev_alloc(p, sizeof(double) * (size_t)P.Nq * P.Nq);
        ws_expand(p, d_ws);
        cudaError_t e = cudaMemcpyAsync(Ws, d_ws, sizeof(double) * (size_t)P.Nq * P.Nq, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        dev_free(p, d_ws);
        if (e != cudaSuccess) throw Error(IGS_E_CUDA, cuda_msg(e, "cudaMemcpyAsync", __FILE__, __LINE__));
    }
    IGS_CUDA(cudaStreamSynchronize(s));
    API_END
}

int igs_get_node_geometry(igs_prob p, double* xy, double* J) {
    API_BEGIN
    REQUIRE(p, IGS_E_INVALID_ARG, "prob is NULL");
    REQUIRE(p->geometry_ready, IGS_E_STATE, "geometry not evaluated yet");
    IGS_CUDA(cudaSetDevice(p->geom->ctx->device));
    const Plan& P = p->plan;
    cudaStream_t s = p->geom->ctx->stream;
    std::vector<double> g(5 * (size_t)P.Nq);
    IGS_CUDA(cudaMemcpyAsync(g.data(), p->d_geo, sizeof(double) * g.size(), cudaMemcpyDeviceToHost, s));
    IGS_CUDA(cudaStreamSynchronize(s));
    for (int m = 0; m < P.Nq; ++m) {
        if (xy) { xy[2 * m] = g[m]; xy[2 * m + 1] = g[P.Nq + m]; }
        if (J) J[m] = g[4 * (size_t)P.Nq + m];
    }
    API_END
}

}  // extern "C"
