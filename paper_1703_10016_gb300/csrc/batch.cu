// Batched form of the assembly (Sect. 5 for many problems at once).  All the
// (problem, tile) units of a batch run in one persistent launch behind one
// batched geometry pass, both captured in a CUDA graph.  The unit order, the
// tile size and the number of CTAs per SM are parameters; igs_batch_tune
// times the candidates on the batch itself and keeps the fastest.
#include <algorithm>
#include <numeric>

#include "igs_internal.h"

using namespace igs;

struct igs_batch_s {
    igs_ctx ctx = nullptr;
    std::vector<igs_prob> probs;
    std::vector<igs_geom> built_for;           // geometry of each problem when the graph was built
    igs_batch_config cfg{32, IGS_ORDER_NATURAL, 0, 0.0f};
    int sms = 0;
    // device side of the current configuration
    BatchGeomF* d_geom = nullptr;
    BatchItemF* d_items = nullptr;
    int2* d_units = nullptr;
    int* d_counter = nullptr;
    int total_nodes = 0, nunits = 0, threads = 0, grid = 0;
    size_t smem = 0;
    cudaGraphExec_t exec = nullptr;
    float last_ms = 0.0f;
};

namespace {

void free_config(igs_batch b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    for (void* q : {(void*)b->d_geom, (void*)b->d_items, (void*)b->d_units, (void*)b->d_counter})
        if (q) cudaFree(q);
    b->d_geom = nullptr;
    b->d_items = nullptr;
    b->d_units = nullptr;
    b->d_counter = nullptr;
}

template <typename T>
T* upload_vec(const std::vector<T>& h, cudaStream_t s) {
    T* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(T) * std::max<size_t>(h.size(), 1));
    if (e != cudaSuccess) throw Error(IGS_E_NO_MEMORY, cuda_msg(e, "cudaMalloc", __FILE__, __LINE__));
    if (!h.empty()) IGS_CUDA(cudaMemcpyAsync(d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s));
    return d;
}

// Per-problem buffers the batch writes: rules, geometry and node records, A.
void prepare_problem(igs_prob p) {
    ensure_rules(p);
    const Plan& P = p->plan;
    const int D1 = P.d + 1;
    if (!p->d_geo) p->d_geo = (double*)dev_alloc(p, sizeof(double) * 5 * (size_t)P.Nq);
    if (!p->d_nodes) {
        p->d_nodes = dev_alloc(p, sizeof(NodeF) * (size_t)P.Nq);
        p->d_P = dev_alloc(p, sizeof(float) * (size_t)P.Nq * D1);
        p->d_Q = dev_alloc(p, sizeof(float) * (size_t)P.Nq * D1);
    }
    if (!p->d_A) p->d_A = dev_alloc(p, sizeof(float) * (size_t)P.n * P.n);
}

// Build the device descriptors, the unit list in the configured order and the graph.
void build(igs_batch b) {
    free_config(b);
    cudaStream_t s = b->ctx->stream;
    const int TI = b->cfg.tile;
    const int np = (int)b->probs.size();
    std::vector<BatchGeomF> geo(np);
    std::vector<BatchItemF> items(np);
    std::vector<int> ntiles(np);
    int node0 = 0, maxthreads = 32;
    size_t smem = 0;
    for (int k = 0; k < np; ++k) {
        igs_prob p = b->probs[k];
        prepare_problem(p);
        const Plan& P = p->plan;
        igs_geom g = p->geom;
        geo[k] = BatchGeomF{g->degree, g->n_ctrl, g->d_knots, g->d_ctrl, g->d_w, p->d_eta, P.Nq, P.d, P.L,
                            p->d_W, p->d_Bt, p->d_geo, (NodeF*)p->d_nodes, (float*)p->d_P, (float*)p->d_Q, node0};
        node0 += P.Nq;
        const int maxr = max_tile_range(P, TI);
        if (maxr > 512) throw Error(IGS_E_INVALID_ARG, "batch: a tile's node range exceeds 512 nodes");
        const int nt = (P.n + TI - 1) / TI;
        items[k] = BatchItemF{tile_args_f(p, maxr), P.d, P.closed, nt};
        items[k].t.AT = nullptr;                     // the batched form does not factor: no A^T
        ntiles[k] = nt * nt;
        maxthreads = std::max(maxthreads, (maxr + 31) / 32 * 32);
        smem = std::max(smem, tile_smem_f(maxr, P.d, TI));
        b->built_for[k] = g;
    }
    // unit order
    std::vector<int2> units;
    units.reserve(std::accumulate(ntiles.begin(), ntiles.end(), size_t(0)));
    std::vector<int> order(np);
    std::iota(order.begin(), order.end(), 0);
    if (b->cfg.order == IGS_ORDER_LARGEST_FIRST)
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return ntiles[x] > ntiles[y]; });
    if (b->cfg.order == IGS_ORDER_INTERLEAVED) {
        const int most = *std::max_element(ntiles.begin(), ntiles.end());
        for (int t = 0; t < most; ++t)
            for (int k = 0; k < np; ++k)
                if (t < ntiles[k]) units.push_back(make_int2(k, t));
    } else {
        for (int k : order)
            for (int t = 0; t < ntiles[k]; ++t) units.push_back(make_int2(k, t));
    }
    b->total_nodes = node0;
    b->nunits = (int)units.size();
    b->threads = maxthreads;
    b->smem = smem;
    const int per_sm = batch_blocks_per_sm(TI, maxthreads, smem);
    if (per_sm < 1) throw Error(IGS_E_INVALID_ARG, "batch: tile does not fit on an SM");
    const int want = b->cfg.ctas_per_sm > 0 ? std::min(b->cfg.ctas_per_sm, per_sm) : per_sm;
    b->cfg.ctas_per_sm = want;
    b->grid = std::max(1, std::min(b->nunits, want * b->sms));
    b->d_geom = upload_vec(geo, s);
    b->d_items = upload_vec(items, s);
    b->d_units = upload_vec(units, s);
    b->d_counter = upload_vec(std::vector<int>{0}, s);
    IGS_CUDA(cudaStreamSynchronize(s));

    // capture: counter reset, geometry pass, persistent assembly
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    IGS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    try {
        IGS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        try {
            IGS_CUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(int), cs));
            batch_geom_f(b->d_geom, np, b->total_nodes, cs);
            batch_assemble_f(TI, b->d_items, b->d_units, b->nunits, b->d_counter, b->grid, b->threads, b->smem, cs);
        } catch (...) {
            cudaStreamEndCapture(cs, &graph);
            if (graph) cudaGraphDestroy(graph);
            throw;
        }
        IGS_CUDA(cudaStreamEndCapture(cs, &graph));
        cudaError_t e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            throw Error(IGS_E_CUDA, cuda_msg(e, "cudaGraphInstantiate", __FILE__, __LINE__));
        }
    } catch (...) {
        cudaStreamDestroy(cs);
        throw;
    }
    cudaStreamDestroy(cs);
}

float run(igs_batch b) {
    bool stale = !b->exec;
    for (size_t k = 0; k < b->probs.size() && !stale; ++k) stale = b->probs[k]->geom != b->built_for[k];
    if (stale) build(b);
    cudaStream_t s = b->ctx->stream;
    cudaEvent_t e0, e1;
    IGS_CUDA(cudaEventCreate(&e0));
    IGS_CUDA(cudaEventCreate(&e1));
    IGS_CUDA(cudaEventRecord(e0, s));
    IGS_CUDA(cudaGraphLaunch(b->exec, s));
    IGS_CUDA(cudaEventRecord(e1, s));
    IGS_CUDA(cudaEventSynchronize(e1));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (igs_prob p : b->probs) {
        p->geometry_ready = 1;
        p->assembled = 1;
        p->factored = 0;
        p->at_ready = 0;                             // a later solve transposes A itself
    }
    b->last_ms = ms;
    return ms;
}

}  // namespace

extern "C" {

int igs_batch_create(igs_ctx ctx, igs_batch* out, const igs_prob* probs, int count) {
    API_BEGIN
    REQUIRE(ctx && out && probs && count > 0, IGS_E_INVALID_ARG, "ctx, out and probs must be set and count > 0");
    for (int k = 0; k < count; ++k) {
        REQUIRE(probs[k], IGS_E_INVALID_ARG, "a problem handle is NULL");
        REQUIRE(probs[k]->geom->ctx == ctx, IGS_E_INVALID_ARG, "problems must belong to ctx");
        REQUIRE(probs[k]->precision == IGS_MIXED, IGS_E_INVALID_ARG, "the batched form runs the MIXED tier");
    }
    IGS_CUDA(cudaSetDevice(ctx->device));
    auto* b = new igs_batch_s();
    b->ctx = ctx;
    b->probs.assign(probs, probs + count);
    b->built_for.assign(count, nullptr);
    IGS_CUDA(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, ctx->device));
    for (igs_prob p : b->probs) p->live_batches++;
    ctx->live_batches++;
    *out = b;
    API_END
}

int igs_batch_destroy(igs_batch b) {
    API_BEGIN
    REQUIRE(b, IGS_E_INVALID_ARG, "batch is NULL");
    IGS_CUDA(cudaSetDevice(b->ctx->device));
    cudaStreamSynchronize(b->ctx->stream);
    free_config(b);
    for (igs_prob p : b->probs) p->live_batches--;
    b->ctx->live_batches--;
    delete b;
    API_END
}

int igs_batch_assemble(igs_batch b, float* ms_out) {
    API_BEGIN
    REQUIRE(b, IGS_E_INVALID_ARG, "batch is NULL");
    IGS_CUDA(cudaSetDevice(b->ctx->device));
    const float ms = run(b);
    if (ms_out) *ms_out = ms;
    API_END
}

int igs_batch_set_config(igs_batch b, const igs_batch_config* cfg) {
    API_BEGIN
    REQUIRE(b && cfg, IGS_E_INVALID_ARG, "batch and cfg must be set");
    REQUIRE(cfg->tile == 16 || cfg->tile == 32, IGS_E_INVALID_ARG, "tile must be 16 or 32");
    REQUIRE(cfg->order >= IGS_ORDER_NATURAL && cfg->order <= IGS_ORDER_LARGEST_FIRST, IGS_E_INVALID_ARG,
            "unknown unit order");
    REQUIRE(cfg->ctas_per_sm >= 0, IGS_E_INVALID_ARG, "ctas_per_sm must be >= 0");
    IGS_CUDA(cudaSetDevice(b->ctx->device));
    b->cfg = *cfg;
    b->cfg.ms = 0.0f;
    free_config(b);
    API_END
}

int igs_batch_get_config(igs_batch b, igs_batch_config* cfg) {
    API_BEGIN
    REQUIRE(b && cfg, IGS_E_INVALID_ARG, "batch and cfg must be set");
    *cfg = b->cfg;
    cfg->ms = b->last_ms;
    API_END
}

int igs_batch_tune(igs_batch b, igs_batch_config* best_out, int reps) {
    API_BEGIN
    REQUIRE(b, IGS_E_INVALID_ARG, "batch is NULL");
    REQUIRE(reps >= 1 && reps <= 100, IGS_E_INVALID_ARG, "reps must be in [1, 100]");
    IGS_CUDA(cudaSetDevice(b->ctx->device));
    igs_batch_config best{32, IGS_ORDER_NATURAL, 0, 1e30f};
    for (int tile : {32, 16})
        for (int order : {IGS_ORDER_NATURAL, IGS_ORDER_INTERLEAVED, IGS_ORDER_LARGEST_FIRST})
            for (int frac : {1, 2}) {
                b->cfg = igs_batch_config{tile, order, 0, 0.0f};
                free_config(b);
                build(b);                                   // sets ctas_per_sm to the occupancy limit
                const int full = b->cfg.ctas_per_sm;
                if (frac == 2) {
                    if (full < 2) continue;
                    b->cfg.ctas_per_sm = full / 2;
                    free_config(b);
                    build(b);
                }
                run(b);                                     // warm-up
                float t = 1e30f;
                for (int r = 0; r < reps; ++r) t = std::min(t, run(b));
                if (t < best.ms) best = igs_batch_config{tile, order, b->cfg.ctas_per_sm, t};
            }
    b->cfg = best;
    free_config(b);
    build(b);
    if (best_out) *best_out = best;
    API_END
}

}  // extern "C"
