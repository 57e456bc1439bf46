// Served form: a request loop around the method (rules, assembly, right-hand
// sides and solve of Sects. 3-5 per request).  `slots` worker threads each own
// a context with its own CUDA stream; a worker takes the oldest queued request
// as soon as its device-memory estimate fits in what the running requests
// leave of the budget (first come, first served: a large request at the head
// is not overtaken), runs it through the library's own entry points (the
// right-hand side beside the factorisation, as igs_solve_data does), stores
// the result and frees its memory share.  Requests on different slots overlap
// on the device; each one's arithmetic is the same as when it runs alone.
// With a cache budget, each slot keeps the problems of its recent requests
// (rules, matrix, factor) resident and reuses them for requests on the same
// discretisation (rules, curve swapped in) or the same curve (factor too).
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "igs_internal.h"

using namespace igs;
using Clock = std::chrono::steady_clock;

namespace {

struct Ticket {
    igs_request req{};
    std::vector<double> knots, ctrl, w;
    int64_t est = 0;
    Clock::time_point t_submit, t_admit, t_done;
    int status = IGS_REQ_QUEUED, error = IGS_OK, slot = -1, n = 0, ir = 0, reuse = IGS_REUSE_NONE;
    std::string msg;
    std::vector<double> alpha, resid;
};

// A resident problem of one slot: its discretisation key, the curve it holds
// (degree, closed, knots, control points, weights, for an exact match), the
// device bytes it keeps and its last use.
struct Resident {
    std::vector<double> key, curve;
    igs_geom g = nullptr;
    igs_prob p = nullptr;
    int64_t bytes = 0;
    uint64_t last = 0;
};

void drop(Resident& r) {
    if (r.p) igs_destroy_problem(r.p);
    if (r.g) igs_destroy_geometry(r.g);
    r.p = nullptr;
    r.g = nullptr;
}

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// Device bytes a request holds at its peak: the matrix, its transpose and the
// factor (n^2 each in the tier type) and, in the FP64 tier, the symmetric copy
// for the residuals (n^2 FP64), the stored
// rules and their construction work arrays, node data, the right-hand sides
// and the double-layer scratch; 25% margin.
int64_t estimate_bytes(const igs_request& r) {
    const int64_t d = r.degree, Nh = r.n_elems, M = (int64_t)r.n_ref * Nh;
    const int64_t n = r.closed ? Nh : Nh + d;
    const int64_t Nq = 2 * d + 2 * M - 1, NE = M + d, D1 = d + 1;
    const int64_t tsz = r.precision == IGS_MIXED ? 4 : 8;
    int64_t b = n * n * (3 * tsz + (r.precision == IGS_MIXED ? 0 : 8));
    const int64_t B = 24 * D1 + 16, R = d + 2, ncols = 2 * B + 4;
    if (Nq < 2 * B + 2 * R + 64) b += Nq * Nq * 12 + NE * Nq * 8;
    else b += ncols * Nq * 8 + ncols * NE * 8 + (2 * B + 2 * R + 4) * Nq * 12 + ncols * 1024 * D1 * 8;
    b += 2 * M * 2 * D1 * D1 * 8;                       // element-moment table
    b += Nq * 160 + n * 64 * 2 * tsz + (int64_t)r.nrhs * (n * 40 + M * 40);
    b += M * igs::kGaussRhs * (7 * 8 + (int64_t)r.nrhs * 8);  // b2 rule: points, weights, geometry, u_D there
    if (r.closed)                                        // double-layer scratch (FP64 slices or treecode moments)
        b += M * igs::kGaussRhs * 28 + (int64_t)r.nrhs * 12 * Nq * 8;
    b += n * 8 * 8;                                      // published solution words
    if (r.precision == IGS_MIXED && n % 4 == 0 && n >= 256)
        b += n * 128 * 4;                                // inverses of the 128-row diagonal blocks
    if (r.precision == IGS_MIXED && n >= 4096)           // split operand images of two 512-column outer blocks
        b += (int64_t)2 * 16 * 2 * (4 * ((n + 255) / 256)) * 4096;
    return b + b / 4 + (1 << 20);
}

}  // namespace

struct igs_server_s {
    int device = 0;
    igs_server_opts opts{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> queue;
    std::unordered_map<int64_t, std::unique_ptr<Ticket>> tickets;
    int64_t next_id = 1, mem_in_use = 0;
    int unfinished = 0;
    bool stop = false;
    std::vector<igs_ctx> ctxs;
    std::vector<std::thread> workers;
    std::vector<std::vector<Resident>> kept;   // per slot, guarded by mu (only the slot's thread uses the problems)
    int64_t kept_bytes = 0;
    uint64_t clock = 0;
};

namespace {

// Take the slot's resident problem for `key` out of its list (nullptr-free
// Resident if none).
Resident take_resident(igs_server s, int slot, const std::vector<double>& key) {
    std::lock_guard<std::mutex> lk(s->mu);
    auto& v = s->kept[slot];
    for (size_t k = 0; k < v.size(); ++k)
        if (v[k].key == key) {
            Resident r = std::move(v[k]);
            v.erase(v.begin() + (long)k);
            s->kept_bytes -= r.bytes;
            return r;
        }
    return Resident{};
}

// Keep a problem resident after its request; trims the slot's least recently
// used problems while all slots together keep more than the cache budget.
void keep_resident(igs_server s, int slot, Resident r) {
    std::vector<Resident> out;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r.last = ++s->clock;
        s->kept_bytes += r.bytes;
        s->kept[slot].push_back(std::move(r));
        auto& v = s->kept[slot];
        while (s->kept_bytes > s->opts.cache_budget && !v.empty()) {
            size_t lru = 0;
            for (size_t k = 1; k < v.size(); ++k)
                if (v[k].last < v[lru].last) lru = k;
            s->kept_bytes -= v[lru].bytes;
            out.push_back(std::move(v[lru]));
            v.erase(v.begin() + (long)lru);
        }
    }
    for (Resident& q : out) drop(q);
}

void run_request(igs_server s, int slot, Ticket& t) {
    igs_ctx ctx = s->ctxs[slot];
    const igs_request& r = t.req;
    Resident res;
    igs_geom g = nullptr;
    auto fail = [&](int rc, const std::string& m) {
        t.error = rc;
        t.msg = m;
    };
    int rc = igs_create_geometry(ctx, &g, r.geom_degree, t.knots.data(), (int)t.knots.size(), t.ctrl.data(),
                                 t.w.empty() ? nullptr : t.w.data(), r.n_ctrl, r.closed);
    std::vector<double> key, curve;
    bool need_asm = false;
    if (rc == IGS_OK) {
        key = {(double)r.degree, (double)r.n_elems, (double)r.n_ref, (double)r.precision, (double)r.closed, g->a, g->b};
        curve = {(double)r.geom_degree, (double)r.closed, (double)t.knots.size(), (double)r.n_ctrl};
        curve.insert(curve.end(), t.knots.begin(), t.knots.end());
        curve.insert(curve.end(), t.ctrl.begin(), t.ctrl.end());
        curve.insert(curve.end(), t.w.begin(), t.w.end());
        if (s->opts.cache_budget > 0) res = take_resident(s, slot, key);
        if (res.p && res.curve == curve) {
            // same curve: matrix and factor are still valid
            igs_destroy_geometry(g);
            g = nullptr;
            t.reuse = IGS_REUSE_FACTOR;
        } else if (res.p) {
            rc = igs_set_geometry(res.p, g);
            if (rc == IGS_OK) {
                igs_destroy_geometry(res.g);
                res.g = g;
                g = nullptr;
                res.curve = curve;
                t.reuse = IGS_REUSE_RULES;
                need_asm = true;
            }
        } else {
            res.key = key;
            res.curve = curve;
            res.g = g;
            g = nullptr;
            rc = igs_create_problem(res.g, &res.p, r.degree, r.n_elems, r.n_ref, r.precision);
            if (rc == IGS_OK) rc = igs_build_weighted_rules(res.p);
            need_asm = true;
        }
    }
    igs_prob p = res.p;
    igs_info info{};
    if (rc == IGS_OK) rc = igs_problem_info(p, &info);
    int64_t count = 0;
    std::vector<double> xy, uD;
    if (rc == IGS_OK) rc = igs_rhs_points(p, nullptr, 0, &count);
    if (rc == IGS_OK) {
        xy.resize(2 * count);
        rc = igs_rhs_points(p, xy.data(), count, &count);
    }
    // the assembly runs on the device while the data callback runs here
    if (rc == IGS_OK && need_asm) rc = igs_assemble(p, nullptr, 0, IGS_MEM_HOST, IGS_F64);
    if (rc != IGS_OK) {
        fail(rc, igs_last_error());
    } else {
        uD.assign((size_t)r.nrhs * count, 0.0);
        if (r.data(r.user, xy.data(), count, r.nrhs, uD.data()) != 0) {
            fail(IGS_E_INVALID_ARG, "the data callback reported an error");
        } else {
            t.n = info.n;
            t.alpha.assign((size_t)r.nrhs * info.n, 0.0);
            t.resid.assign(r.nrhs, 0.0);
            // right-hand side on the problem's second stream beside the factorisation
            rc = igs_solve_data(p, uD.data(), r.nrhs, t.alpha.data(), t.resid.data(), IGS_MEM_HOST);
            igs_timing tm{};
            if (rc == IGS_OK && igs_problem_timing(p, &tm) == IGS_OK) t.ir = tm.ir_iterations;
            if (rc != IGS_OK) fail(rc, igs_last_error());
        }
    }
    if (g) igs_destroy_geometry(g);
    if (t.error == IGS_OK && p && s->opts.cache_budget > 0 && igs_problem_info(p, &info) == IGS_OK &&
        info.device_bytes <= s->opts.cache_budget) {
        res.bytes = info.device_bytes;
        keep_resident(s, slot, std::move(res));
    } else {
        drop(res);
    }
}

void worker(igs_server s, int slot) {
    cudaSetDevice(s->device);
    for (;;) {
        int64_t id = 0;
        Ticket* t = nullptr;
        Resident spill;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            auto fits = [&] {
                const Ticket& head = *s->tickets.at(s->queue.front());
                return s->mem_in_use + s->kept_bytes + head.est <= s->opts.mem_budget;
            };
            s->cv_work.wait(lk, [&] {
                if (s->stop) return true;
                if (s->queue.empty()) return false;
                return fits() || !s->kept[slot].empty();
            });
            if (s->stop && s->queue.empty()) return;
            if (s->queue.empty()) continue;
            if (!fits()) {
                // the oldest request waits for memory: give up this slot's oldest resident problem
                auto& v = s->kept[slot];
                size_t lru = 0;
                for (size_t k = 1; k < v.size(); ++k)
                    if (v[k].last < v[lru].last) lru = k;
                s->kept_bytes -= v[lru].bytes;
                spill = std::move(v[lru]);
                v.erase(v.begin() + (long)lru);
            } else {
                id = s->queue.front();
                s->queue.pop_front();
                t = s->tickets.at(id).get();
                s->mem_in_use += t->est;
                t->status = IGS_REQ_RUNNING;
                t->slot = slot;
                t->t_admit = Clock::now();
            }
        }
        if (!t) {
            drop(spill);
            s->cv_work.notify_all();
            continue;
        }
        // the next queued request may fit as well
        s->cv_work.notify_all();
        run_request(s, slot, *t);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            t->t_done = Clock::now();
            t->status = t->error == IGS_OK ? IGS_REQ_DONE : IGS_REQ_FAILED;
            s->mem_in_use -= t->est;
            s->unfinished--;
        }
        s->cv_work.notify_all();
        s->cv_done.notify_all();
    }
}

void fill_stats(const Ticket& t, igs_request_stats* st) {
    if (!st) return;
    st->status = t.status;
    st->error = t.error;
    st->n = t.n;
    st->nrhs = t.req.nrhs;
    st->ir_iterations = t.ir;
    st->slot = t.slot;
    st->device_bytes = t.est;
    st->reuse = t.reuse;
    st->reserved = 0;
    const bool admitted = t.status != IGS_REQ_QUEUED;
    const bool finished = t.status == IGS_REQ_DONE || t.status == IGS_REQ_FAILED;
    st->queue_ms = admitted ? ms_between(t.t_submit, t.t_admit) : ms_between(t.t_submit, Clock::now());
    st->run_ms = finished ? ms_between(t.t_admit, t.t_done) : 0.0;
    st->latency_ms = finished ? ms_between(t.t_submit, t.t_done) : 0.0;
}

}  // namespace

extern "C" {

int igs_server_create(int device, const igs_server_opts* opts, igs_server* out) {
    API_BEGIN
    REQUIRE(opts && out, IGS_E_INVALID_ARG, "opts and out must be set");
    REQUIRE(opts->slots >= 1 && opts->slots <= 64, IGS_E_INVALID_ARG, "slots must be in [1, 64]");
    REQUIRE(opts->mem_budget > 0, IGS_E_INVALID_ARG, "mem_budget must be positive");
    REQUIRE(opts->cache_budget >= 0, IGS_E_INVALID_ARG, "cache_budget must not be negative");
    auto s = std::make_unique<igs_server_s>();
    s->device = device;
    s->opts = *opts;
    for (int k = 0; k < opts->slots; ++k) {
        igs_ctx c = nullptr;
        const int rc = igs_create(&c, device, nullptr);
        if (rc != IGS_OK) {
            for (igs_ctx q : s->ctxs) igs_destroy(q);
            throw Error(rc, igs_last_error());
        }
        s->ctxs.push_back(c);
    }
    s->kept.resize(opts->slots);
    igs_server raw = s.release();
    for (int k = 0; k < opts->slots; ++k) raw->workers.emplace_back(worker, raw, k);
    *out = raw;
    API_END
}

int igs_server_submit(igs_server s, const igs_request* r, int64_t* ticket) {
    API_BEGIN
    REQUIRE(s && r && ticket, IGS_E_INVALID_ARG, "server, request and ticket must be set");
    REQUIRE(r->data, IGS_E_INVALID_ARG, "request has no data callback");
    REQUIRE(r->nrhs >= 1 && r->nrhs <= 8, IGS_E_INVALID_ARG, "nrhs must be in [1, 8]");
    REQUIRE(r->knots && r->ctrl_xy && r->n_knots > 0 && r->n_ctrl > 0, IGS_E_INVALID_ARG, "curve arrays missing");
    REQUIRE(r->degree >= 2 && r->degree <= 5 && r->n_ref >= 1 && r->n_ref <= 4 && r->n_elems >= 1, IGS_E_INVALID_ARG,
            "degree, n_ref or n_elems out of range");
    REQUIRE(r->precision == IGS_FP64 || r->precision == IGS_MIXED, IGS_E_INVALID_ARG, "bad precision");
    auto t = std::make_unique<Ticket>();
    t->req = *r;
    t->knots.assign(r->knots, r->knots + r->n_knots);
    t->ctrl.assign(r->ctrl_xy, r->ctrl_xy + 2 * (size_t)r->n_ctrl);
    if (r->weights) t->w.assign(r->weights, r->weights + r->n_ctrl);
    t->req.knots = nullptr;
    t->req.ctrl_xy = nullptr;
    t->req.weights = nullptr;
    t->est = estimate_bytes(*r);
    REQUIRE(t->est <= s->opts.mem_budget, IGS_E_ADMISSION_REFUSED,
            "request needs about " + std::to_string(t->est) + " device bytes, above the server budget");
    t->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        REQUIRE(!s->stop, IGS_E_STATE, "server is shutting down");
        const int64_t id = s->next_id++;
        s->tickets.emplace(id, std::move(t));
        s->queue.push_back(id);
        s->unfinished++;
        *ticket = id;
    }
    s->cv_work.notify_all();
    API_END
}

int igs_server_wait(igs_server s, int64_t ticket, int32_t timeout_ms, igs_request_stats* st) {
    API_BEGIN
    REQUIRE(s, IGS_E_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    REQUIRE(it != s->tickets.end(), IGS_E_INVALID_ARG, "unknown ticket");
    Ticket* t = it->second.get();
    auto done = [&] { return t->status == IGS_REQ_DONE || t->status == IGS_REQ_FAILED; };
    if (timeout_ms < 0) s->cv_done.wait(lk, done);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
        fill_stats(*t, st);
        throw Error(IGS_E_TIMEOUT, "request not finished within the timeout");
    }
    fill_stats(*t, st);
    API_END
}

int igs_server_result(igs_server s, int64_t ticket, double* alpha, double* resid, igs_request_stats* st) {
    API_BEGIN
    REQUIRE(s, IGS_E_INVALID_ARG, "server is NULL");
    std::unique_ptr<Ticket> t;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->tickets.find(ticket);
        REQUIRE(it != s->tickets.end(), IGS_E_INVALID_ARG, "unknown ticket");
        const int status = it->second->status;
        REQUIRE(status == IGS_REQ_DONE || status == IGS_REQ_FAILED, IGS_E_STATE, "request not finished");
        t = std::move(it->second);
        s->tickets.erase(it);
    }
    fill_stats(*t, st);
    if (t->status == IGS_REQ_FAILED) throw Error(t->error, t->msg);
    if (alpha) std::copy(t->alpha.begin(), t->alpha.end(), alpha);
    if (resid) std::copy(t->resid.begin(), t->resid.end(), resid);
    API_END
}

int igs_server_drain(igs_server s, int32_t timeout_ms) {
    API_BEGIN
    REQUIRE(s, IGS_E_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto idle = [&] { return s->unfinished == 0; };
    if (timeout_ms < 0) s->cv_done.wait(lk, idle);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), idle))
        throw Error(IGS_E_TIMEOUT, "requests still running after the timeout");
    API_END
}

int igs_server_destroy(igs_server s) {
    API_BEGIN
    REQUIRE(s, IGS_E_INVALID_ARG, "server is NULL");
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_done.wait(lk, [&] { return s->unfinished == 0; });
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (std::thread& w : s->workers) w.join();
    for (auto& v : s->kept)
        for (Resident& r : v) drop(r);
    for (igs_ctx c : s->ctxs) igs_destroy(c);
    delete s;
    API_END
}

}  // extern "C"
