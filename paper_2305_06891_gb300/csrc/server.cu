// Flux-solve server: continuous batching of rad_solve_flux requests over
// resident compressed operators, admitted against a device-memory budget.
//
// Worker threads (the "slots") each own a CUDA stream and take requests
// from one queue; the requests in flight run concurrently on the device.
// A cavity's operator is built (trees + ACA) on its first request and stays
// resident; idle operators are evicted least recently used first when a new
// one does not fit.  The memory accounting covers resident operators, the
// operator being built (estimated from its facet count until its real size
// is known) with its ACA scratch, and every in-flight request's solver
// workspace.

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <thread>

#include "rad_common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Cavity {
    int64_t n = 0;
    std::vector<double> verts;   // host copy, n x 9
    rad_htree* h = nullptr;      // resident operator (null if not resident)
    int64_t bytes = 0;           // its device bytes
    int in_use = 0;              // requests admitted on it
    bool building = false;
    uint64_t last_use = 0;
};

struct Request {
    int64_t ticket = 0, cav = 0;
    const double* eps = nullptr;
    const double* T = nullptr;
    int64_t ldT = 0, m = 0, ldq = 0;
    double sigma = 0.0;
    double* q = nullptr;
    Clock::time_point t_submit, t_start, t_done;
    bool done = false;
    bool builds = false;         // admitted as the builder of its operator
    int64_t hold = 0;            // bytes reserved while in flight
    rad_request_info info{};
};

}  // namespace

struct rad_server {
    rad_server_params p{};
    rad_allocator alloc{};   // copy of the caller's allocator (p.tree.allocator points here)
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::unique_ptr<Cavity>> cavs;
    std::deque<Request*> queue;
    std::map<int64_t, std::unique_ptr<Request>> reqs;
    int64_t next_ticket = 1;
    bool stopping = false;
    std::vector<std::thread> workers;
    int64_t resident = 0, reserved = 0, peak = 0;
    uint64_t tick = 0;
    int in_flight = 0;
    int64_t submitted = 0, completed = 0, failed = 0, builds = 0, evictions = 0;
    std::vector<double> latencies;
    double service_sum = 0.0;

    // device bytes of a cavity's operator before it is built: dense blocks
    // (~900 entries per facet at leaf 64), low-rank factors (~3,500 entries
    // per facet), the FP32 accurate copy when kept, index lists
    int64_t estimate_operator(int64_t n) const {
        const int ns = rad::dtype_size(p.aca.near_dtype), fs = rad::dtype_size(p.aca.factor_dtype);
        const bool acc = p.aca.accurate_dtype == RAD_F32 && p.aca.factor_dtype == RAD_BF16;
        return n * (900ll * ns + 3500ll * fs + (acc ? 3500ll * 4 : 0) + 2048);
    }
    int64_t aca_scratch() const {
        return p.aca.scratch_mib > 0 ? (int64_t)p.aca.scratch_mib << 20 : (int64_t)2 << 30;
    }
    // solver workspace of one request: Krylov basis and vectors (FP64), the
    // FP32 copy, the product workspace, refinement vectors
    int64_t estimate_solve(int64_t n, int64_t m) const {
        const int64_t nc = m + 1;
        return n * nc * 8 * (p.solve.restart + 8) + n * nc * 4 + n * 64 + (16 << 20);
    }
    int64_t used() const { return resident + reserved; }

    // evict idle operators (LRU) until `need` more bytes fit; false if not
    bool make_room(int64_t need, const Cavity* keep) {
        while (used() + need > p.hbm_budget_bytes) {
            Cavity* victim = nullptr;
            for (auto& c : cavs)
                if (c.get() != keep && c->h && c->in_use == 0 && !c->building &&
                    (!victim || c->last_use < victim->last_use))
                    victim = c.get();
            if (!victim) return false;
            victim->h->sync_on_destroy = false;   // its requests have all returned
            rad_htree_free(victim->h);
            victim->h = nullptr;
            resident -= victim->bytes;
            victim->bytes = 0;
            ++evictions;
        }
        return true;
    }

    // next admissible request (under mu), or null
    Request* pick() {
        for (auto it = queue.begin(); it != queue.end(); ++it) {
            Request* r = *it;
            Cavity& c = *cavs[r->cav];
            if (c.building) continue;   // its operator is being built: wait for it
            const int64_t ws = estimate_solve(c.n, r->m);
            int64_t need = ws;
            if (!c.h) need += estimate_operator(c.n) + aca_scratch();
            if (!make_room(need, &c)) {
                // nothing could ever make room: fail instead of waiting forever
                if (in_flight == 0 && resident == 0 && reserved == 0) {
                    r->info.status = RAD_ELIMIT;
                    r->done = true;
                    ++failed;
                    queue.erase(it);
                    cv_done.notify_all();
                    return pick();
                }
                continue;
            }
            r->builds = !c.h;
            if (r->builds) c.building = true;
            ++c.in_use;
            r->hold = need;
            reserved += need;
            peak = std::max(peak, used());
            queue.erase(it);
            return r;
        }
        return nullptr;
    }

    void run(int slot) {
        cudaSetDevice(device);
        cudaStream_t st = nullptr;
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            Request* r = pick();
            if (!r) {
                if (stopping && queue.empty()) break;
                cv_work.wait(lk);
                continue;
            }
            ++in_flight;
            Cavity& c = *cavs[r->cav];
            r->t_start = Clock::now();
            r->info.slot = slot;
            lk.unlock();
            int rc = RAD_OK;
            rad_htree* h = c.h;
            if (r->builds) {
                h = nullptr;
                rc = rad_build_htree(c.n, c.verts.data(), &p.tree, st, &h);
                if (rc == RAD_OK) rc = rad_compress_aca(h, &p.aca, st);
                // resident operators keep the CUDA-core tiles for many-field
                // requests: the tensor-core images (about 1.5 times the
                // operator) would grow a handle past the bytes its admission
                // counted
                if (rc == RAD_OK) rc = rad_htree_set_product_path(h, 0);
            }
            int64_t op_bytes = 0;
            if (r->builds && rc == RAD_OK) {
                rad_htree_stats hs{};
                rad_htree_get_stats(h, &hs);
                op_bytes = hs.bytes_near + hs.bytes_far + hs.bytes_accurate + (int64_t)c.n * 64;
            } else if (r->builds && h) {
                h->sync_on_destroy = false;
                rad_htree_free(h);
                h = nullptr;
            }
            if (r->builds) {
                lk.lock();
                c.building = false;
                const int64_t est = estimate_operator(c.n) + aca_scratch();
                reserved -= est;
                r->hold -= est;
                if (rc == RAD_OK) {
                    c.h = h;
                    c.bytes = op_bytes;
                    resident += op_bytes;
                    peak = std::max(peak, used());
                    ++builds;
                }
                cv_work.notify_all();   // requests waiting on this cavity may go
                lk.unlock();
            }
            rad_solve_info si{};
            if (rc == RAD_OK)
                rc = rad_solve_flux(h, r->eps, r->T, r->ldT, r->m, r->sigma, &p.solve, r->q, r->ldq, &si, st);
            const Clock::time_point t_done = Clock::now();
            lk.lock();
            --in_flight;
            --c.in_use;
            c.last_use = ++tick;
            reserved -= r->hold;
            r->t_done = t_done;
            r->info.status = rc;
            r->info.built = r->builds ? 1 : 0;
            r->info.iters = si.iters;
            r->info.refinements = si.refinements;
            r->info.max_rel_residual = si.max_rel_residual;
            r->info.queue_ms = ms_between(r->t_submit, r->t_start);
            r->info.service_ms = ms_between(r->t_start, t_done);
            r->info.latency_ms = ms_between(r->t_submit, t_done);
            r->done = true;
            if (rc == RAD_OK || rc == RAD_ENOTCONV) {
                ++completed;
                latencies.push_back(r->info.latency_ms);
                service_sum += r->info.service_ms;
            } else {
                ++failed;
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
        lk.unlock();
        cudaStreamDestroy(st);
    }
};

using namespace rad;

extern "C" {

int rad_server_create(const rad_server_params* p, rad_server** out) {
    NvtxRange nv_(__func__);
    try {
        RAD_REQUIRE(p != nullptr && out != nullptr, RAD_EINVAL, "null argument");
        *out = nullptr;
        RAD_REQUIRE(p->slots >= 1 && p->slots <= 64, RAD_EINVAL, "slots must be in [1, 64]");
        RAD_REQUIRE(p->hbm_budget_bytes > 0, RAD_EINVAL, "hbm_budget_bytes must be > 0");
        RAD_REQUIRE(p->tree.leaf_size >= 1 && p->tree.eta_adm > 0.0, RAD_EINVAL, "bad tree parameters");
        RAD_REQUIRE(p->solve.restart >= 1 && p->solve.restart <= 64 && p->solve.tol > 0.0, RAD_EINVAL,
                    "bad solve parameters");
        RAD_REQUIRE(!p->solve.refine || (p->aca.accurate_dtype == RAD_F32 || p->aca.factor_dtype == RAD_F64),
                    RAD_EINVAL, "refinement needs aca.accurate_dtype = RAD_F32 (or the FP64 path)");
        RAD_REQUIRE(!p->tree.allocator || (p->tree.allocator->alloc && p->tree.allocator->free), RAD_EINVAL,
                    "an allocator needs both alloc and free");
        auto s = std::make_unique<rad_server>();
        s->p = *p;
        if (p->tree.allocator) {
            s->alloc = *p->tree.allocator;
            s->p.tree.allocator = &s->alloc;
        }
        RAD_CUDA(cudaGetDevice(&s->device));
        rad_server* raw = s.get();
        for (int k = 0; k < p->slots; ++k) s->workers.emplace_back([raw, k] { raw->run(k); });
        *out = s.release();
        return RAD_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.code;
    } catch (...) {
        set_last_error("server creation failed");
        return RAD_ECUDA;
    }
}

int rad_server_add_cavity(rad_server* s, int64_t n, const double* verts, int64_t* cavity_id) {
    NvtxRange nv_(__func__);
    try {
        RAD_REQUIRE(s && verts && cavity_id, RAD_EINVAL, "null argument");
        RAD_REQUIRE(n >= 1 && n < (int64_t)1 << 28, RAD_EINVAL, "n must be in [1, 2^28)");
        auto c = std::make_unique<Cavity>();
        c->n = n;
        c->verts.resize(9 * (size_t)n);
        if (is_device_ptr(verts)) {
            RAD_CUDA(cudaMemcpy(c->verts.data(), verts, sizeof(double) * 9 * (size_t)n, cudaMemcpyDeviceToHost));
        } else {
            std::memcpy(c->verts.data(), verts, sizeof(double) * 9 * (size_t)n);
        }
        std::lock_guard<std::mutex> lk(s->mu);
        *cavity_id = (int64_t)s->cavs.size();
        s->cavs.push_back(std::move(c));
        return RAD_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.code;
    } catch (...) {
        set_last_error("add_cavity failed");
        return RAD_ECUDA;
    }
}

int rad_server_submit(rad_server* s, int64_t cavity_id, const double* eps, const double* T, int64_t ldT, int64_t m,
                      double sigma, double* q, int64_t ldq, int64_t* ticket) {
    NvtxRange nv_(__func__);
    try {
        RAD_REQUIRE(s && eps && T && q && ticket, RAD_EINVAL, "null argument");
        std::lock_guard<std::mutex> lk(s->mu);
        RAD_REQUIRE(!s->stopping, RAD_EINVAL, "server is shutting down");
        RAD_REQUIRE(cavity_id >= 0 && cavity_id < (int64_t)s->cavs.size(), RAD_EINVAL, "unknown cavity id");
        const int64_t n = s->cavs[cavity_id]->n;
        RAD_REQUIRE(m >= 1 && m <= 1024, RAD_EINVAL, "m must be in [1, 1024]");
        RAD_REQUIRE(ldT >= n && ldq >= n, RAD_EINVAL, "leading dimension smaller than n");
        auto r = std::make_unique<Request>();
        r->ticket = s->next_ticket++;
        r->cav = cavity_id;
        r->eps = eps;
        r->T = T;
        r->ldT = ldT;
        r->m = m;
        r->sigma = sigma;
        r->q = q;
        r->ldq = ldq;
        r->t_submit = Clock::now();
        *ticket = r->ticket;
        s->queue.push_back(r.get());
        s->reqs[r->ticket] = std::move(r);
        ++s->submitted;
        s->cv_work.notify_one();
        return RAD_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.code;
    }
}

int rad_server_wait(rad_server* s, int64_t ticket, rad_request_info* info) {
    NvtxRange nv_(__func__);
    if (!s) {
        set_last_error("null argument");
        return RAD_EINVAL;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        set_last_error("unknown or already collected ticket");
        return RAD_EINVAL;
    }
    Request* r = it->second.get();
    s->cv_done.wait(lk, [r] { return r->done; });
    if (info) *info = r->info;
    const int rc = r->info.status;
    s->reqs.erase(it);
    if (rc != RAD_OK && rc != RAD_ENOTCONV) set_last_error("request failed (see rad_request_info.status)");
    return rc;
}

int rad_server_get_stats(rad_server* s, rad_server_stats* st) {
    if (!s || !st) {
        set_last_error("null argument");
        return RAD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    *st = rad_server_stats{};
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->failed = s->failed;
    st->builds = s->builds;
    st->evictions = s->evictions;
    st->resident_bytes = s->resident;
    st->peak_bytes = s->peak;
    st->in_flight = s->in_flight;
    for (auto& c : s->cavs) st->resident_cavities += c->h ? 1 : 0;
    if (!s->latencies.empty()) {
        std::vector<double> v = s->latencies;
        std::sort(v.begin(), v.end());
        auto pct = [&](double f) {
            // nearest-rank percentile
            const size_t k = (size_t)std::ceil(f * (double)v.size());
            return v[std::min(v.size() - 1, k > 0 ? k - 1 : 0)];
        };
        st->p50_latency_ms = pct(0.50);
        st->p99_latency_ms = pct(0.99);
        st->max_latency_ms = v.back();
        st->mean_service_ms = s->service_sum / (double)v.size();
    }
    return RAD_OK;
}

int rad_server_destroy(rad_server* s) {
    NvtxRange nv_(__func__);
    if (!s) return RAD_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto& c : s->cavs)
        if (c->h) rad_htree_free(c->h);
    delete s;
    return RAD_OK;
}

}  // extern "C"
