// C ABI entry points of librad (declared in include/rad.h).  Every entry
// point catches all C++ exceptions and turns them into status codes.

#include <algorithm>
#include <atomic>
#include <chrono>
#include <exception>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>

#include "rad_common.cuh"

namespace rad {

namespace {
thread_local std::string g_last_error;
}

void fail(int code, const std::string& msg) { throw Error{code, msg}; }
void set_last_error(const std::string& msg) { g_last_error = msg; }

// ------------------------------------------------------------ launch accounting
namespace {
std::atomic<long long> g_launches{0};
struct ProfRec {
    const char* name;
    cudaEvent_t a, b;    // null for a host phase
    double host_ms;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;
}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(); }

bool profiling_enabled() {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    return g_prof_on;
}

ProfScope::ProfScope(const char* name, cudaStream_t st) : s(st) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on) return;
    ProfRec r{name, nullptr, nullptr, 0.0};
    if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    cudaEventRecord(r.a, s);
    idx = (int)g_prof.size();
    g_prof.push_back(r);
}
ProfScope::~ProfScope() {
    if (idx < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (idx < (int)g_prof.size()) cudaEventRecord(g_prof[idx].b, s);
}

HostScope::HostScope(const char* n) : name(n), t0(std::chrono::steady_clock::now()) {}
HostScope::~HostScope() {
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (g_prof_on) g_prof.push_back(ProfRec{name, nullptr, nullptr, ms});
}

// ------------------------------------------------------------ staging
namespace {
struct StageState {
    int depth = 0;
    char* cur = nullptr;
    size_t cap = 0, off = 0;
    std::vector<char*> retired;   // outgrown blocks, freed when the scope ends
};
thread_local StageState g_stage;
}  // namespace

StageScope::StageScope() { ++g_stage.depth; }
StageScope::~StageScope() {
    if (--g_stage.depth > 0) return;
    // unwinding from an error: copies may still be in flight
    if (std::uncaught_exceptions() > 0) (void)cudaDeviceSynchronize();
    for (char* p : g_stage.retired) cudaFreeHost(p);
    g_stage.retired.clear();
    g_stage.off = 0;
}
// Host worker pool: kPoolThreads threads started on first use and kept for
// the life of the process.  One job at a time (try_lock on job_mu).  Parts
// are handed out under the pool mutex together with a check of the job's
// epoch, so a worker that wakes late never touches a finished job; the
// caller runs parts as well and returns once every part has finished.
namespace {
constexpr int kPoolThreads = 15;
struct HostPool {
    std::mutex job_mu;                     // held by the caller for one job
    std::mutex mu;                         // guards everything below
    std::condition_variable cv, done_cv;
    void (*job)(void*, int) = nullptr;
    void* ctx = nullptr;
    int parts = 0, next_part = 0, remaining = 0;
    unsigned long long epoch = 0;
    bool stop = false;
    std::vector<std::thread> th;
    void drain(unsigned long long ep) {
        for (;;) {
            int q;
            void (*j)(void*, int);
            void* c;
            {
                std::lock_guard<std::mutex> lk(mu);
                if (epoch != ep || next_part >= parts) return;
                q = next_part++;
                j = job;
                c = ctx;
            }
            j(c, q);
            std::lock_guard<std::mutex> lk(mu);
            if (--remaining == 0) done_cv.notify_all();
        }
    }
    void worker() {
        unsigned long long seen = 0;
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] { return stop || epoch != seen; });
                if (stop) return;
                seen = epoch;
            }
            drain(seen);
        }
    }
    HostPool() {
        for (int i = 0; i < kPoolThreads; ++i) th.emplace_back([this] { worker(); });
    }
    ~HostPool() {
        {
            std::lock_guard<std::mutex> lk(mu);
            stop = true;
        }
        cv.notify_all();
        for (auto& t : th) t.join();
    }
};
HostPool& host_pool() {
    static HostPool p;
    return p;
}
}  // namespace

bool pool_run(int parts, void (*job)(void*, int), void* ctx) {
    HostPool& p = host_pool();
    std::unique_lock<std::mutex> busy(p.job_mu, std::try_to_lock);
    if (!busy.owns_lock()) return false;
    unsigned long long ep;
    {
        std::lock_guard<std::mutex> lk(p.mu);
        p.job = job;
        p.ctx = ctx;
        p.parts = parts;
        p.next_part = 0;
        p.remaining = parts;
        ep = ++p.epoch;
    }
    p.cv.notify_all();
    p.drain(ep);
    std::unique_lock<std::mutex> lk(p.mu);
    p.done_cv.wait(lk, [&] { return p.remaining == 0; });
    return true;
}

void stage_copy(void* dst, const void* src, size_t bytes) {
    constexpr size_t kPar = 8u << 20;
    if (bytes < kPar) {
        std::memcpy(dst, src, bytes);
        return;
    }
    constexpr int P = 8;
    parallel_parts(P, [&](int q) {
        const size_t b0 = bytes * q / P, b1 = bytes * (q + 1) / P;
        std::memcpy(static_cast<char*>(dst) + b0, static_cast<const char*>(src) + b0, b1 - b0);
    });
}

void* stage_alloc(size_t bytes) {
    StageState& st = g_stage;
    if (st.depth == 0) return nullptr;
    const size_t need = (bytes + 255) / 256 * 256;
    if (st.off + need > st.cap) {
        const size_t cap = std::max<size_t>({need, 2 * st.cap, 16u << 20});
        char* p = nullptr;
        if (cudaMallocHost(&p, cap) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;   // fall back to a pageable copy
        }
        if (st.cur) st.retired.push_back(st.cur);
        st.cur = p;
        st.cap = cap;
        st.off = 0;
    }
    void* r = st.cur + st.off;
    st.off += need;
    return r;
}

static void clear_profile() {
    for (auto& r : g_prof) {
        if (r.a) cudaEventDestroy(r.a);
        if (r.b) cudaEventDestroy(r.b);
    }
    g_prof.clear();
}

// The library's own memory pool of a device (created on first use): a
// stream-ordered pool whose release threshold is raised so that freed memory
// stays cached and repeated builds do not map new pages.  It is separate from
// the device's default pool, whose settings belong to the caller's process.
static cudaMemPool_t library_pool() {
    static std::mutex mu;
    static std::vector<std::pair<int, cudaMemPool_t>> pools;
    int dev = 0;
    RAD_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    for (auto& e : pools)
        if (e.first == dev) return e.second;
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    RAD_CUDA(cudaMemPoolCreate(&pool, &props));
    uint64_t thr = UINT64_MAX;
    RAD_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    pools.push_back({dev, pool});
    return pool;
}

namespace {
thread_local Allocator g_cur_alloc;   // default: the library's pool
}
const Allocator& current_allocator() { return g_cur_alloc; }
AllocScope::AllocScope(const Allocator& a) : prev(g_cur_alloc) { g_cur_alloc = a; }
AllocScope::~AllocScope() { g_cur_alloc = prev; }

static void* raw_get(const rad_allocator& cb, size_t bytes, cudaStream_t s) {
    void* p = nullptr;
    if (cb.alloc) {
        p = cb.alloc(cb.ctx, (uint64_t)bytes, s);
        if (!p) fail(RAD_ENOMEM, "the caller's allocator returned NULL for " + std::to_string(bytes) + " bytes");
        return p;
    }
    RAD_CUDA(cudaMallocFromPoolAsync(&p, bytes, library_pool(), s));
    return p;
}
static void raw_put(const rad_allocator& cb, void* p, size_t bytes, cudaStream_t s) {
    if (cb.alloc) {
        if (cb.free) cb.free(cb.ctx, p, (uint64_t)bytes, s);
        return;
    }
    if (cudaFreeAsync(p, s) != cudaSuccess) (void)cudaGetLastError();
}

#ifdef RAD_CHECK_BOUNDS
// Bounds-checked build: every device allocation carries kGuard canary bytes
// (value kCanary) before and after the bytes handed out.  The guards are
// verified when the memory is returned and after every C-ABI call; a
// changed canary byte means a kernel wrote outside its buffer, and the call
// returns RAD_ECUDA naming the allocation.
namespace {
constexpr size_t kGuard = 256;
constexpr unsigned char kCanary = 0xA5;
std::mutex g_guard_mu;
std::map<void*, size_t> g_guarded;   // handed-out pointer -> bytes
std::string g_guard_error;
bool guards_intact(void* user, size_t bytes) {
    unsigned char g[2 * kGuard];
    unsigned char* base = static_cast<unsigned char*>(user) - kGuard;
    if (cudaMemcpy(g, base, kGuard, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(g + kGuard, static_cast<unsigned char*>(user) + bytes, kGuard, cudaMemcpyDeviceToHost) !=
            cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    for (unsigned char c : g)
        if (c != kCanary) return false;
    return true;
}
}  // namespace
#endif

void* Allocator::get(size_t bytes, cudaStream_t s) const {
    if (bytes == 0) bytes = 16;
#ifdef RAD_CHECK_BOUNDS
    const size_t total = (bytes + 255) / 256 * 256 + 2 * kGuard;
    unsigned char* base = static_cast<unsigned char*>(raw_get(cb, total, s));
    RAD_CUDA(cudaMemsetAsync(base, kCanary, kGuard, s));
    RAD_CUDA(cudaMemsetAsync(base + kGuard + bytes, kCanary, total - kGuard - bytes, s));
    RAD_CUDA(cudaStreamSynchronize(s));   // canaries in place before anyone checks them
    {
        std::lock_guard<std::mutex> lk(g_guard_mu);
        g_guarded[base + kGuard] = bytes;
    }
    return base + kGuard;
#else
    return raw_get(cb, bytes, s);
#endif
}
void Allocator::put(void* p, size_t bytes, cudaStream_t s) const {
    if (!p) return;
    if (bytes == 0) bytes = 16;
#ifdef RAD_CHECK_BOUNDS
    (void)cudaStreamSynchronize(s);
    {
        std::lock_guard<std::mutex> lk(g_guard_mu);
        if (!guards_intact(p, bytes) && g_guard_error.empty())
            g_guard_error = "bounds check: canary overwritten around a device allocation of " +
                            std::to_string(bytes) + " bytes";
        g_guarded.erase(p);
    }
    raw_put(cb, static_cast<unsigned char*>(p) - kGuard, (bytes + 255) / 256 * 256 + 2 * kGuard, s);
#else
    raw_put(cb, p, bytes, s);
#endif
}

// After a C-ABI call: in the bounds-checked build, waits for the device and
// verifies every live allocation's canaries; fails with RAD_ECUDA if one was
// overwritten (during this call or when memory was returned).  A no-op in
// the ordinary build.
void check_bounds_after_call() {
#ifdef RAD_CHECK_BOUNDS
    (void)cudaDeviceSynchronize();
    std::string err;
    {
        // under the lock: no allocation is returned (and reused) while its
        // canaries are read
        std::lock_guard<std::mutex> lk(g_guard_mu);
        for (auto& e : g_guarded)
            if (!guards_intact(e.first, e.second) && g_guard_error.empty())
                g_guard_error = "bounds check: canary overwritten around a device allocation of " +
                                std::to_string(e.second) + " bytes";
        err.swap(g_guard_error);
    }
    if (!err.empty()) fail(RAD_ECUDA, err);
#endif
}

void DevBuf::alloc(size_t b, cudaStream_t s) {
    release(s);
    if (b == 0) return;
    al = current_allocator();
    p = al.get(b, s);
    bytes = b;
}
void DevBuf::release(cudaStream_t s) {
    if (p) al.put(p, bytes, s);
    p = nullptr;
    bytes = 0;
}

Scratch::~Scratch() {
    for (auto& q : ptrs) al.put(q.first, q.second, s);
}
void* Scratch::get(size_t bytes) {
    ptrs.reserve(ptrs.size() + 1);
    void* q = al.get(bytes ? bytes : 16, s);
    ptrs.push_back({q, bytes ? bytes : 16});
    return q;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

const void* to_device(const void* p, size_t bytes, Scratch& ws) {
    if (is_device_ptr(p)) return p;
    void* d = ws.get(bytes);
    RAD_CUDA(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, ws.s));
    return d;
}

// column-major (rows x cols, leading dim ld) host or device array -> compact
// device copy with leading dim rows
static const void* stage_in_2d(const void* p, int64_t rows, int64_t cols, int64_t ld, size_t esz, Scratch& ws) {
    if (is_device_ptr(p)) return p;
    void* d = ws.get(esz * rows * cols);
    RAD_CUDA(cudaMemcpy2DAsync(d, esz * rows, p, esz * ld, esz * rows, cols, cudaMemcpyHostToDevice, ws.s));
    return d;
}

template <class F>
static int guarded(const char* name, F&& f) {
    NvtxRange nv_(name);
    try {
        f();
        check_bounds_after_call();
        return RAD_OK;
    } catch (const Error& e) {
        g_last_error = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        g_last_error = "host allocation failed";
        return RAD_ENOMEM;
    } catch (const std::exception& e) {
        g_last_error = e.what();
        return RAD_ECUDA;
    } catch (...) {
        g_last_error = "unknown error";
        return RAD_ECUDA;
    }
}

static void check_tree_params(int64_t n, const rad_tree_params* p) {
    RAD_REQUIRE(p != nullptr, RAD_EINVAL, "null tree params");
    RAD_REQUIRE(n >= 1 && n < (int64_t)(INT_MAX / 8), RAD_EINVAL, "n must be in [1, 2^28)");
    RAD_REQUIRE(p->leaf_size >= 1, RAD_EINVAL, "leaf_size must be >= 1");
    RAD_REQUIRE(std::isfinite(p->eta_adm) && p->eta_adm > 0.0, RAD_EINVAL, "eta_adm must be > 0");
    RAD_REQUIRE(!p->allocator || (p->allocator->alloc && p->allocator->free), RAD_EINVAL,
                "an allocator needs both alloc and free");
}

// The allocator a new handle keeps (the caller's callbacks, or the pool).
static Allocator handle_allocator(const rad_tree_params* p) {
    Allocator a;
    if (p->allocator) a.cb = *p->allocator;
    return a;
}

}  // namespace rad

using namespace rad;

namespace rad {

void drop_product_graph(const rad_htree* h) {
    if (!h->graph) return;
    if (h->graph->exec) RAD_CUDA(cudaStreamSynchronize(h->graph->stream));
    h->graph.reset();
}

// The graph path of rad_hmatvec (device arrays only).  Returns false when the
// call must take the ordinary path.
static bool product_via_graph(const rad_htree* h, int32_t dtype, const void* x, int64_t ldx, void* y, int64_t ldy,
                              int64_t nrhs, cudaStream_t s) {
    if (profiling_enabled()) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    RAD_CUDA(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return false;   // the caller is capturing: plain launches
    if (!h->graph) h->graph = std::make_unique<ProductGraph>();
    ProductGraph& g = *h->graph;
    std::lock_guard<std::mutex> lk(g.mu);
    const bool same = g.x == x && g.y == y && g.ldx == ldx && g.ldy == ldy && g.nrhs == nrhs && g.dtype == dtype &&
                      g.stream == s;
    if (same && g.exec) {
        RAD_CUDA(cudaGraphLaunch(g.exec, s));
        note_launches(g.kernels);
        return true;
    }
    if (!same) {
        if (g.exec) {
            RAD_CUDA(cudaStreamSynchronize(g.stream));
            RAD_CUDA(cudaGraphExecDestroy(g.exec));
            g.exec = nullptr;
        }
        g.x = x;
        g.y = y;
        g.ldx = ldx;
        g.ldy = ldy;
        g.nrhs = nrhs;
        g.dtype = dtype;
        g.stream = s;
        g.hits = 1;
        return false;
    }
    // second identical call: capture gather + product + scatter once
    const int n = (int)h->n;
    const int nr = (int)nrhs;
    const bool op64 = h->op_is_f64();
    const size_t osz = op64 ? 8 : 4;
    const int ldp = nr == 1 ? 1 : (nr + 3) / 4 * 4;
    g.X.alloc(osz * n * ldp, s);
    g.Y.alloc(osz * n * nr, s);
    g.T.alloc(apply_workspace_bytes(h, nr), s);
    if (!g.capture) RAD_CUDA(cudaStreamCreateWithFlags(&g.capture, cudaStreamNonBlocking));
    const long long k0 = launch_count();
    RAD_CUDA(cudaStreamBeginCapture(g.capture, cudaStreamCaptureModeThreadLocal));
    cudaGraph_t graph = nullptr;
    try {
        gather_user_to_tree(h, dtype, x, ldx, nr, g.X.p, ldp, op64, g.capture);
        apply_tree(h, g.X.p, ldp, g.Y.p, nr, nr, Epi{kStore, nullptr, nullptr, nullptr, 0}, g.T.p, g.capture);
        scatter_tree_to_user(h, g.Y.p, nr, nr, op64, dtype, y, ldy, g.capture);
    } catch (...) {
        cudaStreamEndCapture(g.capture, &graph);
        if (graph) cudaGraphDestroy(graph);
        (void)cudaGetLastError();
        throw;
    }
    RAD_CUDA(cudaStreamEndCapture(g.capture, &graph));
    g.kernels = launch_count() - k0;
    const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    RAD_CUDA(ie);
    RAD_CUDA(cudaGraphLaunch(g.exec, s));
    return true;
}

}  // namespace rad

extern "C" {

int rad_version(void) { return 10200; }

int rad_debug_bounds_checks(void) {
#ifdef RAD_CHECK_BOUNDS
    return 1;
#else
    return 0;
#endif
}

int64_t rad_launch_count(void) { return g_launches.load(); }

int rad_profile_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    clear_profile();
    g_prof_on = on != 0;
    return RAD_OK;
}

int rad_profile_read(int32_t max_kernels, char* names, int64_t* counts, double* total_ms) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::map<std::string, std::pair<int64_t, double>> agg;
    for (auto& r : g_prof) {
        float ms = (float)r.host_ms;
        if (r.a && (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)) {
            (void)cudaGetLastError();
            continue;
        }
        auto& e = agg[r.name];
        e.first += 1;
        e.second += ms;
    }
    int k = 0;
    for (auto& kv : agg) {
        if (k >= max_kernels) break;
        if (names) {
            std::strncpy(names + 48 * k, kv.first.c_str(), 47);
            names[48 * k + 47] = 0;
        }
        if (counts) counts[k] = kv.second.first;
        if (total_ms) total_ms[k] = kv.second.second;
        ++k;
    }
    return (int)agg.size();
}

const char* rad_last_error(void) { return g_last_error.c_str(); }

int rad_build_htree(int64_t n, const double* verts, const rad_tree_params* p, void* stream, rad_htree** out) {
    return guarded(__func__, [&] {
        RAD_REQUIRE(out != nullptr && verts != nullptr, RAD_EINVAL, "null argument");
        *out = nullptr;
        check_tree_params(n, p);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        auto h = std::make_unique<rad_htree>();
        h->n = n;
        h->leaf_size = p->leaf_size;
        h->eta = p->eta_adm;
        h->alloc = handle_allocator(p);
        AllocScope as(h->alloc);
        RAD_CUDA(cudaGetDevice(&h->device));
        Scratch ws(s);
        const double* v = to_device_t(verts, 9 * (size_t)n, ws);
        double* geo_user = ws.get_n<double>(7 * (size_t)n);
        build_geometry_from_tris(h.get(), v, geo_user, s);
        build_trees(h.get(), geo_user, s);
        RAD_CUDA(cudaStreamSynchronize(s));
        *out = h.release();
    });
}

int rad_build_htree_batch(int32_t n_cavities, const int64_t* counts, const double* verts, const rad_tree_params* p,
                          void* stream, rad_htree** out) {
    return guarded(__func__, [&] {
        RAD_REQUIRE(out != nullptr && verts != nullptr && counts != nullptr, RAD_EINVAL, "null argument");
        *out = nullptr;
        RAD_REQUIRE(n_cavities >= 1, RAD_EINVAL, "n_cavities must be >= 1");
        std::vector<int64_t> seg(n_cavities + 1, 0);
        for (int c = 0; c < n_cavities; ++c) {
            RAD_REQUIRE(counts[c] >= 1, RAD_EINVAL, "every cavity needs at least one triangle");
            seg[c + 1] = seg[c] + counts[c];
        }
        const int64_t n = seg[n_cavities];
        check_tree_params(n, p);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        auto h = std::make_unique<rad_htree>();
        h->n = n;
        h->seg = seg;
        h->leaf_size = p->leaf_size;
        h->eta = p->eta_adm;
        h->alloc = handle_allocator(p);
        AllocScope as(h->alloc);
        RAD_CUDA(cudaGetDevice(&h->device));
        Scratch ws(s);
        const double* v = to_device_t(verts, 9 * (size_t)n, ws);
        double* geo_user = ws.get_n<double>(7 * (size_t)n);
        build_geometry_from_tris(h.get(), v, geo_user, s);
        build_trees(h.get(), geo_user, s);
        if (n_cavities > 1) {
            std::vector<int> segrow(n);
            for (int c = 0; c < n_cavities; ++c)
                for (int64_t i = seg[c]; i < seg[c + 1]; ++i) segrow[i] = c;
            h->d_segrow.alloc(sizeof(int) * (size_t)n, s);
            RAD_CUDA(cudaMemcpyAsync(h->d_segrow.p, segrow.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, s));
        }
        RAD_CUDA(cudaStreamSynchronize(s));
        *out = h.release();
    });
}

int rad_build_htree_facets(int64_t n, const double* centroid, const double* normal, const double* area,
                           const rad_tree_params* p, void* stream, rad_htree** out) {
    return guarded(__func__, [&] {
        RAD_REQUIRE(out != nullptr && centroid && normal && area, RAD_EINVAL, "null argument");
        *out = nullptr;
        check_tree_params(n, p);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        auto h = std::make_unique<rad_htree>();
        h->n = n;
        h->leaf_size = p->leaf_size;
        h->eta = p->eta_adm;
        h->alloc = handle_allocator(p);
        AllocScope as(h->alloc);
        RAD_CUDA(cudaGetDevice(&h->device));
        Scratch ws(s);
        const double* c = to_device_t(centroid, 3 * (size_t)n, ws);
        const double* nr = to_device_t(normal, 3 * (size_t)n, ws);
        const double* a = to_device_t(area, (size_t)n, ws);
        double* geo_user = ws.get_n<double>(7 * (size_t)n);
        build_geometry_from_facets(h.get(), c, nr, a, geo_user, s);
        build_trees(h.get(), geo_user, s);
        RAD_CUDA(cudaStreamSynchronize(s));
        *out = h.release();
    });
}

int rad_htree_from_dense(int64_t n, const double* F, void* stream, rad_htree** out) {
    return guarded(__func__, [&] {
        RAD_REQUIRE(out != nullptr && F != nullptr, RAD_EINVAL, "null argument");
        *out = nullptr;
        RAD_REQUIRE(n >= 1 && n <= 46340, RAD_EINVAL, "n must be in [1, 46340]");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        auto h = std::make_unique<rad_htree>();
        h->n = n;
        h->leaf_size = (int)n;
        h->eta = 1.0;
        h->from_dense = true;
        RAD_CUDA(cudaGetDevice(&h->device));
        h->nodes.assign(1, NodeShape{0, (int)n, 0, -1, -1, 1});
        h->boxes.assign(1, NodeBox{{0, 0, 0}, {0, 0, 0}});
        h->depth = 1;
        h->perm_h.resize(n);
        for (int i = 0; i < (int)n; ++i) h->perm_h[i] = i;
        h->perm.alloc(sizeof(int) * n, s);
        h->iperm.alloc(sizeof(int) * n, s);
        h2d(h->perm.as<int>(), h->perm_h, s);
        h2d(h->iperm.as<int>(), h->perm_h, s);
        Scratch ws(s);
        const double* Fd = to_device_t(F, (size_t)n * n, ws);
        load_dense_operator(h.get(), Fd, s);
        *out = h.release();
    });
}

int rad_compress_aca(rad_htree* h, const rad_aca_params* p, void* stream) {
    return guarded(__func__, [&] {
        RAD_REQUIRE(h != nullptr, RAD_EINVAL, "null handle");
        AllocScope as(h->alloc);
        compress(h, p, static_cast<cudaStream_t>(stream));
    });
}


int rad_hmatvec(const rad_htree* h, int32_t dtype, const void* x, int64_t ldx, void* y, int64_t ldy, int64_t nrhs,
                void* stream) {
    return guarded(__func__, [&] {
        RAD_REQUIRE(h != nullptr && x != nullptr && y != nullptr, RAD_EINVAL, "null argument");
        AllocScope as(h->alloc);
        RAD_REQUIRE(h->compressed, RAD_EINVAL, "handle is not compressed (call rad_compress_aca)");
        RAD_REQUIRE(dtype == RAD_F64 || dtype == RAD_F32, RAD_EINVAL, "dtype must be RAD_F64 or RAD_F32");
        RAD_REQUIRE(nrhs >= 1 && nrhs <= 4096, RAD_EINVAL, "nrhs must be in [1, 4096]");
        RAD_REQUIRE(ldx >= h->n && ldy >= h->n, RAD_EINVAL, "leading dimension smaller than n");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        tc_prepare(h, (int)nrhs, s);
        if (is_device_ptr(x) && is_device_ptr(y) && product_via_graph(h, dtype, x, ldx, y, ldy, nrhs, s)) return;
        const int n = (int)h->n;
        const int nr = (int)nrhs;
        const size_t esz = dtype == RAD_F64 ? 8 : 4;
        const bool op64 = h->op_is_f64();
        const size_t osz = op64 ? 8 : 4;
        Scratch ws(s);
        const void* xd = stage_in_2d(x, n, nr, ldx, esz, ws);
        const int64_t ldxd = is_device_ptr(x) ? ldx : n;
        const int ldp = nr == 1 ? 1 : (nr + 3) / 4 * 4;   // padded rows: 16-byte quads in the product
        void* X = ws.get(osz * n * ldp);
        void* Y = ws.get(osz * n * nr);
        void* T = ws.get(apply_workspace_bytes(h, nr));
        gather_user_to_tree(h, dtype, xd, ldxd, nr, X, ldp, op64, s);
        apply_tree(h, X, ldp, Y, nr, nr, Epi{kStore, nullptr, nullptr, nullptr, 0}, T, s);
        if (is_device_ptr(y)) {
            scatter_tree_to_user(h, Y, nr, nr, op64, dtype, y, ldy, s);
        } else {
            void* yd = ws.get(esz * n * nr);
            scatter_tree_to_user(h, Y, nr, nr, op64, dtype, yd, n, s);
            RAD_CUDA(cudaMemcpy2DAsync(y, esz * ldy, yd, esz * n, esz * n, nr, cudaMemcpyDeviceToHost, s));
            RAD_CUDA(cudaStreamSynchronize(s));
            RAD_REQUIRE(!wait_timed_out(), RAD_ECUDA, "a pipelined kernel's wait timed out (results are incomplete)");
        }
    });
}

int rad_solve_flux(const rad_htree* h, const double* eps, const double* T, int64_t ldT, int64_t m, double sigma,
                   const rad_solve_params* p, double* q, int64_t ldq, rad_solve_info* info, void* stream) {
    int solve_status = RAD_OK;
    const int rc = guarded(__func__, [&] {
        RAD_REQUIRE(h != nullptr && eps && T && q && p, RAD_EINVAL, "null argument");
        AllocScope as(h->alloc);
        RAD_REQUIRE(h->compressed, RAD_EINVAL, "handle is not compressed (call rad_compress_aca)");
        RAD_REQUIRE(m >= 1 && m <= 1024, RAD_EINVAL, "m must be in [1, 1024]");
        RAD_REQUIRE(ldT >= h->n && ldq >= h->n, RAD_EINVAL, "leading dimension smaller than n");
        RAD_REQUIRE(p->restart >= 1 && p->restart <= 64, RAD_EINVAL, "restart must be in [1, 64]");
        RAD_REQUIRE(p->max_iter >= 1, RAD_EINVAL, "max_iter must be >= 1");
        RAD_REQUIRE(!p->precond || hlu_handle(p->precond) == h, RAD_EINVAL,
                    "the preconditioner's factors belong to another handle");
        RAD_REQUIRE(p->tol > 0.0 && std::isfinite(p->tol), RAD_EINVAL, "tol must be > 0");
        RAD_REQUIRE(std::isfinite(sigma), RAD_EINVAL, "sigma must be finite");
        RAD_REQUIRE(!p->refine || h->has_accurate, RAD_EINVAL,
                    "refinement needs an accurate operator (compress with accurate_dtype = RAD_F32)");
        RAD_REQUIRE(!p->refine || (p->max_refine >= 1 && p->inner_tol > 0.0 && p->inner_tol < 1.0), RAD_EINVAL,
                    "refinement needs max_refine >= 1 and 0 < inner_tol < 1");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const int n = (int)h->n;
        Scratch ws(s);
        const double* epsd = to_device_t(eps, (size_t)n, ws);
        const double* Td = static_cast<const double*>(stage_in_2d(T, n, m, ldT, 8, ws));
        const int64_t ldTd = is_device_ptr(T) ? ldT : n;
        const bool qdev = is_device_ptr(q);
        double* qd = qdev ? q : ws.get_n<double>((size_t)n * m);
        rad_solve_info local{};
        tc_prepare(h, (int)m + 1, s);
        solve_flux(h, epsd, Td, ldTd, (int)m, sigma, p, qd, qdev ? ldq : n, &local, s);
        if (!qdev) {
            RAD_CUDA(cudaMemcpy2DAsync(q, 8 * ldq, qd, 8 * (size_t)n, 8 * (size_t)n, m, cudaMemcpyDeviceToHost, s));
            RAD_CUDA(cudaStreamSynchronize(s));
        }
        RAD_REQUIRE(!wait_timed_out(), RAD_ECUDA, "a pipelined kernel's wait timed out (results are incomplete)");
        if (info) *info = local;
        solve_status = local.status;
        if (solve_status != RAD_OK) set_last_error("GMRES did not reach the tolerance");
    });
    return rc != RAD_OK ? rc : solve_status;
}

int rad_solve_reflection(const rad_htree* h, const double* eps, const double* B, int64_t ldB, int64_t nrhs,
                         const rad_solve_params* p, double* Y, int64_t ldY, rad_solve_info* info, void* stream) {
    int solve_status = RAD_OK;
    const int rc = guarded(__func__, [&] {
        RAD_REQUIRE(h != nullptr && eps && B && Y && p, RAD_EINVAL, "null argument");
        AllocScope as(h->alloc);
        RAD_REQUIRE(h->compressed, RAD_EINVAL, "handle is not compressed (call rad_compress_aca)");
        RAD_REQUIRE(nrhs >= 1 && nrhs <= 1024, RAD_EINVAL, "nrhs must be in [1, 1024]");
        RAD_REQUIRE(ldB >= h->n && ldY >= h->n, RAD_EINVAL, "leading dimension smaller than n");
        RAD_REQUIRE(p->restart >= 1 && p->restart <= 64, RAD_EINVAL, "restart must be in [1, 64]");
        RAD_REQUIRE(p->max_iter >= 1, RAD_EINVAL, "max_iter must be >= 1");
        RAD_REQUIRE(!p->precond || hlu_handle(p->precond) == h, RAD_EINVAL,
                    "the preconditioner's factors belong to another handle");
        RAD_REQUIRE(p->tol > 0.0 && std::isfinite(p->tol), RAD_EINVAL, "tol must be > 0");
        RAD_REQUIRE(!p->refine || h->has_accurate, RAD_EINVAL,
                    "refinement needs an accurate operator (compress with accurate_dtype = RAD_F32)");
        RAD_REQUIRE(!p->refine || (p->max_refine >= 1 && p->inner_tol > 0.0 && p->inner_tol < 1.0), RAD_EINVAL,
                    "refinement needs max_refine >= 1 and 0 < inner_tol < 1");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const int n = (int)h->n;
        Scratch ws(s);
        const double* epsd = to_device_t(eps, (size_t)n, ws);
        const double* Bd = static_cast<const double*>(stage_in_2d(B, n, nrhs, ldB, 8, ws));
        const int64_t ldBd = is_device_ptr(B) ? ldB : n;
        const bool ydev = is_device_ptr(Y);
        double* Yd = ydev ? Y : ws.get_n<double>((size_t)n * nrhs);
        rad_solve_info local{};
        tc_prepare(h, (int)nrhs, s);
        solve_reflection(h, epsd, Bd, ldBd, (int)nrhs, p, Yd, ydev ? ldY : n, &local, s);
        if (!ydev) {
            RAD_CUDA(cudaMemcpy2DAsync(Y, 8 * ldY, Yd, 8 * (size_t)n, 8 * (size_t)n, nrhs, cudaMemcpyDeviceToHost, s));
            RAD_CUDA(cudaStreamSynchronize(s));
        }
        RAD_REQUIRE(!wait_timed_out(), RAD_ECUDA, "a pipelined kernel's wait timed out (results are incomplete)");
        if (info) *info = local;
        solve_status = local.status;
        if (solve_status != RAD_OK) set_last_error("GMRES did not reach the tolerance");
    });
    return rc != RAD_OK ? rc : solve_status;
}

int rad_htree_get_stats(const rad_htree* h, rad_htree_stats* st) {
    return guarded(__func__, [&] {
        RAD_REQUIRE(h != nullptr && st != nullptr, RAD_EINVAL, "null argument");
        std::memset(st, 0, sizeof(*st));
        st->n = h->n;
        st->leaf_size = h->leaf_size;
        st->n_nodes = (int32_t)h->nodes.size();
        int leaves = 0;
        for (auto& nd : h->nodes) leaves += nd.leaf;
        st->n_leaf_clusters = leaves;
        st->depth = h->depth;
        st->n_blocks = (int64_t)h->blocks.size();
        st->n_admissible = h->n_admissible;
        st->compressed = h->compressed ? 1 : 0;
        st->factor_dtype = h->factor_dtype;
        st->near_dtype = h->near_dtype;
        st->max_rank_used = h->max_rank_used;
        st->n_dense_fallback = h->n_dense_fallback;
        st->near_entries = h->near_entries;
        st->far_entries = h->far_entries;
        st->sum_rank = h->sum_rank;
        st->aca_entries = h->aca_entries;
        st->bytes_near = h->near_entries * dtype_size(h->near_dtype);
        st->bytes_far = h->far_entries * dtype_size(h->factor_dtype);
        st->far_u_entries = h->far_u_entries;
        st->far_v_entries = h->far_v_entries;
        st->n_tiles = h->n_tiles;
        st->bytes_accurate = h->far_pool_acc.p ? h->far_entries * 4 : 0;
        st->tuned = h->tuned;
        st->stream_rows = h->stream_rows;
        st->grid_a1 = h->grid_a1;
        st->grid_b1 = h->grid_b1;
        st->grid_a2 = h->grid_a2;
        st->grid_b2 = h->grid_b2;
        st->product_path = h->mm_path;
        st->closed = h->closed;
        st->one_column_path = h->one_col_path == 1 && h->hmv1_ok ? 1 : 0;
        st->reserved = 0;
    });
}

int rad_htree_export_tree(const rad_htree* h, int32_t* perm, int32_t* begin, int32_t* end, int32_t* level,
                          int32_t* child, double* bbox) {
    return guarded(__func__, [&] {
        RAD_REQUIRE(h != nullptr, RAD_EINVAL, "null handle");
        if (perm) std::memcpy(perm, h->perm_h.data(), sizeof(int32_t) * h->perm_h.size());
        for (size_t q = 0; q < h->nodes.size(); ++q) {
            const NodeShape& nd = h->nodes[q];
            if (begin) begin[q] = nd.begin;
            if (end) end[q] = nd.end;
            if (level) level[q] = nd.level;
            if (child) {
                child[2 * q] = nd.child0;
                child[2 * q + 1] = nd.child1;
            }
            if (bbox)
                for (int k = 0; k < 3; ++k) {
                    bbox[6 * q + k] = h->boxes[q].lo[k];
                    bbox[6 * q + 3 + k] = h->boxes[q].hi[k];
                }
        }
    });
}

int rad_htree_export_blocks(const rad_htree* h, int32_t* row_node, int32_t* col_node, int32_t* admissible,
                            int32_t* rank) {
    return guarded(__func__, [&] {
        RAD_REQUIRE(h != nullptr, RAD_EINVAL, "null handle");
        for (size_t b = 0; b < h->blocks.size(); ++b) {
            const BlockH& bk = h->blocks[b];
            if (row_node) row_node[b] = bk.row_node;
            if (col_node) col_node[b] = bk.col_node;
            if (admissible) admissible[b] = bk.admissible;
            if (rank) rank[b] = bk.rank;
        }
    });
}

int rad_htree_export_block(const rad_htree* h, int64_t block, double* D, double* U, double* V) {
    return guarded(__func__, [&] {
        RAD_REQUIRE(h != nullptr, RAD_EINVAL, "null handle");
        AllocScope as(h->alloc);
        export_block(h, block, D, U, V);
    });
}

int rad_htree_autotune(rad_htree* h, void* stream) {
    return guarded(__func__, [&] {
        RAD_REQUIRE(h != nullptr, RAD_EINVAL, "null argument");
        AllocScope as(h->alloc);
        autotune(h, static_cast<cudaStream_t>(stream));
    });
}

int rad_htree_close_cavity(rad_htree* h, double* row_sums, void* stream) {
    return guarded(__func__, [&] {
        RAD_REQUIRE(h != nullptr, RAD_EINVAL, "null argument");
        AllocScope as(h->alloc);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        Scratch ws(s);
        const int n = (int)h->n;
        double* st = ws.get_n<double>(n);
        close_cavity(h, st, s);
        if (row_sums) {
            double* ud = is_device_ptr(row_sums) ? row_sums : ws.get_n<double>(n);
            scatter_tree_to_user(h, st, 1, 1, true, RAD_F64, ud, n, s);
            if (ud != row_sums)
                RAD_CUDA(cudaMemcpyAsync(row_sums, ud, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        }
        RAD_CUDA(cudaStreamSynchronize(s));
    });
}

int rad_htree_set_product_path(rad_htree* h, int32_t path) {
    return guarded(__func__, [&] {
        RAD_REQUIRE(h != nullptr, RAD_EINVAL, "null argument");
        RAD_REQUIRE(path == 0 || path == 1, RAD_EINVAL, "path must be 0 (CUDA cores) or 1 (tensor cores)");
        RAD_REQUIRE(path == 0 || tc_supported(h), RAD_EINVAL,
                    "the tensor-core path needs a compressed FP32 or BF16 operator");
        AllocScope as(h->alloc);
        drop_product_graph(h);
        if (path == 1) {
            tc_build_images(h, nullptr);
        } else {
            tc_drop_images(h, nullptr);
        }
        h->mm_path = path;
    });
}

int rad_htree_set_one_column_path(rad_htree* h, int32_t path) {
    return guarded(__func__, [&] {
        RAD_REQUIRE(h != nullptr, RAD_EINVAL, "null argument");
        RAD_REQUIRE(path == 0 || path == 1, RAD_EINVAL, "path must be 0 (two launches) or 1 (one fused launch)");
        RAD_REQUIRE(path == 0 || h->hmv1_ok, RAD_EINVAL,
                    "the fused one-column product needs a compressed operator with FP32 dense panels, FP32 or "
                    "BF16 factors and panels of at most 1024 rows");
        drop_product_graph(h);
        h->one_col_path = path;
    });
}

int rad_htree_free(rad_htree* h) {
    return guarded(__func__, [&] { delete h; });
}

}  // extern "C"
