// Internal declarations shared by the librad translation units.
#pragma once

#include <chrono>
#include <condition_variable>

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <cstring>
#include <exception>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "rad.h"

namespace rad {

// NVTX range around one C-ABI call, named after it: visible on the timeline
// of Nsight tools, a no-op when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ------------------------------------------------------------ error plumbing
struct Error {
    int code;
    std::string msg;
};

[[noreturn]] void fail(int code, const std::string& msg);
void set_last_error(const std::string& msg);

#define RAD_CUDA(call)                                                            \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            (void)cudaGetLastError();                                             \
            ::rad::fail(e_ == cudaErrorMemoryAllocation ? RAD_ENOMEM : RAD_ECUDA, \
                        std::string(#call) + " -> " + cudaGetErrorString(e_));    \
        }                                                                         \
    } while (0)

void note_launch();
void note_launches(long long k);
long long launch_count();
#define RAD_CHECK_LAUNCH()                \
    do {                                  \
        ::rad::note_launch();             \
        RAD_CUDA(cudaGetLastError());     \
    } while (0)

// Optional per-kernel event timing (rad_profile_enable).  A scope records a
// start event on construction and a stop event on destruction, on the given
// stream; it costs nothing while profiling is off.
struct ProfScope {
    int idx = -1;
    cudaStream_t s;
    ProfScope(const char* name, cudaStream_t st);
    ~ProfScope();
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;
};

// Host wall time of a phase (names start with "host_"), recorded beside the
// kernel times while profiling is on.
struct HostScope {
    const char* name;
    std::chrono::steady_clock::time_point t0;
    explicit HostScope(const char* n);
    ~HostScope();
    HostScope(const HostScope&) = delete;
    HostScope& operator=(const HostScope&) = delete;
};

#define RAD_REQUIRE(cond, code, msg)          \
    do {                                      \
        if (!(cond)) ::rad::fail(code, msg);  \
    } while (0)

// Bounds-checked build (-DRAD_CHECK_BOUNDS, librad_checked.so): verifies the
// canary words around every device allocation; call before an entry point
// returns RAD_OK.  A no-op in the ordinary build.
void check_bounds_after_call();

// ------------------------------------------------------------ memory helpers
// Where device memory comes from: the caller's rad_allocator callbacks, or
// (cb.alloc == nullptr) the library's own stream-ordered pool of the current
// device, which keeps freed memory cached.
struct Allocator {
    rad_allocator cb{nullptr, nullptr, nullptr};
    void* get(size_t bytes, cudaStream_t s) const;          // fails with RAD_ENOMEM
    void put(void* p, size_t bytes, cudaStream_t s) const;  // never throws
};
// The allocator of the library call running on this thread: entry points
// that work on a handle install the handle's allocator for their duration
// (AllocScope); elsewhere it is the library's pool.
const Allocator& current_allocator();
struct AllocScope {
    Allocator prev;
    explicit AllocScope(const Allocator& a);
    ~AllocScope();
    AllocScope(const AllocScope&) = delete;
    AllocScope& operator=(const AllocScope&) = delete;
};

// A device buffer owned by a handle, from the allocator current at alloc();
// it remembers that allocator and returns the memory to it.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    Allocator al;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(nullptr); }
    // Stream-ordered allocation on stream `s`; release frees in the order of
    // stream `s`.
    void alloc(size_t b, cudaStream_t s);
    void release(cudaStream_t s);
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// Per-call stream-ordered workspace from the current allocator; everything
// is freed (stream-ordered) when the object goes out of scope.
struct Scratch {
    cudaStream_t s;
    Allocator al;
    std::vector<std::pair<void*, size_t>> ptrs;
    explicit Scratch(cudaStream_t st) : s(st), al(current_allocator()) {}
    Scratch(const Scratch&) = delete;
    ~Scratch();
    void* get(size_t bytes);
    template <class T> T* get_n(size_t n) { return static_cast<T*>(get(n * sizeof(T))); }
};

bool is_device_ptr(const void* p);
// Returns a device copy of `count` elements of a host or device array.
const void* to_device(const void* p, size_t bytes, Scratch& ws);
template <class T>
const T* to_device_t(const T* p, size_t n, Scratch& ws) {
    return static_cast<const T*>(to_device(p, n * sizeof(T), ws));
}
// Page-locked staging for the host-to-device uploads of one call (per host
// thread).  While a StageScope is alive, h2d() copies through page-locked
// memory, so the copies are asynchronous DMA instead of staged pageable
// copies.  The code holding the scope synchronises its stream before the
// scope ends (tree build and compression do), so the staging memory is free
// for the next call.
struct StageScope {
    StageScope();
    ~StageScope();
    StageScope(const StageScope&) = delete;
    StageScope& operator=(const StageScope&) = delete;
};
void* stage_alloc(size_t bytes);   // nullptr when no scope is active

// Allocator whose value construction without arguments leaves trivially
// constructible elements uninitialised: host work lists that are filled
// right after resize() skip the zeroing pass.
template <class T>
struct NoInitAlloc : std::allocator<T> {
    template <class U>
    struct rebind {
        using other = NoInitAlloc<U>;
    };
    NoInitAlloc() = default;
    template <class U>
    NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
    template <class U, class... A>
    void construct(U* p, A&&... a) {
        ::new ((void*)p) U(std::forward<A>(a)...);
    }
    template <class U>
    void construct(U* p) {
        ::new ((void*)p) U;
    }
};
template <class T>
using HVec = std::vector<T, NoInitAlloc<T>>;

// Host copy into page-locked staging; 8 threads from 8 MiB.
void stage_copy(void* dst, const void* src, size_t bytes);

template <class T, class Al>
void h2d(T* dst, const std::vector<T, Al>& v, cudaStream_t s) {
    if (v.empty()) return;
    const size_t bytes = v.size() * sizeof(T);
    void* st = bytes >= 4096 ? stage_alloc(bytes) : nullptr;
    if (st) {
        stage_copy(st, v.data(), bytes);
        RAD_CUDA(cudaMemcpyAsync(dst, st, bytes, cudaMemcpyHostToDevice, s));
    } else {
        RAD_CUDA(cudaMemcpyAsync(dst, v.data(), bytes, cudaMemcpyHostToDevice, s));
    }
}

inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Runs job(q) for q = 0 .. parts-1 on the library's host worker pool (the
// caller takes part too); returns false without running anything when the
// pool is busy with another caller's job (e.g. another server thread).
bool pool_run(int parts, void (*job)(void*, int), void* ctx);

// Runs f(q) for q = 0 .. parts-1, parts > 1 on host threads (q = 0 on the
// calling thread): the persistent worker pool, or freshly started threads
// while the pool serves another caller; the first exception thrown by any
// part is rethrown.
template <class F>
void parallel_parts(int parts, F&& f) {
    if (parts <= 1) {
        f(0);
        return;
    }
    std::vector<std::exception_ptr> err(parts);
    auto run = [&](int q) {
        try {
            f(q);
        } catch (...) {
            err[q] = std::current_exception();
        }
    };
    using Run = decltype(run);
    if (!pool_run(parts, [](void* c, int q) { (*static_cast<Run*>(c))(q); }, &run)) {
        std::vector<std::thread> th;
        th.reserve(parts - 1);
        for (int q = 1; q < parts; ++q) th.emplace_back(run, q);
        run(0);
        for (auto& t : th) t.join();
    }
    for (auto& e : err)
        if (e) std::rethrow_exception(e);
}
inline int dtype_size(int dt) { return dt == RAD_F64 ? 8 : dt == RAD_F32 ? 4 : 2; }

// ------------------------------------------------------------ data layout
// Facet geometry in tree order, structure of arrays: 7 x n doubles (cx, cy,
// cz, nx, ny, nz, area) plus an FP32 copy of 10 x n floats in which every
// centroid coordinate is split into hi = fl32(c) and lo = fl32(c - hi), so
// that c_j - c_i = (hi_j - hi_i) + (lo_j - lo_i) keeps ~FP64-relative
// accuracy for nearby facets using FP32 arithmetic only (GB300's FP64 pipe
// is narrow); then nx, ny, nz, area as floats.
struct Geo {
    const double* cx;
    const double* cy;
    const double* cz;
    const double* nx;
    const double* ny;
    const double* nz;
    const double* area;
    const float* xh;
    const float* xl;
    const float* yh;
    const float* yl;
    const float* zh;
    const float* zl;
    const float* fnx;
    const float* fny;
    const float* fnz;
    const float* farea;
};
inline Geo geo_view(const double* base, const float* b32, int64_t n) {
    return Geo{base,         base + n,     base + 2 * n, base + 3 * n, base + 4 * n, base + 5 * n,
               base + 6 * n, b32,          b32 + n,      b32 + 2 * n,  b32 + 3 * n,  b32 + 4 * n,
               b32 + 5 * n,  b32 + 6 * n,  b32 + 7 * n,  b32 + 8 * n,  b32 + 9 * n};
}

// Cluster shape (fixed by n and leaf_size) plus its bounding box.
struct NodeShape {
    int begin, end, level, child0, child1, leaf;
};
struct NodeBox {
    double lo[3], hi[3];
};

// Operator storage ("panels").
//
// Row tile: rows [r0, r0 + rows) of the matrix (a leaf cluster cut into
// pieces of at most 64 rows), leading dimension ld = round_up(rows, 4).  Its
// dense panel (near storage type) holds the tile's rows of every dense block
// that covers it, side by side: kn columns, column-major, at noff; column c
// multiplies row xidx[ixn + c] of X.  Its low-rank panel (factor storage
// type) holds the tile's rows of U for every low-rank block covering it: kf
// columns at foff; column c multiplies row tidx[ixf + c] of T = V^T X.
struct Tile {
    int r0, rows, ld, kn, kf, ixn, ixf, pad;
    long long noff, foff;
};
// Column group: the low-rank blocks whose column cluster is [c0, c0 + n).
// Its V panel stacks their V^T rows: M rows (block b, column l of V_b),
// ld = round_up(M, 4), n columns, column-major at voff (factor storage
// type).  Its rows of T are [toff, toff + M).
struct Group {
    int c0, n, M, ld, toff, pad;
    long long voff;
};
// Phase-1 work item: rows [r0, r0 + rows) (rows <= 64) of group g.
struct GWork {
    int g, r0, rows, pad;
};

constexpr int kTileRows = 64;
constexpr int kMaxRank = 128;

// Leading dimension of the tree-order vector blocks (X, T, Y) used by the
// product for nrhs right-hand sides: 1 for one, else a multiple of 4 so that
// every row starts on a 16-byte boundary.
inline int tree_ld(int nrhs) { return nrhs == 1 ? 1 : (int)((nrhs + 3) / 4 * 4); }

// Canonical leaf block (export order = sorted by (r0, c0)).
struct BlockH {
    int row_node, col_node;
    int r0, r1, c0, c1;
    int admissible;
    int rank;        // -1: stored dense
    int group;       // low-rank: column group holding V^T (else -1)
    int grow;        // low-rank: first row of its V^T in that group
};
// One piece of a block stored in a row tile: tile t, first panel column.
struct Piece {
    int block, tile, col;
};

// Device view of a compressed operator, passed by value to the kernels.
struct OpView {
    int n_tiles;
    const Tile* tiles;
    const void* near_pool;
    const void* far_pool;
    const int* xidx;
    const int* tidx;
    int n_gwork;
    const GWork* gwork;
    const Group* groups;
    int sum_rank;
    int n_sitems;           // far-field items of <= kStreamRows rows for 1-4 columns
    const GWork* sitems;
    const int* torder;      // launch order of the row tiles (heaviest first)
    // one-column product in two launches: phase A runs the far-field items
    // (code >= 0: sitems[code]) and the dense panels of the tiles (code < 0:
    // tile -code-1) together, heaviest first; phase B the low-rank panels of
    // the tiles in forder
    int n_aitems;
    const int* aorder;
    const int* forder;
};

// Rows per far-field item of the streaming (1-4 column) products.
constexpr int kStreamRows = 128;

}  // namespace rad

// The opaque handle (global namespace: it is the C type rad_htree).
// A one-product CUDA graph kept by a handle: rad_hmatvec on device arrays
// captures (gather, product, scatter) on the second identical call (same
// arrays, leading dimensions, columns, dtype and stream) and replays it
// afterwards; its tree-order vectors and workspace belong to the cache.
struct ProductGraph {
    std::mutex mu;
    const void* x = nullptr;
    void* y = nullptr;
    int64_t ldx = 0, ldy = 0, nrhs = 0;
    int dtype = -1;
    cudaStream_t stream = nullptr;
    int hits = 0;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture = nullptr;
    long long kernels = 0;
    rad::DevBuf X, Y, T;
    ~ProductGraph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (capture) cudaStreamDestroy(capture);
    }
};

struct rad_htree {
    // The arrays below may still be read by work queued on any stream when
    // the handle goes away (rad_htree_free, or a call that failed half way):
    // wait for the device before they return to the pool.
    ~rad_htree() {
        if (sync_on_destroy) (void)cudaDeviceSynchronize();
    }
    // false only when the owner knows no queued work reads the handle
    bool sync_on_destroy = true;
    mutable std::unique_ptr<ProductGraph> graph;
    // launch configuration of the streaming products, chosen by
    // rad_htree_autotune: rows per far-field item, and grid sizes (0 = one
    // CTA per work item, else a persistent grid-stride launch) of phase A /
    // phase B for one column (a1, b1) and for 2-4 columns (a2, b2)
    int stream_rows = rad::kStreamRows;
    int grid_a1 = 0, grid_b1 = 0, grid_a2 = 0, grid_b2 = 0;
    int tuned = 0;
    // many-column product of FP32 vectors: 0 = CUDA-core register tiles,
    // 1 = tensor cores (BF16 x 3 split; the default after rad_compress_aca
    // for FP32 and BF16 operators; images built at the first product of 5
    // or more columns, never for one-column use); set by
    // rad_htree_autotune or rad_htree_set_product_path
    int mm_path = 0;
    // tensor-core path: the BF16 chunk images of every work item, the work
    // items (row tiles, far-field slices; heaviest first) and their K-groups
    // (source vector rows of runs of up to 8 panel columns)
    rad::DevBuf tc_img, tc_rows_items, tc_far_items, tc_kgs;
    int tc_n_rows = 0, tc_n_far = 0, tc_r8max = 8;   // items; their largest row count rounded up to 8
    bool tc_ready = false;
    std::mutex tc_mu;                                 // first-use build of the images
    std::vector<int> tc_cnt_h;                        // K-groups per row tile, counted with the operator
    // the last product's two tensor maps (X and T planes), reused while the
    // workspace address and the column-group count stay the same
    struct TcMaps {
        const void* ws = nullptr;
        int G = 0;
        alignas(64) unsigned char map[2][128];
    } tc_maps;
    // one-column product: 1 = the fused single launch (when the operator
    // allows it, hmv1_ok), 0 = the two launches (phase A, phase B); set by
    // rad_htree_autotune or rad_htree_set_one_column_path.  The fused
    // launch's work units (A units, then B units) are rebuilt with the
    // operator.
    int one_col_path = 1;
    rad::DevBuf d_units1;
    int n_units1 = 0, n_a1 = 0;
    bool hmv1_ok = false;
    int closed = 0;   // rows normalised for a closed cavity (rad_htree_close_cavity)
    int64_t n = 0;
    rad::Allocator alloc;   // device memory of the handle and of calls on it
    // segment (cavity) boundaries of a batch handle: cavity c holds facets
    // [seg[c], seg[c+1]) in user order and in tree order; {0, n} otherwise
    std::vector<int64_t> seg;
    rad::DevBuf d_segrow;   // segment of every tree-order row (batches only)
    int leaf_size = 0;
    double eta = 0.0;
    int device = 0;
    bool from_dense = false;

    rad::DevBuf geo;     // 7 x n doubles, tree order
    rad::DevBuf geo32;   // 10 x n floats, tree order (hi/lo centroids)
    rad::DevBuf perm;    // int32, tree position -> facet
    rad::DevBuf iperm;   // int32, facet -> tree position

    std::vector<rad::NodeShape> nodes;
    std::vector<rad::NodeBox> boxes;
    std::vector<int> perm_h;
    int depth = 0;

    std::vector<rad::BlockH> blocks;   // canonical order
    int64_t n_admissible = 0;

    // compressed operator
    bool compressed = false;
    int factor_dtype = RAD_F64;
    int near_dtype = RAD_F64;
    double tol = 0.0;
    int pivoting = RAD_ACA_PARTIAL;
    std::vector<rad::Tile> tiles_h;
    std::vector<rad::Group> groups_h;
    std::vector<rad::GWork> gwork_h;          // far-field items (launch order)
    rad::HVec<rad::Piece> near_pieces, far_pieces;     // per tile, in panel order
    rad::DevBuf near_pool, far_pool;
    rad::DevBuf far_pool_acc;          // FP32 factors kept for refinement
    bool has_accurate = false;         // an accurate operator exists
    rad::DevBuf d_tiles, d_xidx, d_tidx, d_gwork, d_groups, d_sitems, d_torder, d_aorder, d_forder;
    int n_sitems = 0;
    int n_aitems = 0;
    int n_tiles = 0;
    int n_gwork = 0;
    int sum_rank = 0;
    int max_rank_used = 0;
    int64_t n_dense_fallback = 0;
    int64_t near_entries = 0, far_entries = 0, aca_entries = 0;
    int64_t far_u_entries = 0, far_v_entries = 0;
    int64_t stored_near = 0, stored_far = 0;   // elements incl. padding

    rad::OpView view() const {
        rad::OpView v;
        v.n_tiles = n_tiles;
        v.tiles = d_tiles.as<rad::Tile>();
        v.near_pool = near_pool.p;
        v.far_pool = far_pool.p;
        v.xidx = d_xidx.as<int>();
        v.tidx = d_tidx.as<int>();
        v.n_gwork = n_gwork;
        v.gwork = d_gwork.as<rad::GWork>();
        v.groups = d_groups.as<rad::Group>();
        v.sum_rank = sum_rank;
        v.n_sitems = n_sitems;
        v.sitems = d_sitems.as<rad::GWork>();
        v.torder = d_torder.as<int>();
        v.n_aitems = n_aitems;
        v.aorder = d_aorder.as<int>();
        v.forder = d_forder.as<int>();
        return v;
    }
    bool op_is_f64() const { return near_dtype == RAD_F64; }
    // the accurate operator: FP32 factors (the BF16 path's second copy, or
    // the FP32 factors themselves)
    const void* accurate_far_pool() const { return far_pool_acc.p ? far_pool_acc.p : far_pool.p; }
};

namespace rad {
// tree.cu
void build_geometry_from_tris(rad_htree* h, const double* verts_dev, double* geo_user, cudaStream_t s);
void build_geometry_from_facets(rad_htree* h, const double* c, const double* nrm, const double* a,
                                double* geo_user, cudaStream_t s);
void build_trees(rad_htree* h, const double* geo_user, cudaStream_t s);
// aca.cu
void compress(rad_htree* h, const rad_aca_params* p, cudaStream_t s);
void load_dense_operator(rad_htree* h, const double* F_dev_rowmajor, cudaStream_t s);
void export_block(const rad_htree* h, int64_t b, double* D, double* U, double* V);
// hmatvec.cu
// Epilogue of the tree-order product Y = F X (row-major, leading dims ldx/ldy):
//   kStore:   Y = F X
//   kReflect: Y = Xin - (1 - eps) o F X            (C applied, Eq. 11)
//   kResid:   Y = B - (Xin - (1 - eps) o F X)      (residual of Eq. 11)
enum EpiMode { kStore = 0, kReflect = 1, kResid = 2 };
struct Epi {
    int mode;
    const double* eps;   // tree order
    const double* xin;   // FP64 vectors, row-major, leading dim ld64
    const double* b;     // FP64 right-hand sides, leading dim ld64
    int ld64;
};
void apply_tree(const rad_htree* h, const void* X, int ldx, void* Y, int ldy, int nrhs,
                const Epi& epi, void* T_ws, cudaStream_t s);
// The accurate operator (FP32 storage) with FP64 vectors and FP64
// accumulation; T_ws holds apply_workspace_bytes_acc(h, nrhs) bytes.
void apply_tree_acc(const rad_htree* h, const double* X, int ldx, double* Y, int ldy, int nrhs, const Epi& epi,
                    double* T_ws, cudaStream_t s);
size_t apply_workspace_bytes_acc(const rad_htree* h, int nrhs);
size_t apply_workspace_bytes(const rad_htree* h, int nrhs);
// tcgemm.cu: tensor-core panel GEMMs (BF16 x 3 split, FP32 vectors)
bool tc_supported(const rad_htree* h);
void tc_build_images(rad_htree* h, cudaStream_t s);
void tc_prepare(const rad_htree* h, int ncols, cudaStream_t s);
void tc_count_async(rad_htree* h, cudaStream_t s);
void tc_drop_images(rad_htree* h, cudaStream_t s);   // frees stream-ordered on s
size_t tc_workspace_bytes(const rad_htree* h, int nrhs);
void tc_product(const rad_htree* h, const OpView& op, const float* X, int ldx, void* Y, int ldy, int nc,
                const Epi& epi, void* ws, cudaStream_t s);
bool tc_take_timeout();
// hmv1.cu: the fused one-column product (FP32 vectors, FP32 dense panels,
// FP32 or BF16 factors)
void hmv1_plan(rad_htree* h, cudaStream_t s);
void hmv1_product(const rad_htree* h, const float* x, float* T, float* Yn, int* ctr, void* Y, const Epi& epi,
                  cudaStream_t s);
bool hmv1_take_timeout();
// true when a bounded wait of a pipelined kernel gave up since the last call
// (clears the flags)
inline bool wait_timed_out() {
    const bool a = tc_take_timeout();
    const bool b = hmv1_take_timeout();
    return a || b;
}
void build_stream_lists(rad_htree* h, int rows, cudaStream_t s);
void autotune(rad_htree* h, cudaStream_t s);
void close_cavity(rad_htree* h, double* s_tree_out, cudaStream_t s);
void drop_product_graph(const rad_htree* h);
void gather_user_to_tree(const rad_htree* h, int dtype_in, const void* x, int64_t ldx, int nrhs,
                         void* X, int ldX, bool op64, cudaStream_t s);
void scatter_tree_to_user(const rad_htree* h, const void* Y, int ldY, int nrhs, bool op64,
                          int dtype_out, void* y, int64_t ldy, cudaStream_t s);
// hlu.cu: x = U^-1 L^-1 x on tree-order FP64 row-major vectors (n x nc)
void hlu_apply_tree(const rad_hlu* lu, double* X, int nc, cudaStream_t s);
const rad_htree* hlu_handle(const rad_hlu* lu);
// gmres.cu
void solve_flux(const rad_htree* h, const double* eps_dev, const double* T_dev, int64_t ldT,
                int m, double sigma, const rad_solve_params* p, double* q_dev, int64_t ldq,
                rad_solve_info* info, cudaStream_t s);
void solve_reflection(const rad_htree* h, const double* eps_dev, const double* B_dev, int64_t ldB, int nrhs,
                      const rad_solve_params* p, double* Y_dev, int64_t ldY, rad_solve_info* info, cudaStream_t s);
}  // namespace rad
