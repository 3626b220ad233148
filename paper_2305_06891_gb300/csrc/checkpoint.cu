// Checkpoint and resume of a handle: rad_htree_save writes everything a
// handle holds (trees, block partition, the compressed operator and its
// launch lists, tuning choices) into one byte blob; rad_htree_load builds an
// identical handle from it on the current device.  A loaded handle gives the
// same results bit for bit (same operator bits, same kernels).
//
// Blob layout (all little-endian as written by the host): the 8-byte magic
// "RADHTREE", a u32 format version, then a fixed sequence of fields, each a
// u64 byte count followed by that many bytes.  Every read checks the count
// against what remains and against the type's size, so a truncated or
// foreign blob is rejected with RAD_EINVAL before any device work.

#include <cstring>
#include <string>
#include <vector>

#include "rad_common.cuh"

namespace rad {
namespace {

constexpr char kMagic[8] = {'R', 'A', 'D', 'H', 'T', 'R', 'E', 'E'};
constexpr uint32_t kVersion = 2;

// Scalars of the handle, copied as one struct.
struct Scalars {
    int64_t n;
    int32_t leaf_size, from_dense, depth, compressed;
    double eta, tol;
    int64_t n_admissible;
    int32_t factor_dtype, near_dtype, pivoting, has_accurate;
    int32_t n_sitems, n_aitems, n_tiles, n_gwork;
    int32_t sum_rank, max_rank_used;
    int64_t n_dense_fallback, near_entries, far_entries, aca_entries;
    int64_t far_u_entries, far_v_entries, stored_near, stored_far;
    int32_t stream_rows, grid_a1, grid_b1, grid_a2, grid_b2, tuned, mm_path, closed;
    int32_t one_col_path, pad;
};

struct Writer {
    std::vector<unsigned char> out;
    void raw(const void* p, size_t b) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        out.insert(out.end(), c, c + b);
    }
    void field(const void* p, uint64_t b) {
        raw(&b, sizeof b);
        raw(p, b);
    }
    template <class V>
    void vec(const V& v) {
        field(v.data(), sizeof(typename V::value_type) * v.size());
    }
    void dev(const DevBuf& d) {
        const uint64_t b = d.p ? d.bytes : 0;
        raw(&b, sizeof b);
        if (!b) return;
        const size_t at = out.size();
        out.resize(at + b);
        RAD_CUDA(cudaMemcpy(out.data() + at, d.p, b, cudaMemcpyDeviceToHost));
    }
};

struct Reader {
    const unsigned char* p;
    size_t left;
    const unsigned char* take(size_t b) {
        RAD_REQUIRE(b <= left, RAD_EINVAL, "checkpoint blob is truncated");
        const unsigned char* r = p;
        p += b;
        left -= b;
        return r;
    }
    uint64_t count() {
        uint64_t b;
        std::memcpy(&b, take(sizeof b), sizeof b);
        RAD_REQUIRE(b <= left, RAD_EINVAL, "checkpoint blob is truncated");
        return b;
    }
    void field(void* dst, uint64_t want) {
        const uint64_t b = count();
        RAD_REQUIRE(b == want, RAD_EINVAL, "checkpoint field has the wrong size");
        std::memcpy(dst, take(b), b);
    }
    template <class V>
    void vec(V& v) {
        const uint64_t b = count();
        using T = typename V::value_type;
        RAD_REQUIRE(b % sizeof(T) == 0, RAD_EINVAL, "checkpoint array has the wrong size");
        v.resize(b / sizeof(T));
        if (b) std::memcpy(v.data(), take(b), b);
    }
    void dev(DevBuf& d, cudaStream_t s) {
        const uint64_t b = count();
        const unsigned char* src = take(b);
        if (!b) return;
        d.alloc(b, s);
        RAD_CUDA(cudaMemcpyAsync(d.p, src, b, cudaMemcpyHostToDevice, s));
    }
};

// The device buffers of a handle, in blob order.
template <class H>
auto device_buffers(H* h) {
    return std::vector<decltype(&h->geo)>{&h->d_segrow,  &h->geo,     &h->geo32,    &h->perm,     &h->iperm,
                                          &h->near_pool, &h->far_pool, &h->far_pool_acc, &h->d_tiles, &h->d_xidx,
                                          &h->d_tidx,    &h->d_gwork, &h->d_groups, &h->d_sitems, &h->d_torder,
                                          &h->d_aorder,  &h->d_forder};
}

}  // namespace
}  // namespace rad

using namespace rad;

extern "C" {

int rad_htree_save(const rad_htree* h, void* buf, uint64_t* bytes) {
    NvtxRange nv_(__func__);
    try {
        RAD_REQUIRE(h != nullptr && bytes != nullptr, RAD_EINVAL, "null argument");
        RAD_CUDA(cudaDeviceSynchronize());   // every queued write to the handle's buffers is done
        Writer w;
        w.raw(kMagic, sizeof kMagic);
        w.raw(&kVersion, sizeof kVersion);
        Scalars sc{};
        sc.n = h->n;
        sc.leaf_size = h->leaf_size;
        sc.from_dense = h->from_dense;
        sc.depth = h->depth;
        sc.compressed = h->compressed;
        sc.eta = h->eta;
        sc.tol = h->tol;
        sc.n_admissible = h->n_admissible;
        sc.factor_dtype = h->factor_dtype;
        sc.near_dtype = h->near_dtype;
        sc.pivoting = h->pivoting;
        sc.has_accurate = h->has_accurate;
        sc.n_sitems = h->n_sitems;
        sc.n_aitems = h->n_aitems;
        sc.n_tiles = h->n_tiles;
        sc.n_gwork = h->n_gwork;
        sc.sum_rank = h->sum_rank;
        sc.max_rank_used = h->max_rank_used;
        sc.n_dense_fallback = h->n_dense_fallback;
        sc.near_entries = h->near_entries;
        sc.far_entries = h->far_entries;
        sc.aca_entries = h->aca_entries;
        sc.far_u_entries = h->far_u_entries;
        sc.far_v_entries = h->far_v_entries;
        sc.stored_near = h->stored_near;
        sc.stored_far = h->stored_far;
        sc.stream_rows = h->stream_rows;
        sc.grid_a1 = h->grid_a1;
        sc.grid_b1 = h->grid_b1;
        sc.grid_a2 = h->grid_a2;
        sc.grid_b2 = h->grid_b2;
        sc.tuned = h->tuned;
        sc.mm_path = h->mm_path;
        sc.closed = h->closed;
        sc.one_col_path = h->one_col_path;
        w.field(&sc, sizeof sc);
        w.vec(h->seg);
        w.vec(h->nodes);
        w.vec(h->boxes);
        w.vec(h->perm_h);
        w.vec(h->blocks);
        w.vec(h->tiles_h);
        w.vec(h->groups_h);
        w.vec(h->near_pieces);
        w.vec(h->far_pieces);
        for (const DevBuf* d : device_buffers(h)) w.dev(*d);
        const uint64_t need = w.out.size();
        if (buf == nullptr) {
            *bytes = need;
            return RAD_OK;
        }
        RAD_REQUIRE(*bytes >= need, RAD_ELIMIT,
                    "the buffer is smaller than the checkpoint (" + std::to_string(need) + " bytes)");
        std::memcpy(buf, w.out.data(), need);
        *bytes = need;
        return RAD_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.code;
    } catch (const std::bad_alloc&) {
        set_last_error("host allocation failed");
        return RAD_ENOMEM;
    }
}

int rad_htree_load(const void* buf, uint64_t bytes, const rad_tree_params* p, void* stream, rad_htree** out) {
    NvtxRange nv_(__func__);
    try {
        RAD_REQUIRE(buf != nullptr && out != nullptr, RAD_EINVAL, "null argument");
        *out = nullptr;
        RAD_REQUIRE(!p || !p->allocator || (p->allocator->alloc && p->allocator->free), RAD_EINVAL,
                    "an allocator needs both alloc and free");
        Reader r{static_cast<const unsigned char*>(buf), (size_t)bytes};
        RAD_REQUIRE(std::memcmp(r.take(sizeof kMagic), kMagic, sizeof kMagic) == 0, RAD_EINVAL,
                    "not a librad checkpoint");
        uint32_t ver;
        std::memcpy(&ver, r.take(sizeof ver), sizeof ver);
        RAD_REQUIRE(ver == kVersion, RAD_EINVAL, "unsupported checkpoint version");
        Scalars sc{};
        r.field(&sc, sizeof sc);
        RAD_REQUIRE(sc.n >= 1 && sc.n < (int64_t)1 << 28, RAD_EINVAL, "checkpoint: bad facet count");
        auto h = std::make_unique<rad_htree>();
        if (p && p->allocator) h->alloc.cb = *p->allocator;
        AllocScope as(h->alloc);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        RAD_CUDA(cudaGetDevice(&h->device));
        h->n = sc.n;
        h->leaf_size = sc.leaf_size;
        h->from_dense = sc.from_dense != 0;
        h->depth = sc.depth;
        h->compressed = sc.compressed != 0;
        h->eta = sc.eta;
        h->tol = sc.tol;
        h->n_admissible = sc.n_admissible;
        h->factor_dtype = sc.factor_dtype;
        h->near_dtype = sc.near_dtype;
        h->pivoting = sc.pivoting;
        h->has_accurate = sc.has_accurate != 0;
        h->n_sitems = sc.n_sitems;
        h->n_aitems = sc.n_aitems;
        h->n_tiles = sc.n_tiles;
        h->n_gwork = sc.n_gwork;
        h->sum_rank = sc.sum_rank;
        h->max_rank_used = sc.max_rank_used;
        h->n_dense_fallback = sc.n_dense_fallback;
        h->near_entries = sc.near_entries;
        h->far_entries = sc.far_entries;
        h->aca_entries = sc.aca_entries;
        h->far_u_entries = sc.far_u_entries;
        h->far_v_entries = sc.far_v_entries;
        h->stored_near = sc.stored_near;
        h->stored_far = sc.stored_far;
        h->stream_rows = sc.stream_rows;
        h->grid_a1 = sc.grid_a1;
        h->grid_b1 = sc.grid_b1;
        h->grid_a2 = sc.grid_a2;
        h->grid_b2 = sc.grid_b2;
        h->tuned = sc.tuned;
        h->mm_path = sc.mm_path;
        h->closed = sc.closed;
        h->one_col_path = sc.one_col_path;
        r.vec(h->seg);
        r.vec(h->nodes);
        r.vec(h->boxes);
        r.vec(h->perm_h);
        r.vec(h->blocks);
        r.vec(h->tiles_h);
        r.vec(h->groups_h);
        r.vec(h->near_pieces);
        r.vec(h->far_pieces);
        RAD_REQUIRE(h->perm_h.size() == (size_t)h->n && h->boxes.size() == h->nodes.size() &&
                        (int64_t)h->tiles_h.size() == h->n_tiles,
                    RAD_EINVAL, "checkpoint arrays do not fit together");
        for (DevBuf* d : device_buffers(h.get())) r.dev(*d, s);
        RAD_REQUIRE(r.left == 0, RAD_EINVAL, "checkpoint blob has trailing bytes");
        RAD_REQUIRE(h->perm.bytes == sizeof(int) * (size_t)h->n && h->geo.bytes == sizeof(double) * 7 * (size_t)h->n,
                    RAD_EINVAL, "checkpoint device arrays do not fit the facet count");
        // derived data, rebuilt: the fused one-column units now, the
        // tensor-core images at the first many-column product
        if (h->compressed) hmv1_plan(h.get(), s);
        RAD_CUDA(cudaStreamSynchronize(s));
        check_bounds_after_call();
        *out = h.release();
        return RAD_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.code;
    } catch (const std::bad_alloc&) {
        set_last_error("host allocation failed");
        return RAD_ENOMEM;
    }
}

}  // extern "C"
