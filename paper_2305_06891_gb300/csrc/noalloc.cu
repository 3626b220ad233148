// rad_hmatvec_noalloc: the block matrix product Y = F X without any device
// allocation.
//
// Some callers cannot let this library allocate device memory: a serving
// engine or framework that reserves the GPU's memory for its own pool up
// front (a cudaMalloc from here would fail, or would fragment memory the
// caller has budgeted), or code on a latency-critical path that must not
// enter the CUDA allocator at all.  rad_hmatvec takes its scratch (the
// tree-ordered copies of X and Y and the V^T X workspace) from the
// stream-ordered allocator; this variant takes it from one fixed array in
// device memory instead, declared below, which every GPU that loads the
// library holds until the process exits.
//
// The array is shared by all calls on a device and keeps whatever the last
// call left in it; every byte the product reads is written first within the
// same call, so nothing needs clearing.  Calls whose work overlaps on the
// GPU (different streams, or host threads) race on the array and must be
// serialised by the caller.

#include <cstdio>
#include <mutex>
#include <vector>

#include "rad_common.cuh"

namespace rad {
bool profiling_enabled();
}

// Fixed scratch of the allocation-free product (per device).
constexpr size_t kRadNoAllocScratchBytes = 32ull << 20;
static __device__ __align__(256) unsigned char g_rad_noalloc_scratch[kRadNoAllocScratchBytes];

namespace {

std::mutex g_noalloc_mu;
std::vector<std::pair<int, void*>> g_noalloc_addr;  // device -> address of the array

// Device address of the array on the current device.  In host code the
// array's name only stands in for the symbol, so the address is looked up
// once per device (with that device current) and cached.
void* noalloc_scratch() {
    int dev = 0;
    RAD_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    for (auto& e : g_noalloc_addr)
        if (e.first == dev) return e.second;
    void* p = nullptr;
    const cudaError_t rc = cudaGetSymbolAddress(&p, g_rad_noalloc_scratch);
    if (rc != cudaSuccess || p == nullptr) {
        (void)cudaGetLastError();
        rad::fail(RAD_ECUDA, std::string("cudaGetSymbolAddress(fixed scratch) -> ") + cudaGetErrorString(rc));
    }
    g_noalloc_addr.push_back({dev, p});
    return p;
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

using namespace rad;

extern "C" int rad_hmatvec_noalloc(const rad_htree* h, int32_t dtype, const void* x, int64_t ldx, void* y,
                                   int64_t ldy, int64_t nrhs, void* stream) {
    NvtxRange nv_(__func__);
    try {
        RAD_REQUIRE(h != nullptr && x != nullptr && y != nullptr, RAD_EINVAL, "null argument");
        RAD_REQUIRE(h->compressed, RAD_EINVAL, "handle is not compressed (call rad_compress_aca)");
        RAD_REQUIRE(dtype == RAD_F64 || dtype == RAD_F32, RAD_EINVAL, "dtype must be RAD_F64 or RAD_F32");
        RAD_REQUIRE(nrhs >= 1 && nrhs <= 4096, RAD_EINVAL, "nrhs must be in [1, 4096]");
        RAD_REQUIRE(ldx >= h->n && ldy >= h->n, RAD_EINVAL, "leading dimension smaller than n");
        RAD_REQUIRE(is_device_ptr(x) && is_device_ptr(y), RAD_EINVAL,
                    "rad_hmatvec_noalloc needs device arrays (staging host arrays would allocate)");
        RAD_REQUIRE(!profiling_enabled(), RAD_EINVAL,
                    "rad_hmatvec_noalloc cannot run while rad_profile_enable is on (profiling creates events)");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const int n = (int)h->n;
        const int nr = (int)nrhs;
        const bool op64 = h->op_is_f64();
        const size_t osz = op64 ? 8 : 4;
        // the same layout as rad_hmatvec: tree-order X rows padded to
        // tree_ld(nrhs) columns (16-byte rows for the many-column kernels),
        // Y compact, then the V^T X workspace
        const int ldp = tree_ld(nr);
        const size_t bx = round256(osz * (size_t)n * ldp);
        const size_t by = round256(osz * (size_t)n * nr);
        const size_t bt = round256(apply_workspace_bytes(h, nr));
        const size_t need = bx + by + bt;
        if (need > kRadNoAllocScratchBytes) {
            char msg[256];
            std::snprintf(msg, sizeof msg,
                          "rad_hmatvec_noalloc needs %zu bytes of scratch for n=%d, nrhs=%d but its fixed scratch "
                          "holds %zu bytes; use fewer right-hand sides per call or rad_hmatvec",
                          need, n, nr, kRadNoAllocScratchBytes);
            fail(RAD_ELIMIT, msg);
        }
        unsigned char* base = static_cast<unsigned char*>(noalloc_scratch());
        void* X = base;
        void* Y = base + bx;
        void* T = base + bx + by;
        gather_user_to_tree(h, dtype, x, ldx, nr, X, ldp, op64, s);
        apply_tree(h, X, ldp, Y, nr, nr, Epi{kStore, nullptr, nullptr, nullptr, 0}, T, s);
        scatter_tree_to_user(h, Y, nr, nr, op64, dtype, y, ldy, s);
        check_bounds_after_call();
        return RAD_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.code;
    } catch (...) {
        set_last_error("unknown error");
        return RAD_ECUDA;
    }
}
