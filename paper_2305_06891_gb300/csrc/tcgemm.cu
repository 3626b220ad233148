// Tensor-core (tcgen05) panel GEMMs of the many-column product, FP32
// operands at FP32-level accuracy.
//
// The product of one work item (a row tile, or a slice of at most 64 rows of
// a column group's V^T panel) runs transposed on the 5th-generation tensor
// cores: D[M x N] = sum_k A[M x k] B[k x N] with M = the right-hand-side
// columns (64 or 128, the MMA's M), N = the item's rows (rounded up to 8 or
// 16), K = the item's panel columns.  Column k of A is the vector row that
// panel column k multiplies (a row of X, or of T = V^T X); B is the panel
// transposed.  D sits in tensor memory with one lane per right-hand side, so
// the epilogue writes every output row with consecutive lanes on consecutive
// columns.
//
// Accuracy: kind::f16 with BF16 operands and FP32 accumulators.  BF16 keeps
// 8 mantissa bits, so every FP32 operand x is split into three BF16 pieces,
// x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2), which together
// carry its 24 bits; the product takes the six terms a1 b1 (the "main"
// accumulator) and a1 b2 + a2 b1 + a1 b3 + a2 b2 + a3 b1 (a second,
// "correction" accumulator), dropping terms of order 2^-24 relative.  The
// tensor core's accumulation truncates, so the accumulators start from zero
// every 128 panel columns and are added into FP32 registers (round to
// nearest): the rounding stays at the level of an FP32 FFMA loop.
//
// Data movement (no gathers by threads):
//   - panel columns are cut into K-groups: runs of at most 8 columns whose
//     vector rows are consecutive (a dense block's columns, a low-rank
//     block's T rows).  Each K-group's 8 vector rows arrive by one TMA tile
//     copy from vector planes stored group-major, [plane][column group][row]
//     [8 columns]: 8 consecutive rows of a column group are 128 contiguous
//     bytes, so the box (64 elements x G = ceil(columns / 8) groups x 3
//     planes) moves whole 128-byte lines and lands as MN-major core matrices
//     (8 rows of 16 bytes; column groups 128 bytes apart, planes 128 G bytes
//     apart, K-groups one box apart).  The MMA reads M/8 groups per plane:
//     those past G (the next plane's data) only reach rows of D past the
//     last column, which are never read.
//     Panel columns past a run's end are zero in the image, so the box's
//     other rows (neighbouring vector rows, or the zeros the copy fills in
//     past the last row or column group) add nothing;
//   - the panels are split once per operator (at its first product of 5 or
//     more columns, or when the path is selected) into chunk images of 8
//     K-groups, [plane][K-group][8-row group][8 rows][8 columns] (K-major
//     core matrices), rows padded with zeros to a multiple of 8; a chunk
//     moves by one bulk copy.  The K-groups of a row tile are found by one
//     warp walking its gather indices in column order, so the layout does
//     not depend on who builds it.
// Persistent, warp-specialised kernel (one CTA of 192 threads per SM, items
// taken round-robin, heaviest first):
//   - lane 0 of warp 0 issues the copies of every chunk (8 tensor copies and
//     one bulk copy, completing on the stage's "full" mbarrier) into a ring
//     of shared-memory stages, with the K-group rows of the next 32 to 64
//     chunks already in the warp's registers;
//   - lane 0 of warp 1 issues each chunk's 4 k-steps x 6 MMAs into one of
//     four accumulator pairs in tensor memory (so that it runs up to three
//     drains ahead), with descriptors stepped by additions;
//   - warps 2-5 (tensor-memory lane quarters 2, 3, 0, 1) add a pair into
//     FP32 registers after every 2 chunks of an item and write the item's
//     rows at its end (the FP64 epilogue's inputs loaded 16 rows ahead of
//     the stores).
// The roles hand over through mbarriers and never wait for the whole CTA.
// Every wait is bounded: after a bounded number of tries a role raises an
// abort flag that the others see, the CTA records the timeout in a device
// flag (checked by the host at its next synchronisation), waits (bounded)
// for its own copies and MMAs in flight and frees its tensor memory.

#include <cstdint>
#include <cstring>
#include <mutex>
#include <algorithm>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "rad_device.cuh"

namespace rad {

__device__ int g_tc_timeout = 0;

namespace {

constexpr int kKG = 8;                        // panel columns per K-group
constexpr int kGPC = 8;                       // K-groups per chunk (four MMA k-steps)
constexpr int kMaxN = kTileRows;              // rows of an item
constexpr int kDrain = 128 / (kGPC * kKG);    // chunks accumulated in tensor memory between drains (128 columns)
constexpr int kAccBufs = 4;                   // accumulator pairs in tensor memory (MMA runs up to 3 drains ahead)
constexpr uint32_t kTmemCols = 128 * kAccBufs; // each pair: main and correction, <= 64 columns each
constexpr int kThreads = 192;
constexpr int kTFlag = 1 << 30;               // K-group source: a row of T (else of X)

// a K-group's box: 3 planes x G column groups of 8 rows x 16 bytes
__host__ __device__ constexpr int box_bytes(int G) { return 3 * G * 128; }
__host__ __device__ constexpr int chunk_img_bytes(int rows8) { return 3 * kGPC * rows8 * kKG * 2; }
// A stage: the 4 boxes, then one chunk image of the launch's tallest item
// (r8max rows) and 128 bytes that the MMA may read past an image (N rounded
// up to 16), in 1 KiB units; as many stages as fit in kRingBytes.  The MMA
// reads M / 8 column groups of each plane, past the boxes' G when M > 8 G:
// at most 16 M - 128 G bytes past the boxes, inside the image region
// (16 M <= 128 G + 1536 for every M, G the launch can have).
constexpr int kMaxStages = 12;
constexpr int kRingBytes = 220 * 1024;
constexpr size_t kSmemBytes = (size_t)kRingBytes + 1024;
__host__ __device__ constexpr int stage_bytes(int G, int r8max) {
    return (kGPC * box_bytes(G) + chunk_img_bytes(r8max) + 128 + 1023) / 1024 * 1024;
}
__host__ __device__ constexpr int ring_stages(int G, int r8max) {
    return kRingBytes / stage_bytes(G, r8max) < kMaxStages ? kRingBytes / stage_bytes(G, r8max) : kMaxStages;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, no swizzle: lbo = stride of K-adjacent
// core matrices, sbo = stride of the 8-row (K-major) or 8-column (MN-major)
// groups
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;                                   // tcgen05 descriptor version
    return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

// x = x1 + x2 + x3 in BF16 pieces (round to nearest; each difference is
// exact in FP32)
__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
    a = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(a);
    b = __float2bfloat16_rn(r1);
    c = __float2bfloat16_rn(r1 - __bfloat162float(b));
}

// ---------------------------------------------------------------- packing
// K-groups of a tile's panel columns [0, K) with source rows idx[k]: column
// k starts one when it starts a run of consecutive source rows or lies a
// multiple of 8 columns into a run.  The warp walks 32 columns at a time
// (in column order, so the K-groups of a tile do not depend on who builds
// them) and calls f(k, idx[k], rank) for every start k, rank = number of
// starts before it; returns the number of K-groups.
template <class F>
__device__ __forceinline__ int kgroup_scan(const int* __restrict__ idx, int K, F&& f) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int prev = 0, rs = 0, count = 0;     // last source row and run start of the previous window
    for (int base = 0; base < K; base += 32) {
        const int k = base + lane;
        const bool valid = k < K;
        const int v = valid ? idx[k] : 0;
        int pv = __shfl_up_sync(full, v, 1);
        if (lane == 0) pv = prev;
        const bool brk = valid && (k == 0 || v != pv + 1);
        int r = brk ? k : -1;            // run start: last break at or before k
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(full, r, o);
            if (lane >= o) r = max(r, t);
        }
        r = max(r, rs);
        const bool st = valid && ((k - r) & 7) == 0;
        const unsigned m = __ballot_sync(full, st);
        if (st) f(k, v, count + __popc(m & ((1u << lane) - 1u)));
        count += __popc(m);
        prev = __shfl_sync(full, v, 31);
        rs = __shfl_sync(full, r, 31);
    }
    return count;
}

// K-groups of every row tile (dense panel, then U panel): one warp per tile
__global__ void __launch_bounds__(256) tc_count_kernel(const Tile* __restrict__ tiles, int nt,
                                                       const int* __restrict__ xidx, const int* __restrict__ tidx,
                                                       int* __restrict__ cnt) {
    const int t = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (t >= nt) return;
    const Tile tl = tiles[t];
    auto none = [](int, int, int) {};
    const int c = kgroup_scan(xidx + tl.ixn, tl.kn, none) + kgroup_scan(tidx + tl.ixf, tl.kf, none);
    if ((threadIdx.x & 31) == 0) cnt[t] = c;
}

// An item of the image build: its chunk images from byte img, its K-groups
// kgs[kg0 .. kg0 + nkg) of which the first nreal hold columns; panel
// segment 0 (a tile's dense panel, len0 columns, near pool at base0) and
// segment 1 (a tile's U panel or a far item's V^T slice, len1 columns,
// factor pool at base1), leading dimension ld; c0: a far item's first
// vector row.
struct PackItem {
    long long img, base0, base1;
    int kg0, nkg, nreal, rows, ld, len0, len1, far, c0, pad;
};

// What the pack needs of one K-group: its first panel element (pool
// offset), the byte offset of its image slot, the panel's leading dimension
// and rows, and its columns (valid, 0 for padding) and pool (seg: 0 dense
// panels, 1 factor panels).
struct KgDesc {
    long long src, dst;
    int ld, rows, valid, seg;
};

// K-group rows (and their first panel column, kcol) of the row tiles (one
// warp per tile) and of the far items (whose runs are their whole column
// cluster), padded with empty K-groups to whole chunks; then every K-group's
// pack descriptor
__global__ void __launch_bounds__(256) tc_kgroups_kernel(const Tile* __restrict__ tiles, int nt,
                                                         const int* __restrict__ xidx, const int* __restrict__ tidx,
                                                         const PackItem* __restrict__ pk, int n_items,
                                                         int* __restrict__ kgs, int* __restrict__ kcol,
                                                         KgDesc* __restrict__ desc) {
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= n_items) return;
    const int lane = threadIdx.x & 31;
    const PackItem it = pk[i];
    int* kg = kgs + it.kg0;
    int* kc = kcol + it.kg0;
    if (i < nt) {
        const Tile tl = tiles[i];
        const int c0 = kgroup_scan(xidx + tl.ixn, tl.kn, [&](int k, int v, int r) {
            kg[r] = v;
            kc[r] = k;
        });
        kgroup_scan(tidx + tl.ixf, tl.kf, [&](int k, int v, int r) {
            kg[c0 + r] = v | kTFlag;
            kc[c0 + r] = k;
        });
    } else {
        for (int j = lane; j < it.nreal; j += 32) {
            kg[j] = it.c0 + kKG * j;
            kc[j] = kKG * j;
        }
    }
    for (int j = it.nreal + lane; j < it.nkg; j += 32) {
        kg[j] = 0;
        kc[j] = 0;
    }
    __syncwarp();
    // columns of K-group j: up to the next K-group of the same panel, or the
    // panel's end
    const int rows8 = (it.rows + 7) & ~7;
    for (int j = lane; j < it.nkg; j += 32) {
        KgDesc d{0, it.img + (long long)(j / kGPC) * chunk_img_bytes(rows8) + (long long)(j % kGPC) * rows8 * kKG * 2,
                 it.ld, it.rows, 0, it.far};
        if (j < it.nreal) {
            const bool seg1 = it.far || (kg[j] & kTFlag);
            int next = seg1 ? it.len1 : it.len0;
            if (j + 1 < it.nreal && (it.far || (kg[j + 1] & kTFlag)) == seg1) next = kc[j + 1];
            d.valid = next - kc[j];
            d.seg = seg1 ? 1 : 0;
            d.src = (seg1 ? it.base1 : it.base0) + (long long)kc[j] * it.ld;
        }
        desc[it.kg0 + j] = d;
    }
}

// The three BF16 images of every chunk (one warp per chunk of kGPC
// K-groups, which all belong to one item): K-group j of an item in slot
// j % kGPC of chunk j / kGPC, [plane][slot][8-row group][8 rows][8
// columns], rows padded to rows8 and columns past the K-group with zeros.
// The chunk's descriptors are staged in shared memory; the lanes then take
// its (K-group, row) pairs, each splitting the row's 8 columns (reads
// coalesced across consecutive rows) and storing each plane's 16 bytes at
// once.
template <class FS>
__global__ void __launch_bounds__(256) tc_pack_kernel(const float* __restrict__ near_pool,
                                                      const FS* __restrict__ far_pool,
                                                      const KgDesc* __restrict__ desc, int n_kg,
                                                      unsigned char* __restrict__ img) {
    __shared__ KgDesc sd[8][kGPC];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nch = n_kg / kGPC;
    for (int ch = blockIdx.x * 8 + w; ch < nch; ch += gridDim.x * 8) {
        if (lane < kGPC) sd[w][lane] = desc[ch * kGPC + lane];
        __syncwarp();
        const int rows8 = (sd[w][0].rows + 7) & ~7;
        const long long pstride = (long long)kGPC * rows8 * kKG;    // elements of one plane of a chunk
        for (int q = lane; q < kGPC * rows8; q += 32) {
            const int j = q / rows8, n = q - j * rows8;
            const KgDesc d = sd[w][j];
            __nv_bfloat16* c = reinterpret_cast<__nv_bfloat16*>(img + d.dst);
            __align__(16) __nv_bfloat16 p1[kKG], p2[kKG], p3[kKG];
#pragma unroll
            for (int kk = 0; kk < kKG; ++kk) {
                float x = 0.0f;
                if (n < d.rows && kk < d.valid) {
                    const long long at = d.src + n + (long long)kk * d.ld;
                    x = d.seg ? (float)Store<FS>::get(far_pool[at]) : near_pool[at];
                }
                split3(x, p1[kk], p2[kk], p3[kk]);
            }
            const int o = (n >> 3) * 64 + (n & 7) * 8;
            *reinterpret_cast<uint4*>(c + o) = *reinterpret_cast<const uint4*>(p1);
            *reinterpret_cast<uint4*>(c + pstride + o) = *reinterpret_cast<const uint4*>(p2);
            *reinterpret_cast<uint4*>(c + 2 * pstride + o) = *reinterpret_cast<const uint4*>(p3);
        }
        __syncwarp();
    }
}

// vector rows -> three BF16 planes, group-major: element (row i, column
// 8 g + c) of plane p at ((p G + g) rows + i) 8 + c; zero past nc
__global__ void tc_split_rows_kernel(const float* __restrict__ X, int ldx, int rows, int nc, int G,
                                     __nv_bfloat16* __restrict__ P) {
    const long long plane = (long long)G * rows * kKG;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < plane;
         e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e & 7);
        const long long q = e >> 3;
        const int g = (int)(q / rows);
        const long long i = q - (long long)g * rows;
        const int col = 8 * g + c;
        const float x = col < nc ? X[i * ldx + col] : 0.0f;
        __nv_bfloat16 a, b, d;
        split3(x, a, b, d);
        P[e] = a;
        P[plane + e] = b;
        P[2 * plane + e] = d;
    }
}

// ---------------------------------------------------------------- GEMM
// A work item: its image chunks from byte img, its K-groups kgs[kg0 ..
// kg0 + nkg) (nkg a multiple of kGPC), its rows and first output row (the Y
// row of a tile, the T row of a far-field slice).
struct TcItem {
    long long img;
    int kg0, nkg, rows, orow, pad[2];
};

struct TcShared {
    unsigned long long full[kMaxStages], empty[kMaxStages], accf[kAccBufs], acce[kAccBufs];
    uint32_t tmem;
    int abort;
};

__device__ __forceinline__ uint32_t bar_addr(unsigned long long* b) { return smem_u32(b); }
__device__ __forceinline__ void mbar_init(unsigned long long* b, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_addr(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(bar_addr(b)) : "memory");
}
// blocking test of an mbarrier phase: the thread may be suspended in hardware
// for up to about 1 microsecond (the hint, in nanoseconds) instead of
// spinning
constexpr long kTryLimit = 1l << 22;   // tries (each returns within about a microsecond)
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(1000u)
        : "memory");
    return ok != 0;
}
// bounded wait that also gives up once another role has aborted
__device__ __forceinline__ bool role_wait(unsigned long long* b, uint32_t parity, volatile int* abort) {
    const uint32_t a = bar_addr(b);
    for (long it = 0; it < kTryLimit; ++it) {
        if (mbar_try_wait(a, parity)) return true;
        if ((it & 63) == 63 && *abort) return false;
    }
    atomicExch((int*)abort, 1);
    return false;
}
// bounded wait for a phase that completes whatever the other roles do (own
// copies or MMAs in flight), used on the way out
__device__ __forceinline__ void drain_wait(unsigned long long* b, uint32_t parity) {
    const uint32_t a = bar_addr(b);
    for (long it = 0; it < 4096; ++it)
        if (mbar_try_wait(a, parity)) return;
}

// the box of vector rows row .. row + 7: inner coordinate 8 row (elements;
// a multiple of 16 bytes), all column groups and planes
__device__ __forceinline__ void tma_box(unsigned char* dst, const CUtensorMap* tm, int row, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(kKG * row), "r"(0), "r"(0), "r"(bar)
        : "memory");
}

// Output of a launch: rows mode writes Y through the epilogue; far mode
// writes the three BF16 planes of T (group-major, G column groups, nT rows).
struct TcOut {
    void* Y;
    int ldy;
    Epi epi;
    __nv_bfloat16* T;
    int G;
    long long nT;
};

__global__ void __launch_bounds__(kThreads, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmt,
               const TcItem* __restrict__ items, int n_items, const int* __restrict__ kgs,
               const unsigned char* __restrict__ img, int M, int nc, int r8max, int rows_mode, TcOut out) {
    extern __shared__ __align__(1024) unsigned char dsm_raw[];
    __shared__ TcShared sh;
    unsigned char* dsm = dsm_raw + ((1024u - (smem_u32(dsm_raw) & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // boxes hold the G = ceil(nc / 8) column groups that carry data; the MMA
    // reads M / 8 groups per plane, the others (neighbouring data) only
    // reach rows of D past nc, which are never read
    const int G = (nc + 7) >> 3;
    const int S = ring_stages(G, r8max), sb = stage_bytes(G, r8max), bb = box_bytes(G);
    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&sh.full[i], 1);     // the producer's arrival with the expected bytes
            mbar_init(&sh.empty[i], 1);
        }
        for (int i = 0; i < kAccBufs; ++i) {
            mbar_init(&sh.accf[i], 1);
            mbar_init(&sh.acce[i], 128);
        }
        sh.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sh.tmem;
    volatile int* abort = &sh.abort;

    if (warp == 0) {
        // ------------------------------------------------ producer
        // lane 0 issues the copies; the warp loads the K-group rows of the
        // item's chunks 32 at a time, one batch of 32 ahead (lane j holds
        // chunk j's four rows), so that no copy waits on an index load
        int g = 0, pst = 0;          // chunks issued; stage of the next one
        uint32_t pph = 0;            // its use of the stage, mod 2
        bool ok = true;
        const int4 z4 = make_int4(0, 0, 0, 0);
        for (int i = blockIdx.x; i < n_items && ok; i += gridDim.x) {
            const TcItem itm = items[i];
            const int rows8 = (itm.rows + 7) & ~7;
            const int cb = chunk_img_bytes(rows8);
            const int nch = itm.nkg / kGPC;
            const unsigned char* src = img + itm.img;
            constexpr int Q = kGPC / 4;                  // int4 of K-group rows per chunk
            const int4* kq = reinterpret_cast<const int4*>(kgs + itm.kg0);
            int4 cur[Q], nxt[Q];
#pragma unroll
            for (int h = 0; h < Q; ++h) {
                cur[h] = lane < nch ? kq[Q * lane + h] : z4;
                nxt[h] = 32 + lane < nch ? kq[Q * (32 + lane) + h] : z4;
            }
            for (int c = 0; c < nch; ++c) {
                const int j = c & 31;
                if (j == 0 && c > 0) {
#pragma unroll
                    for (int h = 0; h < Q; ++h) {
                        cur[h] = nxt[h];
                        nxt[h] = c + 32 + lane < nch ? kq[Q * (c + 32 + lane) + h] : z4;
                    }
                }
                int r4[kGPC];
#pragma unroll
                for (int h = 0; h < Q; ++h) {
                    r4[4 * h] = __shfl_sync(0xffffffffu, cur[h].x, j);
                    r4[4 * h + 1] = __shfl_sync(0xffffffffu, cur[h].y, j);
                    r4[4 * h + 2] = __shfl_sync(0xffffffffu, cur[h].z, j);
                    r4[4 * h + 3] = __shfl_sync(0xffffffffu, cur[h].w, j);
                }
                if (lane == 0) {
                    if (g >= S && !role_wait(&sh.empty[pst], pph ^ 1u, abort)) {
                        ok = false;
                    } else {
                        unsigned char* stage = dsm + (size_t)pst * sb;
                        const uint32_t fb = bar_addr(&sh.full[pst]);
                        asm volatile(
                            "{\n\t.reg .b64 tk;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 tk, [%0], %1;\n\t}\n" ::"r"(fb),
                            "r"(kGPC * bb + cb)
                            : "memory");
#pragma unroll
                        for (int q = 0; q < kGPC; ++q)
                            tma_box(stage + q * bb, (r4[q] & kTFlag) ? &tmt : &tmx, r4[q] & (kTFlag - 1), fb);
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                                smem_u32(stage + kGPC * bb)),
                            "l"(src + (size_t)c * cb), "r"(cb), "r"(fb)
                            : "memory");
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) break;
                ++g;
                if (++pst == S) {
                    pst = 0;
                    pph ^= 1u;
                }
            }
        }
        // copies still in flight (an aborted run): wait for them, bounded
        if (lane == 0)
            for (int q = g > S ? g - S : 0; q < g; ++q) drain_wait(&sh.full[q % S], (uint32_t)((q / S) & 1));
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            // kind::f16: FP32 D, BF16 A and B, A MN-major (bit 15), B K-major
            const uint32_t ibase = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | ((uint32_t)(M >> 4) << 24);
            const uint32_t dsm_a = smem_u32(dsm);
            // descriptors are built once per item and stepped by adding
            // 16-byte address units (shared addresses stay below 256 KiB, so
            // the 14-bit start field never carries); stage and phase advance
            // by counters
            const uint64_t sstep = (uint64_t)(sb >> 4);
            int st = 0, grp = 0, last_st = -1;
            uint32_t ph = 0, last_ph = 0;
            uint64_t soff = 0;
            bool ok = true;
            TcItem nitm = blockIdx.x < n_items ? items[blockIdx.x] : TcItem{};
            for (int i = blockIdx.x; i < n_items && ok; i += gridDim.x) {
                const TcItem itm = nitm;
                if (i + (int)gridDim.x < n_items) nitm = items[i + gridDim.x];   // one item ahead
                const int rows8 = (itm.rows + 7) & ~7;
                const int N = M > 64 ? (itm.rows + 15) & ~15 : rows8;
                const uint32_t idesc = ibase | ((uint32_t)(N >> 3) << 17);
                const int nch = itm.nkg / kGPC;
                const uint32_t pstride = (uint32_t)(kGPC * rows8 * kKG * 2);   // bytes of one image plane
                // A: plane p of K-groups 2 ks, 2 ks + 1 (boxes bb bytes apart,
                // column groups 128 bytes apart, planes 128 G apart); B: plane
                // p of the image (K-groups rows8 x 16 bytes apart, 8-row groups
                // 128 apart, planes pstride apart)
                const uint64_t adesc = smem_desc(dsm_a, bb, 128);
                const uint64_t bdesc = smem_desc(dsm_a + (uint32_t)(kGPC * bb), rows8 * 16, 128);
                const uint64_t ap = (uint64_t)(8 * G), aks = (uint64_t)((2 * bb) >> 4);
                const uint64_t bp = (uint64_t)(pstride >> 4), bks = (uint64_t)(2 * rows8);
                int cd = 0;                                    // chunk within the drain group
                for (int c = 0; c < nch; ++c) {
                    const int buf = grp % kAccBufs;
                    if (cd == 0 && grp >= kAccBufs) {
                        ok = role_wait(&sh.acce[buf], (uint32_t)((grp / kAccBufs - 1) & 1), abort);
                        if (!ok) break;
                    }
                    ok = role_wait(&sh.full[st], ph, abort);
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t dm = tmem + (uint32_t)(128 * buf), dc = dm + 64;
                    uint64_t a1 = adesc + soff, b1 = bdesc + soff;
#pragma unroll
                    for (int ks = 0; ks < kGPC / 2; ++ks) {
                        const uint32_t acc = (cd == 0 && ks == 0) ? 0u : 1u;
                        const uint64_t a2 = a1 + ap, a3 = a2 + ap, b2 = b1 + bp, b3 = b2 + bp;
                        mma_bf16(dm, a1, b1, idesc, acc);
                        mma_bf16(dc, a1, b2, idesc, acc);
                        mma_bf16(dc, a2, b1, idesc, 1u);
                        mma_bf16(dc, a1, b3, idesc, 1u);
                        mma_bf16(dc, a2, b2, idesc, 1u);
                        mma_bf16(dc, a3, b1, idesc, 1u);
                        a1 += aks;
                        b1 += bks;
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     bar_addr(&sh.empty[st]))
                                 : "memory");
                    last_st = st;
                    last_ph = ph;
                    if (++cd == kDrain || c == nch - 1) {
                        asm volatile(
                            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                bar_addr(&sh.accf[buf]))
                            : "memory");
                        ++grp;
                        cd = 0;
                    }
                    soff += sstep;
                    if (++st == S) {
                        st = 0;
                        ph ^= 1u;
                        soff = 0;
                    }
                }
            }
            // MMAs still in flight (an aborted run): the last commit
            if (last_st >= 0) drain_wait(&sh.empty[last_st], last_ph);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ drainers and epilogue
        // lane quarter q holds D rows 32 q .. 32 q + 31 for M = 128, rows
        // 16 q .. 16 q + 15 (in lanes 0-15) for M = 64; D row = column m
        const int q = warp & 3;
        const int m = M > 64 ? 32 * q + lane : (lane < 16 ? 16 * q + lane : nc);
        const bool live = (M > 64 ? 32 * q : 16 * q) < nc;   // warp-uniform
        const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16);
        int grp = 0;
        bool ok = true;
        TcItem nitm = blockIdx.x < n_items ? items[blockIdx.x] : TcItem{};
        for (int i = blockIdx.x; i < n_items && ok; i += gridDim.x) {
            const TcItem itm = nitm;
            if (i + (int)gridDim.x < n_items) nitm = items[i + gridDim.x];   // one item ahead
            const int rows8 = (itm.rows + 7) & ~7;
            const int N = M > 64 ? (itm.rows + 15) & ~15 : rows8;
            const int nch = itm.nkg / kGPC;
            float racc[kMaxN];
#pragma unroll
            for (int n = 0; n < kMaxN; ++n) racc[n] = 0.0f;
            const int ngr = (nch + kDrain - 1) / kDrain;
            for (int gg = 0; gg < ngr; ++gg, ++grp) {
                const int buf = grp % kAccBufs;
                ok = role_wait(&sh.accf[buf], (uint32_t)((grp / kAccBufs) & 1), abort);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (live) {
#pragma unroll
                    for (int c16 = 0; c16 < kMaxN / 16; ++c16) {
                        if (16 * c16 >= N) break;
                        uint32_t r[32];
                        const uint32_t ad = lane_addr + (uint32_t)(128 * buf + 16 * c16);
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                            "[%16];"
                            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                              "=r"(r[14]), "=r"(r[15])
                            : "r"(ad));
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                            "[%16];"
                            : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                              "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                            : "r"(ad + 64));
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            racc[16 * c16 + j] += __uint_as_float(r[j]) + __uint_as_float(r[16 + j]);
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(&sh.acce[buf]);
            }
            // one outcome for all four drainer warps (named barrier 1)
            uint32_t all_ok;
            asm volatile(
                "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
                "bar.red.and.pred q, 1, 128, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
                : "=r"(all_ok)
                : "r"((uint32_t)ok)
                : "memory");
            ok = all_ok != 0;
            if (!ok) break;
            if (m < nc) {
                if (rows_mode && out.epi.mode == kStore) {
                    float* Y = static_cast<float*>(out.Y) + (long long)itm.orow * out.ldy + m;
#pragma unroll
                    for (int n = 0; n < kMaxN; ++n)
                        if (n < itm.rows) Y[(long long)n * out.ldy] = racc[n];
                } else if (rows_mode) {
                    // FP64 epilogue (Eq. 11 products): the inputs of 16 rows are
                    // loaded (read-only path) before any of their results is
                    // stored, so the loads overlap instead of alternating with
                    // the stores
                    const Epi& e = out.epi;
                    const bool resid = e.mode == kResid;
#pragma unroll
                    for (int n0 = 0; n0 < kMaxN; n0 += 16) {
                        if (n0 >= itm.rows) break;
                        double ev[16], xv[16], bv[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int row = itm.orow + n0 + j;
                            const bool in = n0 + j < itm.rows;
                            ev[j] = in ? __ldg(e.eps + row) : 0.0;
                            xv[j] = in ? __ldg(e.xin + (long long)row * e.ld64 + m) : 0.0;
                            bv[j] = in && resid ? __ldg(e.b + (long long)row * e.ld64 + m) : 0.0;
                        }
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            if (n0 + j >= itm.rows) continue;
                            double w = xv[j] - (1.0 - ev[j]) * (double)racc[n0 + j];
                            if (resid) w = bv[j] - w;
                            static_cast<double*>(out.Y)[(long long)(itm.orow + n0 + j) * out.ldy + m] = w;
                        }
                    }
                } else {
                    const long long plane = (long long)out.G * out.nT * kKG;
                    __nv_bfloat16* t0 = out.T + ((long long)(m >> 3) * out.nT + itm.orow) * kKG + (m & 7);
#pragma unroll
                    for (int n = 0; n < kMaxN; ++n) {
                        if (n < itm.rows) {
                            __nv_bfloat16 a, b, d;
                            split3(racc[n], a, b, d);
                            t0[n * kKG] = a;
                            t0[plane + n * kKG] = b;
                            t0[2 * plane + n * kKG] = d;
                        }
                    }
                }
            }
        }
    }
    if (tid == 0 && *abort) atomicExch(&g_tc_timeout, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

inline size_t align256(size_t b) { return (b + 255) / 256 * 256; }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        (void)cudaGetLastError();
    });
    RAD_REQUIRE(fn != nullptr, RAD_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    return fn;
}

// Tensor map over three group-major BF16 planes of `rows` rows and G column
// groups, seen as 3-D: (rows x 8 elements of a column group, G groups, 3
// planes), so that 8 consecutive rows of a group are one contiguous 128-byte
// line of the box (one core matrix).  Box = 64 elements x G groups x 3
// planes; rows past `rows` read as zeros.
void encode_planes(CUtensorMap* tm, const __nv_bfloat16* base, long long rows, int G) {
    const cuuint64_t dims[3] = {(cuuint64_t)rows * kKG, (cuuint64_t)G, 3};
    const cuuint64_t strides[2] = {(cuuint64_t)rows * 16, (cuuint64_t)rows * 16 * G};
    const cuuint32_t box[3] = {(cuuint32_t)(kKG * kKG), (cuuint32_t)G, 3};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUresult r = encode_fn()(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(base), dims,
                                   strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    RAD_REQUIRE(r == CUDA_SUCCESS, RAD_ECUDA, "tensor map encoding failed");
}

}  // namespace

// ---------------------------------------------------------------- host side
bool tc_supported(const rad_htree* h) { return h->compressed && !h->op_is_f64() && !h->from_dense; }

void tc_drop_images(rad_htree* h, cudaStream_t s) {
    h->tc_maps.ws = nullptr;
    h->tc_img.release(s);
    h->tc_rows_items.release(s);
    h->tc_far_items.release(s);
    h->tc_kgs.release(s);
    h->tc_n_rows = h->tc_n_far = 0;
    h->tc_ready = false;
}

// The K-groups and chunk images of every work item (row tiles and far-field
// slices) for the tensor-core path: the tiles' K-group counts on the device
// (one read back), the layout on the host, K-groups and images on the device.
void tc_build_images(rad_htree* h, cudaStream_t s) {
    RAD_REQUIRE(tc_supported(h), RAD_EINVAL, "tensor-core products need an FP32 or BF16 operator");
    if (h->tc_ready) return;
    HostScope hs_("host_tc_build");
    const int nt = h->n_tiles, nw = h->n_gwork;
    Scratch ws(s);
    // per-tile K-group counts and the far items: kept with the operator by
    // rad_compress_aca, else (a loaded checkpoint) read back here
    if ((int)h->tc_cnt_h.size() != nt) {
        tc_count_async(h, s);
        RAD_CUDA(cudaStreamSynchronize(s));
    }
    if ((int)h->gwork_h.size() != nw) {
        h->gwork_h.resize(nw);
        if (nw > 0)
            RAD_CUDA(cudaMemcpyAsync(h->gwork_h.data(), h->d_gwork.p, sizeof(GWork) * nw, cudaMemcpyDeviceToHost, s));
        RAD_CUDA(cudaStreamSynchronize(s));
    }
    const std::vector<int>& cnt = h->tc_cnt_h;
    const std::vector<GWork>& gw = h->gwork_h;
    std::vector<PackItem> pk;
    pk.reserve((size_t)nt + nw);
    std::vector<TcItem> rows_items, far_items;
    long long img = 0;
    int kg = 0;
    auto add = [&](PackItem p, int orow, std::vector<TcItem>& list) {
        const int rows8 = (p.rows + 7) & ~7;
        p.nkg = (p.nreal + kGPC - 1) / kGPC * kGPC;
        p.kg0 = kg;
        p.img = img;
        pk.push_back(p);
        list.push_back(TcItem{img, kg, p.nkg, p.rows, orow, {0, 0}});
        kg += p.nkg;
        img += (long long)(p.nkg / kGPC) * chunk_img_bytes(rows8);
    };
    for (int t = 0; t < nt; ++t) {
        const Tile& tl = h->tiles_h[t];
        add(PackItem{0, tl.noff, tl.foff, 0, 0, cnt[t], tl.rows, tl.ld, tl.kn, tl.kf, 0, 0, 0}, tl.r0, rows_items);
    }
    for (int w = 0; w < nw; ++w) {
        const Group& g = h->groups_h[gw[w].g];
        add(PackItem{0, 0, g.voff + gw[w].r0, 0, 0, (g.n + kKG - 1) / kKG, gw[w].rows, g.ld, 0, g.n, 1, g.c0, 0},
            g.toff + gw[w].r0, far_items);
    }
    // the launch order: heaviest first
    auto heavy = [](const TcItem& a, const TcItem& b) {
        return (long long)a.nkg * ((a.rows + 7) & ~7) > (long long)b.nkg * ((b.rows + 7) & ~7);
    };
    std::stable_sort(rows_items.begin(), rows_items.end(), heavy);
    std::stable_sort(far_items.begin(), far_items.end(), heavy);

    h->tc_img.alloc((size_t)std::max<long long>(img, 16), s);
    h->tc_rows_items.alloc(sizeof(TcItem) * std::max<size_t>(1, rows_items.size()), s);
    h->tc_far_items.alloc(sizeof(TcItem) * std::max<size_t>(1, far_items.size()), s);
    h->tc_kgs.alloc(sizeof(int) * (size_t)std::max(kGPC, kg), s);
    if (!rows_items.empty())
        RAD_CUDA(cudaMemcpyAsync(h->tc_rows_items.p, rows_items.data(), sizeof(TcItem) * rows_items.size(),
                                 cudaMemcpyHostToDevice, s));
    if (!far_items.empty())
        RAD_CUDA(cudaMemcpyAsync(h->tc_far_items.p, far_items.data(), sizeof(TcItem) * far_items.size(),
                                 cudaMemcpyHostToDevice, s));
    if (!pk.empty()) {
        PackItem* d_pk = ws.get_n<PackItem>(pk.size());
        int* d_kcol = ws.get_n<int>((size_t)std::max(kGPC, kg));
        KgDesc* d_desc = ws.get_n<KgDesc>((size_t)std::max(kGPC, kg));
        RAD_CUDA(cudaMemcpyAsync(d_pk, pk.data(), sizeof(PackItem) * pk.size(), cudaMemcpyHostToDevice, s));
        ProfScope ps_("tc_pack", s);
        const int ni = (int)pk.size();
        tc_kgroups_kernel<<<(unsigned)((ni + 7) / 8), 256, 0, s>>>(h->d_tiles.as<Tile>(), nt, h->d_xidx.as<int>(),
                                                                   h->d_tidx.as<int>(), d_pk, ni,
                                                                   h->tc_kgs.as<int>(), d_kcol, d_desc);
        RAD_CHECK_LAUNCH();
        static int sms = 0;
        static std::once_flag once;
        std::call_once(once, [] {
            int dev = 0;
            RAD_CUDA(cudaGetDevice(&dev));
            RAD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        });
        const unsigned grid = (unsigned)std::min<long long>((kg / kGPC + 7) / 8, 16ll * sms);
        if (kg > 0) {
            if (h->factor_dtype == RAD_F32)
                tc_pack_kernel<float><<<grid, 256, 0, s>>>(h->near_pool.as<float>(), h->far_pool.as<float>(), d_desc,
                                                           kg, h->tc_img.as<unsigned char>());
            else
                tc_pack_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(h->near_pool.as<float>(),
                                                                   h->far_pool.as<__nv_bfloat16>(), d_desc, kg,
                                                                   h->tc_img.as<unsigned char>());
            RAD_CHECK_LAUNCH();
        }
    }
    h->tc_n_rows = (int)rows_items.size();
    h->tc_n_far = (int)far_items.size();
    h->tc_r8max = 8;
    for (const auto* v : {&rows_items, &far_items})
        for (const TcItem& it : *v) h->tc_r8max = std::max(h->tc_r8max, (it.rows + 7) & ~7);
    h->tc_ready = true;
}

// K-groups per row tile into h->tc_cnt_h (complete at the stream's next
// synchronisation)
void tc_count_async(rad_htree* h, cudaStream_t s) {
    const int nt = h->n_tiles;
    h->tc_cnt_h.assign(nt, 0);
    if (nt == 0) return;
    Scratch ws(s);
    int* d_cnt = ws.get_n<int>(nt);
    tc_count_kernel<<<(unsigned)((nt + 7) / 8), 256, 0, s>>>(h->d_tiles.as<Tile>(), nt, h->d_xidx.as<int>(),
                                                             h->d_tidx.as<int>(), d_cnt);
    RAD_CHECK_LAUNCH();
    RAD_CUDA(cudaMemcpyAsync(h->tc_cnt_h.data(), d_cnt, sizeof(int) * nt, cudaMemcpyDeviceToHost, s));
}

// Builds the tensor-core images on first use: the product path is the
// tensor cores and a product of ncols >= 5 columns is coming.  The build
// synchronises the stream, so it is skipped while the stream is being
// captured into a graph (that product then runs on the CUDA-core tiles).
void tc_prepare(const rad_htree* hc, int ncols, cudaStream_t s) {
    rad_htree* h = const_cast<rad_htree*>(hc);
    if (ncols < 5 || h->mm_path != 1 || h->tc_ready || !tc_supported(h)) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    if (cs != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> lk(h->tc_mu);
    if (!h->tc_ready) tc_build_images(h, s);
}

// Workspace of one tensor-core product of up to 96 columns: the split
// planes of X (n rows) and of T (sum_rank rows), G = ceil(columns / 8)
// column groups each.
size_t tc_workspace_bytes(const rad_htree* h, int nrhs) {
    const int G = (std::min(96, nrhs) + 7) / 8;
    return align256((size_t)3 * h->n * G * kKG * 2) + align256((size_t)3 * std::max(1, h->sum_rank) * G * kKG * 2) + 256;
}

// Y = F X for nc <= 96 FP32 columns (rows of X at stride ldx), epilogue as
// in apply_tree; ws holds tc_workspace_bytes(h, nc) bytes.
void tc_product(const rad_htree* h, const OpView& op, const float* X, int ldx, void* Y, int ldy, int nc,
                const Epi& epi, void* ws, cudaStream_t s) {
    RAD_REQUIRE(h->tc_ready, RAD_EINVAL, "tensor-core images missing (select the path first)");
    RAD_REQUIRE(nc >= 1 && nc <= 96, RAD_EINVAL, "tensor-core product: 1 to 96 columns per launch");
    const int G = (nc + 7) / 8;
    const int M = nc <= 64 ? 64 : 128;
    const int n = (int)h->n;
    const long long nT = std::max(1, op.sum_rank);
    unsigned char* base = reinterpret_cast<unsigned char*>(align256(reinterpret_cast<uintptr_t>(ws)));
    __nv_bfloat16* Xs = reinterpret_cast<__nv_bfloat16*>(base);
    __nv_bfloat16* Ts = reinterpret_cast<__nv_bfloat16*>(base + align256((size_t)3 * n * G * kKG * 2));
    static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
    CUtensorMap tmx, tmt;
    {
        // encoding is a driver call: reuse the last maps of this handle when
        // the workspace and the column groups are the same
        rad_htree* hm = const_cast<rad_htree*>(h);
        std::lock_guard<std::mutex> lk(hm->tc_mu);
        if (hm->tc_maps.ws != ws || hm->tc_maps.G != G) {
            encode_planes(&tmx, Xs, n, G);
            encode_planes(&tmt, Ts, nT, G);
            std::memcpy(hm->tc_maps.map[0], &tmx, 128);
            std::memcpy(hm->tc_maps.map[1], &tmt, 128);
            hm->tc_maps.ws = ws;
            hm->tc_maps.G = G;
        } else {
            std::memcpy(&tmx, hm->tc_maps.map[0], 128);
            std::memcpy(&tmt, hm->tc_maps.map[1], 128);
        }
    }
    static std::once_flag configured;
    static int sms = 0;
    std::call_once(configured, [&] {
        RAD_CUDA(cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
        int dev = 0;
        RAD_CUDA(cudaGetDevice(&dev));
        RAD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    });
    const int r8max = h->tc_r8max;
    const size_t smem = (size_t)ring_stages(G, r8max) * stage_bytes(G, r8max) + 1024;
    {
        ProfScope ps_("tc_split", s);
        const long long tot = (long long)G * n * kKG;
        tc_split_rows_kernel<<<(unsigned)std::min<long long>((tot + 255) / 256, 4096), 256, 0, s>>>(X, ldx, n, nc, G, Xs);
    }
    RAD_CHECK_LAUNCH();
    const unsigned char* img = h->tc_img.as<unsigned char>();
    const int* kgs = h->tc_kgs.as<int>();
    if (h->tc_n_far > 0) {
        TcOut o{nullptr, 0, epi, Ts, G, nT};
        ProfScope ps_("hmm_far_vt", s);
        tc_gemm_kernel<<<std::min(h->tc_n_far, sms), kThreads, smem, s>>>(
            tmx, tmt, h->tc_far_items.as<TcItem>(), h->tc_n_far, kgs, img, M, nc, r8max, 0, o);
        RAD_CHECK_LAUNCH();
    }
    {
        TcOut o{Y, ldy, epi, nullptr, G, nT};
        ProfScope ps_("hmm_rows", s);
        tc_gemm_kernel<<<std::min(h->tc_n_rows, sms), kThreads, smem, s>>>(
            tmx, tmt, h->tc_rows_items.as<TcItem>(), h->tc_n_rows, kgs, img, M, nc, r8max, 1, o);
    }
    RAD_CHECK_LAUNCH();
}

// Reads and clears the timeout flag of the tensor-core kernels.
bool tc_take_timeout() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_timeout, sizeof(int)) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_tc_timeout, &z, sizeof(int));
    }
    return v != 0;
}

}  // namespace rad
