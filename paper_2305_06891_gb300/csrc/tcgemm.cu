// Tensor-core (tcgen05) panel GEMMs of the many-column product, FP32
// operands at FP32-level accuracy.
//
// A panel times gathered vector rows, D[64 x N] += A[64 x K] B[K x N], runs
// on the 5th-generation tensor cores (kind::f16 with BF16 operands, FP32
// accumulators in tensor memory).  BF16 keeps 8 mantissa bits, so every
// FP32 operand x is split into three BF16 pieces, x1 = bf16(x),
// x2 = bf16(x - x1), x3 = bf16(x - x1 - x2), which together carry its 24
// bits; the product takes the six terms a1 b1 (the "main" accumulator) and
// a1 b2 + a2 b1 + a1 b3 + a2 b2 + a3 b1 (a second, "correction" accumulator),
// dropping terms of order 2^-24 relative.  The tensor core's accumulation
// truncates, so the accumulators start from zero every 128 panel columns
// and are added into FP32 registers (round to nearest): the rounding stays
// at the level of an FP32 FFMA loop (measured below it).
//
// The split is never done inside the kernel:
//   - panels (dense blocks, U and V^T factors) are split once, when the path
//     is selected, into three 64 x 32 BF16 images per chunk of 32 panel
//     columns, laid out as the MMA reads them (K-major core matrices of
//     8 rows x 16 bytes, no swizzle: 8-row groups 512 bytes apart, K-adjacent
//     cores 128 bytes apart), zero-padded past the panel's rows and columns;
//   - vector rows (X, and T = V^T X) are split once per product into three
//     BF16 planes of N8 = 8 ceil(nc / 8) columns; a gathered row lands in
//     shared memory by 16-byte copies as MN-major core matrices (8 columns x
//     8 rows of 16 bytes; 8-column groups 512 bytes apart, K-adjacent cores
//     128 bytes apart), which the MMA reads with the B-transpose bit set.
// Persistent, warp-specialised kernel (one CTA of 256 threads per SM,
// items taken round-robin, heaviest first): warps 0-2 copy chunks (12 KiB of
// panel images by one bulk copy, 3 x N8 x 32 x 2 bytes of gathered vector
// rows by 16-byte copies) into a ring of six shared-memory stages; one thread of warp 3 issues every chunk's 2
// k-steps x 6 MMAs (M = 64, K = 16) into one of two accumulator pairs in
// tensor memory; warps 4-7 (whose tensor-memory lane quarters hold rows
// 16 q .. 16 q + 15 in lanes 0-15) add a pair into FP32 registers after
// every 4 chunks of an item and write the item's rows at its end.  The roles
// hand over through mbarriers (stage full / empty, accumulators full /
// empty) and never wait for the whole CTA.  Every wait is bounded: after
// a bounded number of tries a role raises an abort flag that the others see, the CTA
// records the timeout in a device flag (checked by the host at its next
// synchronisation) and frees its tensor memory.

#include <cstdint>
#include <mutex>

#include "rad_device.cuh"

namespace rad {

__device__ int g_tc_timeout = 0;

namespace {

constexpr int kKC = 32;                          // panel columns per chunk
constexpr int kImg = kTileRows * kKC * 2;        // one BF16 image of a chunk: 4 KiB
constexpr int kChunkBytes = 3 * kImg;            // the three split images
constexpr int kGrp = (kKC / 8) * 128;            // 512: 8-row / 8-column group stride
constexpr uint32_t kCorrCol = 128;               // correction accumulator: 128 columns after the main one
constexpr int kMaxN8 = 96;

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
// One chunk of a panel: rows [0, rows) and columns [k0, k0 + 32) of the
// column-major panel at pool + src (leading dimension ld, K columns in all).
struct PackJob {
    long long src;
    int ld, rows, k0, K;
    long long chunk;
};
template <class FS>
__global__ void __launch_bounds__(256) tc_pack_kernel(const FS* __restrict__ pool, const PackJob* __restrict__ jobs,
                                                      unsigned char* __restrict__ img) {
    const PackJob j = jobs[blockIdx.x];
    unsigned char* dst = img + j.chunk * kChunkBytes;
    for (int e = threadIdx.x; e < kTileRows * kKC; e += blockDim.x) {
        const int m = e % kTileRows, k = e / kTileRows;
        float x = 0.0f;
        if (m < j.rows && j.k0 + k < j.K) x = (float)Store<FS>::get(pool[j.src + m + (long long)(j.k0 + k) * j.ld]);
        __nv_bfloat16 a, b, c;
        split3(x, a, b, c);
        const int off = (m >> 3) * kGrp + (k >> 3) * 128 + (m & 7) * 16 + (k & 7) * 2;
        *reinterpret_cast<__nv_bfloat16*>(dst + off) = a;
        *reinterpret_cast<__nv_bfloat16*>(dst + kImg + off) = b;
        *reinterpret_cast<__nv_bfloat16*>(dst + 2 * kImg + off) = c;
    }
}

// vector rows -> three BF16 planes of N8 columns (zero past nc)
__global__ void tc_split_rows_kernel(const float* __restrict__ X, int ldx, int rows, int nc, int N8,
                                     __nv_bfloat16* __restrict__ P, long long plane) {
    const long long total = (long long)rows * N8;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / N8;
        const int c = (int)(e - i * N8);
        const float x = c < nc ? X[i * ldx + c] : 0.0f;
        __nv_bfloat16 a, b, d;
        split3(x, a, b, d);
        P[e] = a;
        P[plane + e] = b;
        P[2 * plane + e] = d;
    }
}

// ---------------------------------------------------------------- GEMM
__device__ __forceinline__ void cp16(void* sdst, const void* gsrc, bool pred) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(sdst)), "l"(gsrc),
                 "r"(pred ? 16 : 0));
}

// One K segment of a work item: nch chunk images from img, and the vector
// rows idx[k] (or base + k) of three BF16 planes (plane elements apart, N8
// columns) for k < K.
struct Seg {
    const unsigned char* img;
    int nch, K;
    const __nv_bfloat16* B;
    long long plane;
    const int* idx;
    int base;
};

__host__ __device__ constexpr int b_plane_bytes(int N8) { return (N8 / 8) * kGrp; }
__host__ __device__ constexpr int stage_bytes(int N8) { return kChunkBytes + 3 * b_plane_bytes(N8); }

constexpr int kProducers = 96;     // warps 0-2 copy chunks into the stage ring
constexpr int kMmaWarp = 3;        // lane 0 issues the MMAs
constexpr int kDrainers = 128;     // warps 4-7 read the accumulators (lane quarters 0-3)
constexpr int kDrain = 4;          // chunks accumulated in tensor memory between drains
constexpr int kRingStages = 6;     // chunks in flight
constexpr int kMaxBlkAll = kMaxN8 / 8;

// chunk c of a segment into a stage, by producer thread pt (0 .. 95): the
// three panel images (12 KiB, contiguous) by one bulk copy that completes
// on the stage's "full" mbarrier, the gathered vector rows by 16-byte
// copies
__device__ __forceinline__ void issue_chunk(const Seg& sg, int c, int N8, unsigned char* st, int pt, uint32_t full) {
    if (pt == 0) {
        const unsigned char* a = sg.img + (size_t)c * kChunkBytes;
        asm volatile("{\n\t.reg .b64 tk;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 tk, [%0], %1;\n\t}\n" ::"r"(full),
                     "r"(kChunkBytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                smem_u32(st)),
            "l"(a), "r"(kChunkBytes), "r"(full)
            : "memory");
    }
    // warp w copies plane w: the chunk's 32 row indices are read once per
    // warp (one coalesced load, lane k holding row k) and handed out by
    // shuffles, so the copies do not wait on dependent index loads
    unsigned char* b = st + kChunkBytes + (pt >> 5) * b_plane_bytes(N8);
    const int lane = pt & 31, q = pt >> 5;
    const int nj = N8 / 8;
    const int k0 = c * kKC;
    const bool okl = k0 + lane < sg.K;
    const int myrow = okl ? (sg.idx ? sg.idx[k0 + lane] : sg.base + k0 + lane) : 0;
    const __nv_bfloat16* plane = sg.B + q * sg.plane;
    for (int it = 0; it < nj; ++it) {
        const int r = it * 32 + lane;               // copy r of this plane: row k, 16-byte piece j
        const int k = r / nj, j = r - k * nj;
        const int row = __shfl_sync(0xffffffffu, myrow, k);
        const bool ok = k0 + k < sg.K;
        const __nv_bfloat16* src = ok ? plane + (long long)row * N8 + 8 * j : sg.B;
        cp16(b + j * kGrp + (k >> 3) * 128 + (k & 7) * 16, src, ok);
    }
}

struct TcShared {
    unsigned long long full[kRingStages], empty[kRingStages], accf[2], acce[2];
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
// spinning, which keeps shared memory free for the copies being waited for
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

// The work items of one launch: tiles (rows) or far-field items (far_vt).
struct Items {
    bool rows;
    OpView op;
    const long long* first;    // rows: tile_near0; far_vt: item0
    const long long* first2;   // rows: tile_far0
    const unsigned char* img;
    const __nv_bfloat16 *Xs, *Ts;
    long long xplane, tplane;
    __device__ __forceinline__ int count() const { return rows ? op.n_tiles : op.n_gwork; }
    // the two segments of item i (the second is empty for far-field items)
    __device__ __forceinline__ void segs(int i, Seg& s0, Seg& s1) const {
        if (rows) {
            const int ti = op.torder[i];
            const Tile t = op.tiles[ti];
            s0 = Seg{img + first[ti] * (long long)kChunkBytes, (t.kn + kKC - 1) / kKC, t.kn, Xs, xplane,
                     op.xidx + t.ixn, 0};
            s1 = Seg{img + first2[ti] * (long long)kChunkBytes, (t.kf + kKC - 1) / kKC, t.kf, Ts, tplane,
                     op.tidx + t.ixf, 0};
        } else {
            const GWork w = op.gwork[i];
            const Group gr = op.groups[w.g];
            s0 = Seg{img + first[i] * (long long)kChunkBytes, (gr.n + kKC - 1) / kKC, gr.n, Xs, xplane, nullptr,
                     gr.c0};
            s1 = Seg{nullptr, 0, 0, nullptr, 0, nullptr, 0};
        }
    }
};

__device__ __forceinline__ void epilogue_tc(const Epi& epi, void* Y, int ldy, int row, int col, float acc) {
    if (epi.mode == kStore) {
        static_cast<float*>(Y)[(long long)row * ldy + col] = acc;
    } else {
        const double e = epi.eps[row];
        double w = epi.xin[(long long)row * epi.ld64 + col] - (1.0 - e) * (double)acc;
        if (epi.mode == kResid) w = epi.b[(long long)row * epi.ld64 + col] - w;
        static_cast<double*>(Y)[(long long)row * ldy + col] = w;
    }
}

// Persistent, warp-specialised panel GEMM: CTA b takes items b, b + grid,
// ... (heaviest first).  Producers fill a ring of kRingStages chunk stages
// (cp.async, arriving on the stage's "full" mbarrier when the copies land);
// the MMA thread waits "full", issues the chunk's 12 MMAs into one of two
// tensor-memory accumulator pairs and commits them to the stage's "empty"
// mbarrier (the producers' licence to refill it); after every kDrain chunks
// of an item (and at its end) it commits the pair to "acc full"; the
// drainers add the pair to FP32 registers, release it ("acc empty") and,
// at the end of an item, write its rows.
__global__ void __launch_bounds__(256, 1) tc_gemm_kernel(Items it, int nc, int N8, void* Y, int ldy, Epi epi,
                                                          __nv_bfloat16* Tout, long long tplane_out) {
    extern __shared__ __align__(1024) unsigned char dsm[];
    __shared__ TcShared sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int sb = stage_bytes(N8);
    if (tid == 0) {
        for (int i = 0; i < kRingStages; ++i) {
            mbar_init(&sh.full[i], kProducers + 1);   // 96 copy arrivals + the bulk copy's expect_tx
            mbar_init(&sh.empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&sh.accf[i], 1);
            mbar_init(&sh.acce[i], kDrainers);
        }
        sh.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sh.tmem;
    volatile int* abort = &sh.abort;
    const int n_items = it.count();

    if (warp < kProducers / 32) {
        // ------------------------------------------------ producers
        int g = 0;   // global chunk counter of this CTA
        for (int i = blockIdx.x; i < n_items && !*abort; i += gridDim.x) {
            Seg s0, s1;
            it.segs(i, s0, s1);
            const int nch = s0.nch + s1.nch;
            for (int c = 0; c < nch; ++c, ++g) {
                const int st = g % kRingStages, use = g / kRingStages;
                if (use > 0) {
                    // warp-uniform outcome: the copies below shuffle across the warp
                    const bool w = __all_sync(0xffffffffu, role_wait(&sh.empty[st], (uint32_t)((use - 1) & 1), abort));
                    if (!w) break;
                }
                unsigned char* stage = dsm + (size_t)st * sb;
                const uint32_t fb = bar_addr(&sh.full[st]);
                if (c < s0.nch) issue_chunk(s0, c, N8, stage, tid, fb);
                else issue_chunk(s1, c - s0.nch, N8, stage, tid, fb);
                asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar_addr(&sh.full[st]))
                             : "memory");
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc =
                (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((uint32_t)(N8 >> 3) << 17) | (4u << 24);
            const uint32_t bp = b_plane_bytes(N8);
            const uint64_t dbase = smem_desc(smem_u32(dsm), 128, kGrp);   // stage 0, plane 0, k-step 0
            int g = 0, grp = 0;
            bool ok = true;
            for (int i = blockIdx.x; i < n_items && ok; i += gridDim.x) {
                Seg s0, s1;
                it.segs(i, s0, s1);
                const int nch = s0.nch + s1.nch;
                for (int c = 0; c < nch && ok; ++c, ++g) {
                    const int buf = grp & 1;
                    if (c % kDrain == 0 && grp >= 2) {
                        ok = role_wait(&sh.acce[buf], (uint32_t)(((grp >> 1) - 1) & 1), abort);
                        if (!ok) break;
                    }
                    const int st = g % kRingStages, use = g / kRingStages;
                    ok = role_wait(&sh.full[st], (uint32_t)(use & 1), abort);
                    if (!ok) break;
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    // descriptors differ only in the start address (bits
                    // 0-13, 16-byte units; shared addresses stay below 256 KiB
                    // so adding an offset never carries out of the field)
                    const uint64_t da = dbase + (uint64_t)((st * sb) >> 4);
                    const uint64_t db = da + (uint64_t)(kChunkBytes >> 4);
                    const uint32_t dm = tmem + (uint32_t)(256 * buf), dc = dm + kCorrCol;
#pragma unroll
                    for (int ks = 0; ks < kKC / 16; ++ks) {
                        const uint64_t ko = (uint64_t)(ks * 256 >> 4);
                        const uint32_t acc = (c % kDrain == 0 && ks == 0) ? 0u : 1u;
                        const uint64_t a1 = da + ko, a2 = a1 + (kImg >> 4), a3 = a2 + (kImg >> 4);
                        const uint64_t b1 = db + ko, b2 = b1 + (bp >> 4), b3 = b2 + (bp >> 4);
                        mma_bf16(dm, a1, b1, idesc, acc);
                        mma_bf16(dc, a1, b2, idesc, acc);
                        mma_bf16(dc, a2, b1, idesc, 1u);
                        mma_bf16(dc, a1, b3, idesc, 1u);
                        mma_bf16(dc, a2, b2, idesc, 1u);
                        mma_bf16(dc, a3, b1, idesc, 1u);
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     bar_addr(&sh.empty[st]))
                                 : "memory");
                    if (c % kDrain == kDrain - 1 || c == nch - 1) {
                        asm volatile(
                            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                bar_addr(&sh.accf[buf]))
                            : "memory");
                        ++grp;
                    }
                }
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ drainers and epilogue
        const int q = warp & 3;                       // lane quarter
        const int row = 16 * q + lane;                 // accumulator row of this thread (lanes 0-15)
        const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16);
        const int nblk = N8 / 8;
        int grp = 0;
        bool ok = true;
        for (int i = blockIdx.x; i < n_items && ok; i += gridDim.x) {
            Seg s0, s1;
            it.segs(i, s0, s1);
            const int nch = s0.nch + s1.nch;
            float racc[kMaxBlkAll][8];
#pragma unroll
            for (int b = 0; b < kMaxBlkAll; ++b)
#pragma unroll
                for (int j = 0; j < 8; ++j) racc[b][j] = 0.0f;
            const int ngr = (nch + kDrain - 1) / kDrain;
            for (int gg = 0; gg < ngr; ++gg, ++grp) {
                const int buf = grp & 1;
                ok = role_wait(&sh.accf[buf], (uint32_t)((grp >> 1) & 1), abort);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int b0 = 0; b0 < kMaxBlkAll; b0 += 3) {
                    uint32_t r[3][16];
#pragma unroll
                    for (int t = 0; t < 3; ++t) {
                        const int b = b0 + t;
                        if (b < nblk) {
                            const uint32_t ad = lane_addr + (uint32_t)(256 * buf) + 8 * b;
                            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                         : "=r"(r[t][0]), "=r"(r[t][1]), "=r"(r[t][2]), "=r"(r[t][3]),
                                           "=r"(r[t][4]), "=r"(r[t][5]), "=r"(r[t][6]), "=r"(r[t][7])
                                         : "r"(ad));
                            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                         : "=r"(r[t][8]), "=r"(r[t][9]), "=r"(r[t][10]), "=r"(r[t][11]),
                                           "=r"(r[t][12]), "=r"(r[t][13]), "=r"(r[t][14]), "=r"(r[t][15])
                                         : "r"(ad + kCorrCol));
                        }
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int t = 0; t < 3; ++t)
                        if (b0 + t < nblk)
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                racc[b0 + t][j] += __uint_as_float(r[t][j]) + __uint_as_float(r[t][8 + j]);
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(&sh.acce[buf]);
            }
            // one outcome for all four drainer warps (they meet at the
            // epilogue's named barrier below); a warp that gave up arrives
            // here too, the others within their own bounded waits
            uint32_t all_ok;
            asm volatile(
                "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
                "bar.red.and.pred q, 1, 128, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
                : "=r"(all_ok)
                : "r"((uint32_t)ok)
                : "memory");
            ok = all_ok != 0;
            if (!ok) break;
            // epilogue of item i
            if (it.rows) {
                // through a shared-memory tile, so that rows are written
                // (and xin / b read) coalesced; the four drainer warps meet
                // at named barrier 1
                const Tile t = it.op.tiles[it.op.torder[i]];
                float* tile = reinterpret_cast<float*>(dsm + (size_t)kRingStages * sb);
                const int ldt = N8 + 1;
                if (lane < 16)
#pragma unroll
                    for (int b = 0; b < kMaxBlkAll; ++b)
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (b < nblk) tile[row * ldt + 8 * b + j] = racc[b][j];
                asm volatile("bar.sync 1, 128;" ::: "memory");
                for (int e = tid - 128; e < t.rows * nc; e += kDrainers) {
                    const int r = e / nc, col = e - r * nc;
                    epilogue_tc(epi, Y, ldy, t.r0 + r, col, tile[r * ldt + col]);
                }
                asm volatile("bar.sync 1, 128;" ::: "memory");
            } else if (lane < 16) {
                {
                    const GWork w = it.op.gwork[i];
                    const Group gr = it.op.groups[w.g];
                    if (row < w.rows) {
                        // 8 columns of each plane per 16-byte store (rows of
                        // N8 BF16 are 16-byte aligned)
                        const long long base = (long long)(gr.toff + w.r0 + row) * N8;
#pragma unroll
                        for (int b = 0; b < kMaxBlkAll; ++b) {
                            if (b >= nblk) continue;
                            __align__(16) __nv_bfloat16 p1[8], p2[8], p3[8];
#pragma unroll
                            for (int j = 0; j < 8; ++j) split3(8 * b + j < nc ? racc[b][j] : 0.0f, p1[j], p2[j], p3[j]);
                            *reinterpret_cast<uint4*>(Tout + base + 8 * b) = *reinterpret_cast<const uint4*>(p1);
                            *reinterpret_cast<uint4*>(Tout + tplane_out + base + 8 * b) = *reinterpret_cast<const uint4*>(p2);
                            *reinterpret_cast<uint4*>(Tout + 2 * tplane_out + base + 8 * b) =
                                *reinterpret_cast<const uint4*>(p3);
                        }
                    }
                }
            }
        }
    }
    if (tid == 0 && *abort) atomicExch(&g_tc_timeout, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// Chunk images and split vector planes of one product.
struct TcArgs {
    const unsigned char* img;
    const long long* tile_near0;   // first chunk of every tile's dense panel
    const long long* tile_far0;    // first chunk of every tile's U panel
    const long long* item0;        // first chunk of every far-field item
    const __nv_bfloat16* Xs;       // three planes of n x N8
    __nv_bfloat16* Ts;             // three planes of sum_rank x N8
    long long xplane, tplane;
    int nc, N8;
};

inline size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

// ---------------------------------------------------------------- host side
bool tc_supported(const rad_htree* h) { return h->compressed && !h->op_is_f64() && !h->from_dense; }

void tc_drop_images(rad_htree* h) {
    h->tc_img.release(nullptr);
    h->tc_tile_near0.release(nullptr);
    h->tc_tile_far0.release(nullptr);
    h->tc_item0.release(nullptr);
    h->tc_ready = false;
}

// The three BF16 chunk images of every panel (dense and U panels per tile,
// V^T panels per far-field item), built once for the tensor-core path.
void tc_build_images(rad_htree* h, cudaStream_t s) {
    RAD_REQUIRE(tc_supported(h), RAD_EINVAL, "tensor-core products need an FP32 or BF16 operator");
    if (h->tc_ready) return;
    std::vector<GWork> gw(h->n_gwork);
    if (h->n_gwork > 0)
        RAD_CUDA(cudaMemcpyAsync(gw.data(), h->d_gwork.p, sizeof(GWork) * gw.size(), cudaMemcpyDeviceToHost, s));
    RAD_CUDA(cudaStreamSynchronize(s));
    const int nt = h->n_tiles;
    std::vector<long long> near0(std::max(1, nt)), far0(std::max(1, nt)), item0(std::max<size_t>(1, gw.size()));
    std::vector<PackJob> jn, jf;   // near pool jobs, factor pool jobs
    long long cur = 0;
    for (int t = 0; t < nt; ++t) {
        const Tile& tl = h->tiles_h[t];
        near0[t] = cur;
        for (int k0 = 0; k0 < tl.kn; k0 += kKC) jn.push_back(PackJob{tl.noff, tl.ld, tl.rows, k0, tl.kn, cur++});
        far0[t] = cur;
        for (int k0 = 0; k0 < tl.kf; k0 += kKC) jf.push_back(PackJob{tl.foff, tl.ld, tl.rows, k0, tl.kf, cur++});
    }
    for (size_t w = 0; w < gw.size(); ++w) {
        const Group& g = h->groups_h[gw[w].g];
        item0[w] = cur;
        for (int k0 = 0; k0 < g.n; k0 += kKC)
            jf.push_back(PackJob{g.voff + gw[w].r0, g.ld, gw[w].rows, k0, g.n, cur++});
    }
    h->tc_img.alloc((size_t)std::max<long long>(cur, 1) * kChunkBytes, s);
    h->tc_tile_near0.alloc(sizeof(long long) * near0.size(), s);
    h->tc_tile_far0.alloc(sizeof(long long) * far0.size(), s);
    h->tc_item0.alloc(sizeof(long long) * item0.size(), s);
    RAD_CUDA(cudaMemcpyAsync(h->tc_tile_near0.p, near0.data(), sizeof(long long) * near0.size(), cudaMemcpyHostToDevice, s));
    RAD_CUDA(cudaMemcpyAsync(h->tc_tile_far0.p, far0.data(), sizeof(long long) * far0.size(), cudaMemcpyHostToDevice, s));
    RAD_CUDA(cudaMemcpyAsync(h->tc_item0.p, item0.data(), sizeof(long long) * item0.size(), cudaMemcpyHostToDevice, s));
    Scratch ws(s);
    for (int pass = 0; pass < 2; ++pass) {
        const std::vector<PackJob>& jv = pass == 0 ? jn : jf;
        if (jv.empty()) continue;
        PackJob* d = ws.get_n<PackJob>(jv.size());
        RAD_CUDA(cudaMemcpyAsync(d, jv.data(), sizeof(PackJob) * jv.size(), cudaMemcpyHostToDevice, s));
        ProfScope ps_("tc_pack", s);
        if (pass == 0) {
            tc_pack_kernel<float><<<(unsigned)jv.size(), 256, 0, s>>>(h->near_pool.as<float>(), d, h->tc_img.as<unsigned char>());
        } else if (h->factor_dtype == RAD_F32) {
            tc_pack_kernel<float><<<(unsigned)jv.size(), 256, 0, s>>>(h->far_pool.as<float>(), d, h->tc_img.as<unsigned char>());
        } else {
            tc_pack_kernel<__nv_bfloat16><<<(unsigned)jv.size(), 256, 0, s>>>(h->far_pool.as<__nv_bfloat16>(), d,
                                                                               h->tc_img.as<unsigned char>());
        }
        RAD_CHECK_LAUNCH();
    }
    RAD_CUDA(cudaStreamSynchronize(s));   // the host job lists go out of scope
    h->tc_ready = true;
}

// Workspace of one tensor-core product of up to kMaxN8 columns: the split
// planes of X (n rows) and of T (sum_rank rows).
size_t tc_workspace_bytes(const rad_htree* h, int nrhs) {
    const int N8 = std::min(kMaxN8, (nrhs + 7) / 8 * 8);
    return align256((size_t)3 * h->n * N8 * 2) + align256((size_t)3 * std::max(1, h->sum_rank) * N8 * 2) + 256;
}

// Y = F X for nc <= 96 FP32 columns (rows of X at stride ldx), epilogue as
// in apply_tree; ws holds tc_workspace_bytes(h, nc) bytes.
void tc_product(const rad_htree* h, const OpView& op, const float* X, int ldx, void* Y, int ldy, int nc,
                const Epi& epi, void* ws, cudaStream_t s) {
    RAD_REQUIRE(h->tc_ready, RAD_EINVAL, "tensor-core images missing (select the path first)");
    const int N8 = (nc + 7) / 8 * 8;
    const int n = (int)h->n;
    unsigned char* base = reinterpret_cast<unsigned char*>(align256(reinterpret_cast<uintptr_t>(ws)));
    TcArgs ta;
    ta.img = h->tc_img.as<unsigned char>();
    ta.tile_near0 = h->tc_tile_near0.as<long long>();
    ta.tile_far0 = h->tc_tile_far0.as<long long>();
    ta.item0 = h->tc_item0.as<long long>();
    ta.xplane = (long long)n * N8;
    ta.tplane = (long long)std::max(1, h->sum_rank) * N8;
    ta.Xs = reinterpret_cast<const __nv_bfloat16*>(base);
    ta.Ts = reinterpret_cast<__nv_bfloat16*>(base + align256((size_t)3 * ta.xplane * 2));
    ta.nc = nc;
    ta.N8 = N8;
    const size_t smem = (size_t)kRingStages * stage_bytes(N8) + (size_t)kTileRows * (N8 + 1) * 4;
    static std::once_flag configured;
    static int sms = 0;
    std::call_once(configured, [&] {
        RAD_CUDA(cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kRingStages * stage_bytes(kMaxN8) + kTileRows * (kMaxN8 + 1) * 4));
        int dev = 0;
        RAD_CUDA(cudaGetDevice(&dev));
        RAD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    });
    {
        ProfScope ps_("tc_split", s);
        const long long tot = ta.xplane;
        tc_split_rows_kernel<<<(unsigned)std::min<long long>((tot + 255) / 256, 4096), 256, 0, s>>>(
            X, ldx, n, nc, N8, const_cast<__nv_bfloat16*>(ta.Xs), ta.xplane);
    }
    RAD_CHECK_LAUNCH();
    if (op.n_gwork > 0) {
        Items it{false, op, ta.item0, nullptr, ta.img, ta.Xs, ta.Ts, ta.xplane, ta.tplane};
        ProfScope ps_("hmm_far_vt", s);
        tc_gemm_kernel<<<std::min(op.n_gwork, sms), 256, smem, s>>>(it, nc, N8, nullptr, 0, epi, ta.Ts, ta.tplane);
        RAD_CHECK_LAUNCH();
    }
    {
        Items it{true, op, ta.tile_near0, ta.tile_far0, ta.img, ta.Xs, ta.Ts, ta.xplane, ta.tplane};
        ProfScope ps_("hmm_rows", s);
        tc_gemm_kernel<<<std::min(op.n_tiles, sms), 256, smem, s>>>(it, nc, N8, Y, ldy, epi, nullptr, 0);
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
