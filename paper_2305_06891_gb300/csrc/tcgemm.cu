// Tensor-core (tcgen05) panel GEMMs of the many-column product, FP32
// operands at FP32-level accuracy.
//
// A panel times gathered vector rows, D[64 x N] += A[64 x K] B[K x N], runs
// on the 5th-generation tensor cores with the accumulator in tensor memory.
// TF32 alone keeps 10 mantissa bits, far from the 1e-6 this product must
// meet, so every operand is split into hi = tf32(x) (rounded to nearest) and
// lo = tf32(x - hi) and the product takes all four terms hi*hi + hi*lo +
// lo*hi + lo*lo: the inputs lose about 2^-23 relative and the accumulation
// is FP32, as for an FP32 FFMA loop.
//
// Per CTA (256 threads, one work item): chunks of KC = 32 panel columns and
// their 32 gathered rows are loaded from global memory into registers
// (16-byte vectors), split, and stored into shared memory as K-major
// 8 x 16-byte core matrices (no swizzle; the stride between 8-row groups is
// padded by 16 bytes to spread shared-memory banks).  Two stages: while one
// thread issues the 16 MMAs of chunk c (4 k-steps of 8 x 4 terms) and
// commits them to the stage's mbarrier, the threads load chunk c + 1.  A
// stage is rewritten only after its previous MMAs completed.  The M = 64
// accumulator lives in tensor-memory lanes 0-15 of each 32-lane quarter
// (rows 16 q .. 16 q + 15 in quarter q); warps w and w + 4 read quarter w for
// the two halves of the columns.
//
// Every wait is bounded: after kWaitLimit polls a CTA records the timeout in
// a device flag (checked by the host at its next synchronisation), skips the
// rest of its work, waits (bounded) for its own MMAs and frees its tensor
// memory.

#include <cstdint>
#include <mutex>

#include "rad_device.cuh"

namespace rad {

__device__ int g_tc_timeout = 0;

namespace {

constexpr int kKC = 32;                  // panel columns per chunk
constexpr int kCoreBytes = 128;          // 8 rows x 16 bytes
constexpr int kGroupStride = (kKC / 4) * kCoreBytes + 16;   // 8-row group stride (SBO)
constexpr int kTmemCols = 256;           // main accumulator at 0, corrections at 128
constexpr uint32_t kCorrCol = 128;
constexpr long kWaitLimit = 1l << 26;     // polls (well beyond any real MMA latency)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((kCoreBytes >> 4) & 0x3FFF) << 16;        // K-adjacent cores
    d |= (uint64_t)((kGroupStride >> 4) & 0x3FFF) << 32;      // 8-row groups
    d |= (uint64_t)1 << 46;                                   // tcgen05 descriptor version
    return d;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

// non-blocking poll of an mbarrier phase (test_wait returns at once; the
// blocking try_wait may suspend the thread for a time slice)
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long it = 0; it < kWaitLimit; ++it)
        if (mbar_try(bar, parity)) return true;
    return false;
}

// split x into two TF32 values (round to nearest, ties away from zero):
// hi = tf32(x), lo = tf32(x - hi)
__device__ __forceinline__ float tf32_rn(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}

// A chunk element source: panel column k (FP32 or BF16 storage)
__device__ __forceinline__ float4 load_quad(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 load_quad(const __nv_bfloat16* p) {
    const uint2 q = *reinterpret_cast<const uint2*>(p);
    return make_float4(__uint_as_float(q.x << 16), __uint_as_float(q.x & 0xffff0000u), __uint_as_float(q.y << 16),
                       __uint_as_float(q.y & 0xffff0000u));
}

// One K segment: panel A (column-major, leading dimension lda, rows_pad
// rows used) times rows of B selected by idx (or base + k when idx is null).
template <class AS>
struct Seg {
    const AS* A;
    long long lda;
    int rows_pad;
    int K;
    const float* B;
    int ldb;
    const int* idx;
    int base;
};

// store element (r, k) of a K-major operand split into hi / lo
__device__ __forceinline__ void put_split(unsigned char* hi, unsigned char* lo, int r, int k, float x) {
    const int off = (r >> 3) * kGroupStride + (k >> 2) * kCoreBytes + (r & 7) * 16 + (k & 3) * 4;
    const float h = tf32_rn(x);
    *reinterpret_cast<float*>(hi + off) = h;
    *reinterpret_cast<float*>(lo + off) = tf32_rn(x - h);
}

// Raw chunk staging: the KC panel columns (64 rows each, storage type AS)
// and the KC gathered vector rows (N8 floats each) land in shared memory by
// cp.async, kRawStages chunks ahead of the split pass.
constexpr int kRawStages = 3;
// bytes of one raw stage (FP32 panel columns are the larger case)
__host__ __device__ constexpr int raw_stage_bytes(int N8) { return kKC * kTileRows * 4 + kKC * N8 * 4; }
template <class AS>
__device__ __forceinline__ int raw_a_bytes() { return kKC * kTileRows * (int)sizeof(AS); }

__device__ __forceinline__ void cp16(void* sdst, const void* gsrc, bool pred) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(sdst)), "l"(gsrc),
                 "r"(pred ? 16 : 0));
}
__device__ __forceinline__ void cp8(void* sdst, const void* gsrc, bool pred) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(smem_u32(sdst)), "l"(gsrc),
                 "r"(pred ? 8 : 0));
}

// issue the copies of chunk k0 .. k0 + KC of one segment into raw stage st
// (entries past K or past the vector's columns are zero-filled)
template <class AS>
__device__ __forceinline__ void issue_chunk(const Seg<AS>& sg, int k0, int nq_load, int N8, unsigned char* st) {
    AS* ra = reinterpret_cast<AS*>(st);
    float* rb = reinterpret_cast<float*>(st + raw_a_bytes<AS>());
    const int tid = threadIdx.x;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int u = tid + 256 * i;            // u < 512 = 32 columns x 16 row quads
        const int k = u >> 4, mq = u & 15;
        const bool ok = k0 + k < sg.K && 4 * mq < sg.rows_pad;
        const AS* src = ok ? sg.A + (long long)(k0 + k) * sg.lda + 4 * mq : sg.A;
        if constexpr (sizeof(AS) == 4) cp16(ra + k * kTileRows + 4 * mq, src, ok);
        else cp8(ra + k * kTileRows + 4 * mq, src, ok);
    }
    const int nq = N8 / 4;
    for (int u = tid; u < kKC * nq; u += 256) {
        const int k = u / nq, q = u - k * nq;
        const bool ok = k0 + k < sg.K && q < nq_load;
        const float* src = sg.B;
        if (ok) src = sg.B + (long long)(sg.idx ? sg.idx[k0 + k] : sg.base + k0 + k) * sg.ldb + 4 * q;
        cp16(rb + k * N8 + 4 * q, src, ok);
    }
}

__device__ __forceinline__ float4 raw_quad(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 raw_quad(const __nv_bfloat16* p) { return load_quad(p); }

// split pass: raw stage -> K-major hi / lo core matrices
template <class AS>
__device__ __forceinline__ void split_chunk(const unsigned char* raw, unsigned char* st, int a_bytes, int b_bytes,
                                            int N8) {
    const AS* ra = reinterpret_cast<const AS*>(raw);
    const float* rb = reinterpret_cast<const float*>(raw + raw_a_bytes<AS>());
    unsigned char* Ahi = st;
    unsigned char* Alo = st + a_bytes;
    unsigned char* Bhi = st + 2 * a_bytes;
    unsigned char* Blo = st + 2 * a_bytes + b_bytes;
    const int tid = threadIdx.x;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int u = tid + 256 * i;
        const int k = u >> 4, m = 4 * (u & 15);
        const float4 v = raw_quad(ra + k * kTileRows + m);
        put_split(Ahi, Alo, m, k, v.x);
        put_split(Ahi, Alo, m + 1, k, v.y);
        put_split(Ahi, Alo, m + 2, k, v.z);
        put_split(Ahi, Alo, m + 3, k, v.w);
    }
    const int nq = N8 / 4;
    for (int u = tid; u < kKC * nq; u += 256) {
        const int k = u / nq, q = u - k * nq;
        const float4 v = *reinterpret_cast<const float4*>(rb + k * N8 + 4 * q);
        const int n = 4 * q;
        put_split(Bhi, Blo, n, k, v.x);
        put_split(Bhi, Blo, n + 1, k, v.y);
        put_split(Bhi, Blo, n + 2, k, v.z);
        put_split(Bhi, Blo, n + 3, k, v.w);
    }
}

// tcgen05.ld of 8 accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld8(uint32_t addr, float v[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

constexpr int kMaxBlk = 6;   // 8-column blocks per warp half (N <= 96)

// Adds one chunk's accumulators (main hi*hi at column 0, corrections at
// column kCorrCol) to this thread's FP32 registers: rows 16 (w % 4) + lane
// of the accumulator (lanes 0-15), 8-column blocks [b0, b1) of its half.
__device__ __forceinline__ void drain_add(uint32_t tmem, int b0, int b1, float (&racc)[kMaxBlk][8]) {
    const int warp = threadIdx.x >> 5;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll
    for (int i = 0; i < kMaxBlk; ++i) {
        const int b = b0 + i;
        if (b < b1) {
            float v[8], w[8];
            tmem_ld8(lane_addr + 8 * b, v);
            tmem_ld8(lane_addr + kCorrCol + 8 * b, w);
#pragma unroll
            for (int j = 0; j < 8; ++j) racc[i][j] += v[j] + w[j];
        }
    }
}

// racc = sum over the segments of A_s B_s for one 64-row item (rows and
// blocks as in drain_add); returns false if a wait timed out.
//
// The tensor cores accumulate a chunk (32 k) at a time, starting from zero:
// hi*hi into the main accumulator, the three correction terms into a
// second one; each chunk is then added into FP32 registers.  Summing long
// panels inside the tensor core would carry its accumulation rounding over
// all K; per chunk it stays at FP32 level.
template <class AS0, class AS1>
__device__ bool tc_item(const Seg<AS0>& s0, const Seg<AS1>& s1, int nseg, int N8, int nc_load, unsigned char* smem,
                        uint32_t tmem, uint32_t bar0, uint32_t bar1, int b0, int b1, float (&racc)[kMaxBlk][8]) {
    (void)bar1;
    const int a_bytes = 8 * kGroupStride;             // 64 rows
    const int b_bytes = (N8 / 8) * kGroupStride;
    const int raw_bytes = raw_stage_bytes(N8);
    unsigned char* hilo = smem + kRawStages * raw_bytes;
    const int nq_load = (nc_load + 3) / 4;            // quads read from memory
    const int c0n = (s0.K + kKC - 1) / kKC;
    const int c1n = nseg > 1 ? (s1.K + kKC - 1) / kKC : 0;
    const int nch = c0n + c1n;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N8 >> 3) << 17) | (4u << 24);
#pragma unroll
    for (int i = 0; i < kMaxBlk; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) racc[i][j] = 0.0f;
    if (nch == 0) return true;
    auto issue = [&](int c) {
        if (c < nch) {
            unsigned char* st = smem + (c % kRawStages) * raw_bytes;
            if (c < c0n) issue_chunk<AS0>(s0, c * kKC, nq_load, N8, st);
            else issue_chunk<AS1>(s1, (c - c0n) * kKC, nq_load, N8, st);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    for (int c = 0; c < kRawStages; ++c) issue(c);
    bool ok = true;
    for (int c = 0; c < nch; ++c) {
        asm volatile("cp.async.wait_group %0;\n" ::"n"(kRawStages - 1) : "memory");   // chunk c landed
        if (c >= 1) {
            // MMAs of chunk c-1 done: accumulators readable, hi/lo free
            ok = ok && mbar_wait(bar0, (c - 1) & 1);
            ok = __syncthreads_and(ok);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            drain_add(tmem, b0, b1, racc);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        } else {
            __syncthreads();
        }
        const unsigned char* raw = smem + (c % kRawStages) * raw_bytes;
        if (c < c0n) split_chunk<AS0>(raw, hilo, a_bytes, b_bytes, N8);
        else split_chunk<AS1>(raw, hilo, a_bytes, b_bytes, N8);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        issue(c + kRawStages);                         // refill the raw stage just split
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ahi = smem_u32(hilo), alo = ahi + a_bytes, bhi = ahi + 2 * a_bytes, blo = bhi + b_bytes;
#pragma unroll
            for (int k8 = 0; k8 < kKC / 8; ++k8) {
                const uint32_t ko = k8 * 2 * kCoreBytes;
                const uint32_t acc = k8 > 0 ? 1u : 0u;
                mma_tf32(tmem, smem_desc(ahi + ko), smem_desc(bhi + ko), idesc, acc);
                mma_tf32(tmem + kCorrCol, smem_desc(alo + ko), smem_desc(blo + ko), idesc, acc);
                mma_tf32(tmem + kCorrCol, smem_desc(ahi + ko), smem_desc(blo + ko), idesc, 1u);
                mma_tf32(tmem + kCorrCol, smem_desc(alo + ko), smem_desc(bhi + ko), idesc, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar0)
                         : "memory");
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (ok) {
        ok = mbar_wait(bar0, (nch - 1) & 1);
        ok = __syncthreads_and(ok);
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            drain_add(tmem, b0, b1, racc);
        }
    } else {
        __syncthreads();
    }
    return ok;
}

struct TcShared {
    unsigned long long bar[2];
    uint32_t tmem;
};

__device__ __forceinline__ void tc_setup(TcShared& sh) {
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sh.bar[0])), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sh.bar[1])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_teardown(TcShared& sh) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sh.tmem), "r"(kTmemCols));
}

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

// 8-column blocks [b0, b1) of the accumulator read by this thread's warp half
__device__ __forceinline__ void drain_blocks(int N8, int& b0, int& b1) {
    const int nblk = N8 / 8, half = threadIdx.x >> 7;
    b0 = half ? (nblk + 1) / 2 : 0;
    b1 = half ? nblk : (nblk + 1) / 2;
}

// Y rows of every tile = epilogue([dense | U] [X gathered ; T gathered]).
template <class FS>
__global__ void __launch_bounds__(256, 2)
tc_rows_kernel(OpView op, const float* __restrict__ X, int ldx, const float* __restrict__ T, int ldt, void* Y, int ldy,
               int nc, int N8, Epi epi) {
    extern __shared__ __align__(1024) unsigned char dsm[];
    __shared__ TcShared sh;
    tc_setup(sh);
    const uint32_t tmem = sh.tmem;
    const Tile t = op.tiles[op.torder[blockIdx.x]];
    const Seg<float> s0{static_cast<const float*>(op.near_pool) + t.noff, t.ld, t.ld, t.kn, X, ldx,
                        op.xidx + t.ixn, 0};
    const Seg<FS> s1{static_cast<const FS*>(op.far_pool) + t.foff, t.ld, t.ld, t.kf, T, ldt, op.tidx + t.ixf, 0};
    int b0, b1;
    drain_blocks(N8, b0, b1);
    float racc[kMaxBlk][8];
    const bool ok = tc_item<float, FS>(s0, s1, 2, N8, nc, dsm, tmem, smem_u32(&sh.bar[0]), smem_u32(&sh.bar[1]), b0,
                                       b1, racc);
    const int lane = threadIdx.x & 31, row = 16 * ((threadIdx.x >> 5) & 3) + lane;
    if (ok) {
        if (lane < 16 && row < t.rows)
#pragma unroll
            for (int i = 0; i < kMaxBlk; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int col = 8 * (b0 + i) + j;
                    if (b0 + i < b1 && col < nc) epilogue_tc(epi, Y, ldy, t.r0 + row, col, racc[i][j]);
                }
    } else if (threadIdx.x == 0) {
        atomicExch(&g_tc_timeout, 1);
    }
    tc_teardown(sh);
}

// T rows of every far-field item = V^T panel rows times X rows c0 .. c0 + n.
template <class FS>
__global__ void __launch_bounds__(256, 2)
tc_far_vt_kernel(OpView op, const float* __restrict__ X, int ldx, float* __restrict__ T, int ldt, int nc, int N8) {
    extern __shared__ __align__(1024) unsigned char dsm[];
    __shared__ TcShared sh;
    tc_setup(sh);
    const uint32_t tmem = sh.tmem;
    const GWork w = op.gwork[blockIdx.x];
    const Group gr = op.groups[w.g];
    const int rows_pad = (w.rows + 3) / 4 * 4;
    const Seg<FS> s0{static_cast<const FS*>(op.far_pool) + gr.voff + w.r0, gr.ld, rows_pad, gr.n, X, ldx, nullptr,
                     gr.c0};
    int b0, b1;
    drain_blocks(N8, b0, b1);
    float racc[kMaxBlk][8];
    const bool ok = tc_item<FS, FS>(s0, s0, 1, N8, nc, dsm, tmem, smem_u32(&sh.bar[0]), smem_u32(&sh.bar[1]), b0, b1,
                                    racc);
    const int lane = threadIdx.x & 31, row = 16 * ((threadIdx.x >> 5) & 3) + lane;
    if (ok) {
        if (lane < 16 && row < w.rows)
#pragma unroll
            for (int i = 0; i < kMaxBlk; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int col = 8 * (b0 + i) + j;
                    if (b0 + i < b1 && col < nc) T[(long long)(gr.toff + w.r0 + row) * ldt + col] = racc[i][j];
                }
    } else if (threadIdx.x == 0) {
        atomicExch(&g_tc_timeout, 1);
    }
    tc_teardown(sh);
}

size_t tc_smem_bytes(int N8) {
    return (size_t)kRawStages * raw_stage_bytes(N8) + 2 * 8 * kGroupStride + 2 * (N8 / 8) * kGroupStride;
}

}  // namespace

// Launchers (FP32 vectors; FS = panel storage of the low-rank factors).
// X and T rows must be 16-byte aligned with leading dimensions that are
// multiples of 4 (the vector quads are read 16 bytes at a time).
template <class FS>
void tc_rows(const OpView& op, const float* X, int ldx, const float* T, int ldt, void* Y, int ldy, int nc,
             const Epi& epi, cudaStream_t s) {
    const int N8 = (nc + 7) / 8 * 8;
    const size_t bytes = tc_smem_bytes(N8);
    static std::once_flag configured;
    std::call_once(configured, [&] {
        RAD_CUDA(cudaFuncSetAttribute(tc_rows_kernel<FS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)tc_smem_bytes(96)));
    });
    { ProfScope ps_("hmm_rows", s); tc_rows_kernel<FS><<<op.n_tiles, 256, bytes, s>>>(op, X, ldx, T, ldt, Y, ldy, nc, N8, epi); }
    RAD_CHECK_LAUNCH();
}
template <class FS>
void tc_far_vt(const OpView& op, const float* X, int ldx, float* T, int ldt, int nc, cudaStream_t s) {
    const int N8 = (nc + 7) / 8 * 8;
    const size_t bytes = tc_smem_bytes(N8);
    static std::once_flag configured;
    std::call_once(configured, [&] {
        RAD_CUDA(cudaFuncSetAttribute(tc_far_vt_kernel<FS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)tc_smem_bytes(96)));
    });
    { ProfScope ps_("hmm_far_vt", s); tc_far_vt_kernel<FS><<<op.n_gwork, 256, bytes, s>>>(op, X, ldx, T, ldt, nc, N8); }
    RAD_CHECK_LAUNCH();
}
template void tc_rows<float>(const OpView&, const float*, int, const float*, int, void*, int, int, const Epi&,
                             cudaStream_t);
template void tc_rows<__nv_bfloat16>(const OpView&, const float*, int, const float*, int, void*, int, int, const Epi&,
                                     cudaStream_t);
template void tc_far_vt<float>(const OpView&, const float*, int, float*, int, int, cudaStream_t);
template void tc_far_vt<__nv_bfloat16>(const OpView&, const float*, int, float*, int, int, cudaStream_t);

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
