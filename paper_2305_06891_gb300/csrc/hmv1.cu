// The one-column block low-rank product y = F x of §5.2 in one launch
// (FP32 vectors; FP32 dense panels; FP32 or BF16 factor panels).
//
// Work units, each a contiguous column-major panel times a vector:
//   A units   T[toff .. toff + M) = V_g^T x[c0 .. c0 + n)     (column group g)
//             Yn[r0 .. r0 + rows) = D_t x(xidx)               (row tile t, dense)
//   B units   y[r0 .. r0 + rows)  = epilogue(Yn + U_t T(tidx)) (row tile t, low rank)
// A units are handed out first, heaviest first, then B units, by one atomic
// ticket per unit, so a unit is only taken by a CTA that is running; B units
// read T and Yn only after every A unit has been written (a device counter),
// and no A unit waits for anything, so the launch needs no co-residency.
//
// Each CTA is a pipeline with two rings in shared memory: kSlots chunk
// slots (descriptor, index slice, gathered vector entries) and kStages
// panel stages (up to kChunk bytes of panel columns).  The slot ring runs
// further ahead than the stage ring, so a chunk's vector entries (an index
// load, then the entries: two memory latencies) are in place when its
// panel columns (one latency) land:
//   warp 8 (one thread)  takes tickets, publishes each chunk in a slot and
//                        copies the chunk's slice of the index list into it
//                        (1-D bulk copy, cp.async.bulk);
//   warp 9               gathers the chunk's vector entries (x[c0 + j],
//                        x[xidx[j]] or T[tidx[j]]) into the slot by 4-byte
//                        asynchronous copies; for B units it first waits for
//                        the A-unit counter;
//   warp 10 (one thread) copies each chunk's panel columns into a stage with
//                        one bulk copy;
//   warps 0-7            multiply: thread (q, g) takes rows 4q .. 4q + 3 and
//                        columns g, g + G, ... of every chunk of the unit,
//                        accumulating in registers; at the end of a unit the
//                        G partial sums of a row are added in a fixed order
//                        and the unit's rows are written.
// Every row of T, Yn and y is written by one CTA with a fixed summation
// order: results do not depend on the schedule.  All waits are bounded
// (time and tests); a wait that gives up raises the CTA's abort flag and a
// device flag that the host reads at its next synchronisation, and the CTA
// waits for its own copies in flight before it exits.

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <vector>

#include "rad_device.cuh"
#include "rad_pipe.cuh"

namespace rad {

__device__ int g_hmv1_timeout = 0;

namespace {

// kind: 0 = V^T panel of a column group (x contiguous from src),
//       1 = dense panel of a tile (x gathered through xidx from src),
//       2 = U panel of a tile (T gathered through tidx from src).
struct Unit1 {
    long long off;   // panel offset in elements of its pool
    int ld;          // panel rows (a multiple of 4, at most kMaxLd)
    int k;           // panel columns
    int kind;
    int src;
    int out;         // kind 0: first row of T; kinds 1, 2: first row of the tile
    int rows;        // rows written
};
static_assert(sizeof(Unit1) == 32, "Unit1 layout");

constexpr int kStages = 4;                    // panel stages
constexpr int kChunk = 22528;                 // panel bytes per stage
constexpr int kSlots = 6;                     // chunk slots (descriptor, indices, vector entries)
constexpr int kCols = 128;                    // panel columns per chunk at most
constexpr int kMaxLd = 1024;                  // 256 consumer threads x 4 rows
constexpr int kConsumers = 256;
constexpr int kDescWarp = kConsumers / 32;
constexpr int kGatherWarp = kDescWarp + 1;
constexpr int kPanelWarp = kDescWarp + 2;
constexpr int kThreads = kConsumers + 96;     // + descriptor, gather and panel warps
constexpr int kIdx = kCols + 8;               // index slice (16-byte aligned start, padded end)
constexpr int kMaxG = 16;                     // column classes of a unit (partial sums per row)

struct Desc {
    Unit1 u;
    int unit, col0, nc, shift, pad[4];
};
struct alignas(16) Slot {
    float x[kCols];
    int idx[kIdx];
};
static_assert(sizeof(Slot) % 16 == 0 && kChunk % 16 == 0, "slot and stage alignment");
constexpr size_t kDynSmem = (size_t)kStages * kChunk + (size_t)kSlots * sizeof(Slot);

struct Shared {
    unsigned long long pfull[kStages], pempty[kStages];
    unsigned long long dpub[kSlots], dfull[kSlots], gfull[kSlots], dempty[kSlots];
    Desc desc[kSlots];
    float part[2][4 * kConsumers];
    int abort;
};

template <class S> struct Quad;
template <> struct Quad<float> {
    static __device__ __forceinline__ void load(const unsigned char* p, float v[4]) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
};
template <> struct Quad<__nv_bfloat16> {
    static __device__ __forceinline__ void load(const unsigned char* p, float v[4]) {
        const uint2 q = *reinterpret_cast<const uint2*>(p);
        v[0] = __uint_as_float(q.x << 16); v[1] = __uint_as_float(q.x & 0xffff0000u);
        v[2] = __uint_as_float(q.y << 16); v[3] = __uint_as_float(q.y & 0xffff0000u);
    }
};

// panel columns per chunk: as many as fit a stage (at most kCols); for BF16
// panels whose columns are not 16-byte multiples an even count, so that
// every chunk starts on a 16-byte boundary
__host__ __device__ __forceinline__ int chunk_cols(int ld, int es) {
    int c = kChunk / (ld * es);
    c = c < kCols ? c : kCols;
    if (es == 2 && (ld & 7)) c &= ~1;
    return c < 1 ? 1 : c;
}

struct Args {
    const Unit1* units;
    int n_units, n_a;
    const float* near_pool;
    const void* far_pool;
    const int* xidx;
    const int* tidx;
    const float* x;
    float* T;
    float* Yn;
    void* Y;
    Epi epi;
    int* ctr;   // [0] next ticket, [1] A units written
};

__device__ __forceinline__ void raise_timeout() { atomicExch(&g_hmv1_timeout, 1); }

// AND of `ok` over the 256 consumer threads (named barrier 2)
__device__ __forceinline__ bool all_consumers(bool ok) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.and.pred p, 2, %2, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)ok), "r"(kConsumers)
        : "memory");
    return r != 0;
}

template <class FS>
__global__ void __launch_bounds__(kThreads, 2) hmv1_fused(Args a) {
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ Shared sh;
    unsigned char* panels = dsm;
    Slot* slots = reinterpret_cast<Slot*>(dsm + (size_t)kStages * kChunk);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            pipe::bar_init(&sh.pfull[i], 1);                   // panel thread (panel bytes)
            pipe::bar_init(&sh.pempty[i], kConsumers / 32);    // consumer warps
        }
        for (int i = 0; i < kSlots; ++i) {
            pipe::bar_init(&sh.dpub[i], 1);                    // descriptor thread (descriptor written)
            pipe::bar_init(&sh.dfull[i], 1);                   // descriptor thread (index bytes)
            pipe::bar_init(&sh.gfull[i], 32);                  // gather lanes
            pipe::bar_init(&sh.dempty[i], kConsumers / 32);    // consumer warps
        }
        sh.abort = 0;
        pipe::bar_init_fence();
    }
    __syncthreads();
    volatile int* abort = &sh.abort;

    if (warp == kDescWarp) {
        // ------------------------------------------------ tickets, descriptors, index slices
        if (lane != 0) return;
        uint32_t issued = 0;                    // slot d has an index copy outstanding ...
        uint32_t par[kSlots];                   // ... in its phase of parity par[d]
        int c = 0;
        bool ok = true;
        // the next unit's ticket is taken while the current unit's last two
        // chunks are published and its descriptor is read with the last one,
        // so neither latency stalls the rings, yet a CTA holds at most one
        // unit beyond the chunks in its rings (the last A units are not
        // queued behind a long backlog)
        int t = atomicAdd(&a.ctr[0], 1);
        Unit1 u{};
        if (t < a.n_units) u = a.units[t];
        while (ok) {
            int d = c % kSlots;
            uint32_t ph = (uint32_t)(c / kSlots) & 1u;
            if (t >= a.n_units) {
                if (!pipe::bar_wait(&sh.dempty[d], ph ^ 1u, abort)) {
                    ok = false;
                    break;
                }
                sh.desc[d].unit = -1;   // end marker
                pipe::bar_arrive(&sh.dpub[d]);
                pipe::bar_arrive(&sh.dfull[d]);
                return;
            }
            const int es = u.kind == 1 ? 4 : (int)sizeof(FS);
            const int cpc = chunk_cols(u.ld, es);
            const int nch = u.k > 0 ? (u.k + cpc - 1) / cpc : 1;
            int tn = a.n_units;
            Unit1 un{};
            for (int ch = 0; ch < nch; ++ch, ++c) {
                d = c % kSlots;
                ph = (uint32_t)(c / kSlots) & 1u;
                if (!pipe::bar_wait(&sh.dempty[d], ph ^ 1u, abort)) {
                    ok = false;
                    break;
                }
                if (ch == (nch > 1 ? nch - 2 : 0)) tn = atomicAdd(&a.ctr[0], 1);
                if (ch == nch - 1 && tn < a.n_units) un = a.units[tn];
                const int col0 = ch * cpc;
                const int nc = u.k > 0 ? min(cpc, u.k - col0) : 0;
                Desc& ds = sh.desc[d];
                ds.u = u;
                ds.unit = t;
                ds.col0 = col0;
                ds.nc = nc;
                ds.shift = 0;
                if (u.kind != 0 && nc > 0) {
                    const int* list = u.kind == 1 ? a.xidx : a.tidx;
                    const long long e0 = (long long)u.src + col0, a0 = e0 & ~3ll;
                    ds.shift = (int)(e0 - a0);
                    const uint32_t ib = (uint32_t)(((ds.shift + nc + 3) & ~3) * 4);
                    pipe::bar_arrive(&sh.dpub[d]);
                    pipe::bar_arrive_tx(&sh.dfull[d], ib);
                    pipe::bulk_g2s(slots[d].idx, list + a0, ib, &sh.dfull[d]);
                    issued |= 1u << d;
                    par[d] = ph;
                } else {
                    pipe::bar_arrive(&sh.dpub[d]);
                    pipe::bar_arrive(&sh.dfull[d]);
                }
            }
            t = tn;
            u = un;
        }
        // gave up: wait for this CTA's index copies still in flight
        raise_timeout();
        volatile int never = 0;
        for (int d = 0; d < kSlots; ++d)
            if (issued >> d & 1u) (void)pipe::bar_wait(&sh.dfull[d], par[d], &never);
        return;
    }

    if (warp == kPanelWarp) {
        // ------------------------------------------------ panel columns
        if (lane != 0) return;
        uint32_t issued = 0;
        uint32_t par[kStages];
        bool ok = true;
        for (int c = 0;; ++c) {
            const int d = c % kSlots, s = c % kStages;
            const uint32_t phd = (uint32_t)(c / kSlots) & 1u, ph = (uint32_t)(c / kStages) & 1u;
            if (!pipe::bar_wait(&sh.dpub[d], phd, abort) || !pipe::bar_wait(&sh.pempty[s], ph ^ 1u, abort)) {
                ok = false;
                break;
            }
            const Desc& ds = sh.desc[d];
            if (ds.unit < 0) {
                pipe::bar_arrive(&sh.pfull[s]);
                break;
            }
            const Unit1 u = ds.u;
            const int es = u.kind == 1 ? 4 : (int)sizeof(FS);
            const unsigned char* base = u.kind == 1 ? reinterpret_cast<const unsigned char*>(a.near_pool)
                                                    : static_cast<const unsigned char*>(a.far_pool);
            const uint32_t pb = (uint32_t)((((long long)ds.nc * u.ld * es) + 15) & ~15ll);
            if (pb > 0) {
                pipe::bar_arrive_tx(&sh.pfull[s], pb);
                pipe::bulk_g2s(panels + (size_t)s * kChunk, base + (u.off + (long long)ds.col0 * u.ld) * es, pb,
                               &sh.pfull[s]);
                issued |= 1u << s;
                par[s] = ph;
            } else {
                pipe::bar_arrive(&sh.pfull[s]);
            }
        }
        if (ok) return;
        raise_timeout();
        volatile int never = 0;
        for (int s = 0; s < kStages; ++s)
            if (issued >> s & 1u) (void)pipe::bar_wait(&sh.pfull[s], par[s], &never);
        return;
    }

    if (warp == kGatherWarp) {
        // ------------------------------------------------ vector entries
        bool ready = false;   // every A unit written (checked once)
        for (int c = 0;; ++c) {
            const int d = c % kSlots;
            const uint32_t ph = (uint32_t)(c / kSlots) & 1u;
            if (!__all_sync(0xffffffffu, pipe::bar_wait(&sh.dfull[d], ph, abort))) {
                if (lane == 0) raise_timeout();
                break;
            }
            const Desc& ds = sh.desc[d];
            if (ds.unit < 0) {
                pipe::bar_arrive(&sh.gfull[d]);
                break;
            }
            const int kind = ds.u.kind, nc = ds.nc;
            float* xs = slots[d].x;
            if (kind == 0) {
                const float* v = a.x + ds.u.src + ds.col0;
                for (int j = lane; j < nc; j += 32) pipe::cp4(xs + j, v + j);
            } else {
                if (kind == 2 && !ready) {
                    if (!__all_sync(0xffffffffu, pipe::count_wait(&a.ctr[1], a.n_a, abort))) {
                        if (lane == 0) raise_timeout();
                        pipe::bar_arrive(&sh.gfull[d]);
                        break;
                    }
                    ready = true;
                }
                const int* ix = slots[d].idx + ds.shift;
                const float* v = kind == 1 ? a.x : a.T;
                for (int j = lane; j < nc; j += 32) pipe::cp4(xs + j, v + ix[j]);
            }
            pipe::cp_arrive(&sh.gfull[d]);
        }
        pipe::cp_wait_all();
        return;
    }

    // ---------------------------------------------------- consumers
    // Each warp follows the chunk sequence on its own; the 256 consumers
    // meet only at the start of a unit (agreeing on the wait outcome and
    // reading the unit) and at its end (partial sums).  A warp whose wait
    // gives up inside a unit counts its remaining chunks without touching
    // them (it knows how many there are) and reports at the unit's end, so
    // every consumer reaches every barrier.
    int c = 0;
    int pbuf = 0;   // partial-sum buffer of this unit (two, alternating)
    for (;;) {
        int s = c % kStages, d = c % kSlots;
        bool ok = pipe::bar_wait(&sh.pfull[s], (uint32_t)(c / kStages) & 1u, abort);
        ok = pipe::bar_wait(&sh.gfull[d], (uint32_t)(c / kSlots) & 1u, abort) && ok;
        if (!all_consumers(ok)) {
            if (tid == 0) raise_timeout();
            break;
        }
        if (sh.desc[d].unit < 0) break;
        const Unit1 u = sh.desc[d].u;
        const int es = u.kind == 1 ? 4 : (int)sizeof(FS);
        const int cpc = chunk_cols(u.ld, es);
        const int nch = u.k > 0 ? (u.k + cpc - 1) / cpc : 1;
        const int quads = u.ld >> 2;
        const int G = min(kConsumers / quads, kMaxG);
        const int q = tid % quads, g = tid / quads;
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        bool wok = true;
        for (int ch = 0; ch < nch; ++ch, ++c) {
            s = c % kStages;
            d = c % kSlots;
            if (ch > 0 && wok) {
                bool w = pipe::bar_wait(&sh.pfull[s], (uint32_t)(c / kStages) & 1u, abort);
                w = pipe::bar_wait(&sh.gfull[d], (uint32_t)(c / kSlots) & 1u, abort) && w;
                wok = __all_sync(0xffffffffu, w);
            }
            if (!wok) continue;   // the stage and slot are left alone: no release
            const int nc = u.k > 0 ? min(cpc, u.k - ch * cpc) : 0;
            if (g < G) {
                const unsigned char* P = panels + (size_t)s * kChunk + 4 * q * es;
                const float* xs = slots[d].x;
                const uint32_t cstride = (uint32_t)(u.ld * es);
                if (u.kind == 1) {
#pragma unroll 4
                    for (int j = g; j < nc; j += G) {
                        float v[4];
                        Quad<float>::load(P + (uint32_t)j * cstride, v);
                        const float xv = xs[j];
#pragma unroll
                        for (int r = 0; r < 4; ++r) acc[r] = fmaf(v[r], xv, acc[r]);
                    }
                } else {
#pragma unroll 4
                    for (int j = g; j < nc; j += G) {
                        float v[4];
                        Quad<FS>::load(P + (uint32_t)j * cstride, v);
                        const float xv = xs[j];
#pragma unroll
                        for (int r = 0; r < 4; ++r) acc[r] = fmaf(v[r], xv, acc[r]);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) {
                pipe::bar_arrive(&sh.pempty[s]);
                pipe::bar_arrive(&sh.dempty[d]);
            }
        }
        // end of the unit: rows summed over the G column classes in order
        float* part = sh.part[pbuf];
        pbuf ^= 1;
#pragma unroll
        for (int r = 0; r < 4; ++r) part[4 * tid + r] = acc[r];
        if (!all_consumers(wok)) {
            if (tid == 0) raise_timeout();
            break;
        }
        if (u.kind == 2 && tid < u.rows) (void)pipe::ld_acquire(&a.ctr[1]);
        for (int row = tid; row < u.rows; row += kConsumers) {
            float sum = 0.0f;
            for (int gg = 0; gg < G; ++gg) sum += part[4 * gg * quads + row];
            if (u.kind == 0) {
                a.T[u.out + row] = sum;
            } else if (u.kind == 1) {
                a.Yn[u.out + row] = sum;
            } else {
                const int i = u.out + row;
                const float yv = __ldcg(a.Yn + i) + sum;
                if (a.epi.mode == kStore) {
                    static_cast<float*>(a.Y)[i] = yv;
                } else {
                    const double e = a.epi.eps[i];
                    double w = a.epi.xin[(long long)i * a.epi.ld64] - (1.0 - e) * (double)yv;
                    if (a.epi.mode == kResid) w = a.epi.b[(long long)i * a.epi.ld64] - w;
                    static_cast<double*>(a.Y)[i] = w;
                }
            }
        }
        if (u.kind != 2) {
            // every row of T / Yn written before the count moves (the
            // barrier orders the CTA's stores before thread 0's release)
            asm volatile("bar.sync 1, %0;" ::"r"(kConsumers) : "memory");
            if (tid == 0) pipe::red_release_add(&a.ctr[1], 1);
        }
    }
}

template <class FS>
int fused_grid(int units) {
    static int per_sm = -1, sms = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        const int smem = (int)kDynSmem;
        RAD_CUDA(cudaFuncSetAttribute(hmv1_fused<FS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        int dev = 0;
        RAD_CUDA(cudaGetDevice(&dev));
        RAD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        RAD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hmv1_fused<FS>, kThreads, smem));
        per_sm = std::max(1, per_sm);
    });
    return std::max(1, std::min(units, per_sm * sms));
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

// Builds the unit list of the fused product when the operator allows it:
// FP32 vectors and dense panels, FP32 or BF16 factors, every panel at most
// kMaxLd rows, 16-byte aligned panel and index-list starts and 16 bytes of
// slack after each index list (a chunk's index slice is copied in whole
// 16-byte words).
void hmv1_plan(rad_htree* h, cudaStream_t s) {
    h->hmv1_ok = false;
    h->n_units1 = h->n_a1 = 0;
    h->d_units1.release(s);
    if (h->near_dtype != RAD_F32 || (h->factor_dtype != RAD_F32 && h->factor_dtype != RAD_BF16)) return;
    const int fes = h->factor_dtype == RAD_BF16 ? 2 : 4;
    if (!aligned16(h->near_pool.p) || !aligned16(h->far_pool.p) || !aligned16(h->d_xidx.p) ||
        !aligned16(h->d_tidx.p))
        return;
    long long nx = 0, nf = 0;
    for (const Tile& t : h->tiles_h) {
        nx = std::max(nx, (long long)t.ixn + t.kn);
        nf = std::max(nf, (long long)t.ixf + t.kf);
        if (t.ld % 4 || t.ld > kMaxLd || t.ld < t.rows || (t.noff * 4) % 16 || (t.foff * fes) % 16) return;
    }
    if (h->d_xidx.bytes < sizeof(int) * (size_t)(nx + 4) || h->d_tidx.bytes < sizeof(int) * (size_t)(nf + 4)) return;
    std::vector<Unit1> a, b;
    std::vector<long long> ka, kb;
    for (const Group& gr : h->groups_h) {
        if (gr.ld % 4 || gr.ld > kMaxLd || (gr.voff * fes) % 16) return;
        a.push_back(Unit1{gr.voff, gr.ld, gr.n, 0, gr.c0, gr.toff, gr.M});
        ka.push_back((long long)gr.ld * gr.n * fes);
    }
    for (const Tile& t : h->tiles_h) {
        a.push_back(Unit1{t.noff, t.ld, t.kn, 1, t.ixn, t.r0, t.rows});
        ka.push_back((long long)t.ld * t.kn * 4);
        b.push_back(Unit1{t.foff, t.ld, t.kf, 2, t.ixf, t.r0, t.rows});
        kb.push_back((long long)t.ld * t.kf * fes);
    }
    // heaviest first within each class (stable: ties keep the natural order)
    auto sorted = [](const std::vector<Unit1>& v, const std::vector<long long>& key) {
        std::vector<int> o(v.size());
        for (size_t i = 0; i < o.size(); ++i) o[i] = (int)i;
        std::stable_sort(o.begin(), o.end(), [&](int x, int y) { return key[x] > key[y]; });
        std::vector<Unit1> r;
        r.reserve(v.size());
        for (int i : o) r.push_back(v[i]);
        return r;
    };
    std::vector<Unit1> all = sorted(a, ka);
    const std::vector<Unit1> bs = sorted(b, kb);
    all.insert(all.end(), bs.begin(), bs.end());
    h->d_units1.alloc(sizeof(Unit1) * all.size(), s);
    h2d(h->d_units1.as<Unit1>(), all, s);
    h->n_units1 = (int)all.size();
    h->n_a1 = (int)a.size();
    h->hmv1_ok = true;
}

void hmv1_product(const rad_htree* h, const float* x, float* T, float* Yn, int* ctr, void* Y, const Epi& epi,
                  cudaStream_t s) {
    Args a{h->d_units1.as<Unit1>(), h->n_units1, h->n_a1, h->near_pool.as<float>(), h->far_pool.p,
           h->d_xidx.as<int>(), h->d_tidx.as<int>(), x, T, Yn, Y, epi, ctr};
    RAD_CUDA(cudaMemsetAsync(ctr, 0, 2 * sizeof(int), s));
    const int smem = (int)kDynSmem;
    if (h->factor_dtype == RAD_BF16) {
        const int grid = fused_grid<__nv_bfloat16>(h->n_units1);
        ProfScope ps_("hmv_fused", s);
        hmv1_fused<__nv_bfloat16><<<grid, kThreads, smem, s>>>(a);
    } else {
        const int grid = fused_grid<float>(h->n_units1);
        ProfScope ps_("hmv_fused", s);
        hmv1_fused<float><<<grid, kThreads, smem, s>>>(a);
    }
    RAD_CHECK_LAUNCH();
}

// Reads and clears the timeout flag of the fused product.
bool hmv1_take_timeout() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_hmv1_timeout, sizeof(int)) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_hmv1_timeout, &z, sizeof(int));
    }
    return v != 0;
}

}  // namespace rad
