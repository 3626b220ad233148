// A6: the block low-rank matrix-vector product y = F x of §5.2, in tree
// order, in two phases over the panel storage:
//   phase 1  T = V^T X      one column group (a column cluster's low-rank
//                           blocks, V^T rows stacked) at a time
//   phase 2  Y = [D | U] [X(xidx); T(tidx)]   one row tile at a time
// Every row tile is owned by one CTA: no atomics, a fixed summation order,
// deterministic results.  Panels are contiguous and column-major, so a CTA
// streams each of them front to back with fully coalesced loads.
//
// One right-hand side: thread (r, g) of a CTA takes row r of the panel and
// every G-th column starting at g, so one CTA-wide step reads G * ld
// consecutive elements; partial rows are summed over g in shared memory in a
// fixed order.
// Many right-hand sides: a panel GEMM.  Chunks of KC panel columns (A) and
// the KC gathered rows of X or T they multiply (B) are staged in shared
// memory, double buffered through registers; each thread accumulates a
// 4-row x RN-column tile (FP32 or FP64 FFMA).
//
// Epilogues fuse the reflection operator of Eq. (11):
//   kReflect: w = xin - (1 - eps) o (F x)
//   kResid:   r = b - (xin - (1 - eps) o (F x))

#include <algorithm>
#include <mutex>

#include <type_traits>

#include "rad_device.cuh"

namespace rad {

namespace {

template <class AT>
__device__ __forceinline__ void epilogue(const Epi& epi, void* Y, int ldy, int row, int col, AT acc) {
    if (epi.mode == kStore) {
        static_cast<AT*>(Y)[(long long)row * ldy + col] = acc;
    } else {
        const double e = epi.eps[row];
        double w = epi.xin[(long long)row * epi.ld64 + col] - (1.0 - e) * (double)acc;
        if (epi.mode == kResid) w = epi.b[(long long)row * epi.ld64 + col] - w;
        static_cast<double*>(Y)[(long long)row * ldy + col] = w;
    }
}

// ---------------------------------------------------------------- 1 RHS
// Four consecutive stored elements (16-byte aligned for FP32, 8 for BF16,
// 32 for FP64) converted to the accumulation type.
template <class S, class AT> struct Vec4;
template <> struct Vec4<float, float> {
    static __device__ __forceinline__ void load(const float* p, float v[4]) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
};
template <> struct Vec4<double, double> {
    static __device__ __forceinline__ void load(const double* p, double v[4]) {
        const double2 a = reinterpret_cast<const double2*>(p)[0];
        const double2 b = reinterpret_cast<const double2*>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};
template <> struct Vec4<float, double> {
    static __device__ __forceinline__ void load(const float* p, double v[4]) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
};
template <> struct Vec4<__nv_bfloat16, float> {
    static __device__ __forceinline__ void load(const __nv_bfloat16* p, float v[4]) {
        const uint2 q = *reinterpret_cast<const uint2*>(p);
        v[0] = __uint_as_float(q.x << 16); v[1] = __uint_as_float(q.x & 0xffff0000u);
        v[2] = __uint_as_float(q.y << 16); v[3] = __uint_as_float(q.y & 0xffff0000u);
    }
};

// Number of panel columns a streaming thread keeps in flight (its 4 rows of
// each, plus the matching vector entries): 8 for FP32 panels (measured
// faster on the FP32 operators), 4 for BF16 and FP64 panels (measured
// faster on the BF16 operator; FP64 keeps its register budget).
template <class S> struct InFlight { static constexpr int v = 4; };
template <> struct InFlight<float> { static constexpr int v = 8; };

// acc[0..3] += sum over panel columns c = g, g + G, ... of the 4 rows at P
// of column c times v[idx[c]] (v[base + c] when idx is null); InFlight<S>
// columns per step, summed pairwise before they reach the accumulators
template <class S, class AT>
__device__ __forceinline__ void stream_panel4(const S* __restrict__ P, long long ld, int kcols, int g, int G,
                                              const int* __restrict__ idx, const AT* __restrict__ v, AT acc[4],
                                              int base = 0) {
    constexpr int U = InFlight<S>::v;
    int c = g;
    for (; c + (U - 1) * G < kcols; c += U * G) {
        AT a[U][4], x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) Vec4<S, AT>::load(P + (long long)(c + u * G) * ld, a[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) x[u] = idx ? v[idx[c + u * G]] : v[base + c + u * G];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            AT p[U];
#pragma unroll
            for (int u = 0; u < U; ++u) p[u] = a[u][r] * x[u];
#pragma unroll
            for (int w = 1; w < U; w *= 2)
#pragma unroll
                for (int u = 0; u + w < U; u += 2 * w) p[u] += p[u + w];
            acc[r] += p[0];
        }
    }
    for (; c < kcols; c += G) {
        AT a0[4];
        Vec4<S, AT>::load(P + (long long)c * ld, a0);
        const AT x0 = idx ? v[idx[c]] : v[base + c];
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r] += a0[r] * x0;
    }
}

// acc[k][0..3] += sum over panel columns c = g, g + G, ... of the 4 rows at
// P of column c times V[idx[c]][k] (V[base + c][k] when idx is null), for
// the NCOL columns k of V's rows; four panel columns in flight per step
// (FP32 / BF16 panels).
template <class S, class AT, int NCOL>
__device__ __forceinline__ void stream_cols(const S* __restrict__ P, long long ld, int kcols, int g, int G,
                                            const int* __restrict__ idx, const AT* __restrict__ V, int ldv,
                                            AT (&acc)[NCOL][4], int base = 0) {
    constexpr int U = 4;
    int c = g;
    // FP64 panels (the plain FP64 path) keep one column per step: their
    // wider registers cost more occupancy than the extra loads in flight gain
    if constexpr (sizeof(S) != 8)
    for (; c + (U - 1) * G < kcols; c += U * G) {
        AT a[U][4];
        const AT* vr[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            Vec4<S, AT>::load(P + (long long)(c + u * G) * ld, a[u]);
            vr[u] = V + (long long)(idx ? idx[c + u * G] : base + c + u * G) * ldv;
        }
#pragma unroll
        for (int k = 0; k < NCOL; ++k) {
            AT xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) xv[u] = vr[u][k];
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[k][r] += (a[0][r] * xv[0] + a[1][r] * xv[1]) + (a[2][r] * xv[2] + a[3][r] * xv[3]);
        }
    }
    for (; c < kcols; c += G) {
        AT a[4];
        Vec4<S, AT>::load(P + (long long)c * ld, a);
        const AT* vr = V + (long long)(idx ? idx[c] : base + c) * ldv;
#pragma unroll
        for (int k = 0; k < NCOL; ++k) {
            const AT xv = vr[k];
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[k][r] += a[r] * xv;
        }
    }
}

// ---------------------------------------------------------------- 2-4 RHS
// Streaming kernels for a few right-hand sides: one pass over every panel,
// thread (q, g) owns rows 4q .. 4q+3 for all NCOL columns.
template <class FS, class AT, int NCOL>
__device__ __forceinline__ void far_vt_stream_item(int it_, OpView op, const AT* __restrict__ X, int ldx,
                                                     AT* __restrict__ T, int ldt) {
    __shared__ AT part[NCOL][1024];
    const GWork w = op.sitems[it_];
    const Group gr = op.groups[w.g];
    const int quads = (w.rows + 3) / 4;
    const int G = 256 / quads;
    const int q = threadIdx.x % quads, jg = threadIdx.x / quads;
    const long long ld = gr.ld;
    AT acc[NCOL][4] = {};
    if (jg < G)
        stream_cols<FS, AT, NCOL>(static_cast<const FS*>(op.far_pool) + gr.voff + w.r0 + 4 * q, ld, gr.n, jg, G,
                                  nullptr, X, ldx, acc, gr.c0);
#pragma unroll
    for (int c = 0; c < NCOL; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) part[c][4 * threadIdx.x + r] = acc[c][r];
    __syncthreads();
    if ((int)threadIdx.x < w.rows) {
        const int rr = threadIdx.x;
#pragma unroll
        for (int c = 0; c < NCOL; ++c) {
            AT sum = 0;
            for (int g = 0; g < G; ++g) sum += part[c][4 * (g * quads) + rr];
            T[(long long)(gr.toff + w.r0 + rr) * ldt + c] = sum;
        }
    }
}

template <class FS, class AT, int NCOL>
__global__ void __launch_bounds__(256) far_vt_stream(OpView op, const AT* __restrict__ X, int ldx, AT* __restrict__ T, int ldt) {
    // grid-stride over the work items: one CTA per item, or a persistent grid
    for (int it = blockIdx.x; it < op.n_sitems; it += gridDim.x) {
        far_vt_stream_item<FS, AT, NCOL>(it, op, X, ldx, T, ldt);
        __syncthreads();
    }
}


// ---------------------------------------------------------------- 1 RHS, two phases
// Phase A: far-field items (T = V^T x, at most 128 rows of a column group)
// and the tiles' dense panels (Yn = near x) in one launch, heaviest first, so
// that the short items fill the tail of the long ones.  Phase B: the tiles'
// low-rank panels, Y = epilogue(Yn + U T).
template <class NS, class FS, class AT>
__device__ __forceinline__ void
single_phase_a_item(int it_, OpView op, const AT* __restrict__ x, AT* __restrict__ T, AT* __restrict__ Yn) {
    __shared__ AT part[1024];
    const int code = op.aorder[it_];
    AT acc[4] = {0, 0, 0, 0};
    int quads, G, rows;
    if (code >= 0) {
        const GWork w = op.sitems[code];
        const Group gr = op.groups[w.g];
        quads = (w.rows + 3) / 4;
        G = 256 / quads;
        rows = w.rows;
        const int q = threadIdx.x % quads, jg = threadIdx.x / quads;
        if (jg < G)
            stream_panel4<FS, AT>(static_cast<const FS*>(op.far_pool) + gr.voff + w.r0 + 4 * q, gr.ld, gr.n, jg, G,
                                  nullptr, x, acc, gr.c0);
    } else {
        const Tile t = op.tiles[-code - 1];
        quads = t.ld / 4;
        G = 256 / quads;
        rows = t.rows;
        const int q = threadIdx.x % quads, g = threadIdx.x / quads;
        if (g < G)
            stream_panel4<NS, AT>(static_cast<const NS*>(op.near_pool) + t.noff + 4 * q, t.ld, t.kn, g, G,
                                  op.xidx + t.ixn, x, acc);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) part[4 * threadIdx.x + r] = acc[r];
    __syncthreads();
    if ((int)threadIdx.x < rows) {
        const int rr = threadIdx.x;
        AT sum = 0;
        for (int g = 0; g < G; ++g) sum += part[4 * (g * quads) + rr];
        if (code >= 0) {
            const GWork w = op.sitems[code];
            T[op.groups[w.g].toff + w.r0 + rr] = sum;
        } else {
            Yn[op.tiles[-code - 1].r0 + rr] = sum;
        }
    }
}

template <class NS, class FS, class AT>
__global__ void __launch_bounds__(256) single_phase_a(OpView op, const AT* __restrict__ x, AT* __restrict__ T, AT* __restrict__ Yn) {
    // grid-stride over the work items: one CTA per item, or a persistent grid
    for (int it = blockIdx.x; it < op.n_aitems; it += gridDim.x) {
        single_phase_a_item<NS, FS, AT>(it, op, x, T, Yn);
        __syncthreads();
    }
}


template <class FS, class AT>
__device__ __forceinline__ void
single_phase_b_item(int it_, OpView op, const AT* __restrict__ T, const AT* __restrict__ Yn, void* Y, Epi epi) {
    __shared__ AT part[1024];
    const Tile t = op.tiles[op.forder[it_]];
    const int quads = t.ld / 4;
    const int G = 256 / quads;
    const int q = threadIdx.x % quads, g = threadIdx.x / quads;
    AT acc[4] = {0, 0, 0, 0};
    if (g < G && t.kf > 0)
        stream_panel4<FS, AT>(static_cast<const FS*>(op.far_pool) + t.foff + 4 * q, t.ld, t.kf, g, G,
                              op.tidx + t.ixf, T, acc);
#pragma unroll
    for (int r = 0; r < 4; ++r) part[4 * threadIdx.x + r] = acc[r];
    __syncthreads();
    if ((int)threadIdx.x < t.rows) {
        const int row = threadIdx.x;
        AT s = Yn[t.r0 + row];
        for (int gg = 0; gg < G; ++gg) s += part[4 * (gg * quads) + row];
        epilogue<AT>(epi, Y, 1, t.r0 + row, 0, s);
    }
}

template <class FS, class AT>
__global__ void __launch_bounds__(256) single_phase_b(OpView op, const AT* __restrict__ T, const AT* __restrict__ Yn, void* Y, Epi epi) {
    // grid-stride over the work items: one CTA per item, or a persistent grid
    for (int it = blockIdx.x; it < op.n_tiles; it += gridDim.x) {
        single_phase_b_item<FS, AT>(it, op, T, Yn, Y, epi);
        __syncthreads();
    }
}


template <class NS, class FS, class AT, int NCOL>
__device__ __forceinline__ void
rows_stream_item(int it_, OpView op, const AT* __restrict__ X, int ldx, const AT* __restrict__ T, int ldt, void* Y, int ldy,
            Epi epi) {
    __shared__ AT part[NCOL][1024];
    const Tile t = op.tiles[op.torder[it_]];
    const int quads = t.ld / 4;
    const int G = 256 / quads;
    const int q = threadIdx.x % quads, g = threadIdx.x / quads;
    AT acc[NCOL][4] = {};
    if (g < G) {
        stream_cols<NS, AT, NCOL>(static_cast<const NS*>(op.near_pool) + t.noff + 4 * q, t.ld, t.kn, g, G,
                                  op.xidx + t.ixn, X, ldx, acc);
        stream_cols<FS, AT, NCOL>(static_cast<const FS*>(op.far_pool) + t.foff + 4 * q, t.ld, t.kf, g, G,
                                  op.tidx + t.ixf, T, ldt, acc);
    }
#pragma unroll
    for (int c = 0; c < NCOL; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) part[c][4 * threadIdx.x + r] = acc[c][r];
    __syncthreads();
    if ((int)threadIdx.x < t.rows) {
        const int row = threadIdx.x;
#pragma unroll
        for (int c = 0; c < NCOL; ++c) {
            AT sum = 0;
            for (int gg = 0; gg < G; ++gg) sum += part[c][4 * (gg * quads) + row];
            epilogue<AT>(epi, Y, ldy, t.r0 + row, c, sum);
        }
    }
}

template <class NS, class FS, class AT, int NCOL>
__global__ void __launch_bounds__(256) rows_stream(OpView op, const AT* __restrict__ X, int ldx, const AT* __restrict__ T, int ldt, void* Y, int ldy, Epi epi) {
    // grid-stride over the work items: one CTA per item, or a persistent grid
    for (int it = blockIdx.x; it < op.n_tiles; it += gridDim.x) {
        rows_stream_item<NS, FS, AT, NCOL>(it, op, X, ldx, T, ldt, Y, ldy, epi);
        __syncthreads();
    }
}


// ---------------------------------------------------------------- double-float
// FP64-grade sums on the FP32 pipe (GB300's FP64 pipe is narrow): a value is
// an unevaluated pair hi + lo of floats; products of a stored FP32 entry with
// a pair use the exact FMA product error, sums the error-free two-sum.
struct DF {
    float h, l;
};
__device__ __forceinline__ void df_fma(DF& acc, float a, const DF& x) {
    const float p = __fmul_rn(a, x.h);
    const float pe = __fmaf_rn(a, x.h, -p);                 // a*x.h - p, exactly
    const float s = __fadd_rn(acc.h, p);
    const float bp = __fsub_rn(s, acc.h);
    const float se = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    acc.h = s;
    acc.l = __fadd_rn(acc.l, __fadd_rn(__fadd_rn(se, pe), __fmul_rn(a, x.l)));
}
__device__ __forceinline__ DF df_norm(DF v) {
    const float s = __fadd_rn(v.h, v.l);
    return DF{s, __fsub_rn(v.l, __fsub_rn(s, v.h))};
}

__global__ void to_df_kernel(const double* __restrict__ X, int ldx, int n, int nc, DF* __restrict__ out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * nc) return;
    const int p = (int)(e / nc), c = (int)(e - (long long)p * nc);
    const double x = X[(long long)p * ldx + c];
    const float h = __double2float_rn(x);
    out[e] = DF{h, __double2float_rn(x - (double)h)};
}

// Double-float counterpart of stream_cols (idx null: rows base + c): the
// loads of four panel columns are issued together, the double-float updates
// then run in column order (the same arithmetic as one column at a time).
template <int NCOL>
__device__ __forceinline__ void stream_cols_df(const float* __restrict__ P, long long ld, int kcols, int g, int G,
                                               const int* __restrict__ idx, const DF* __restrict__ V,
                                               DF (&acc)[NCOL][4], int base = 0) {
    constexpr int U = 4;
    int c = g;
    for (; c + (U - 1) * G < kcols; c += U * G) {
        float a[U][4];
        const DF* vr[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            Vec4<float, float>::load(P + (long long)(c + u * G) * ld, a[u]);
            vr[u] = V + (long long)(idx ? idx[c + u * G] : base + c + u * G) * NCOL;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int k = 0; k < NCOL; ++k) {
                const DF xv = vr[u][k];
#pragma unroll
                for (int r = 0; r < 4; ++r) df_fma(acc[k][r], a[u][r], xv);
            }
    }
    for (; c < kcols; c += G) {
        float a[4];
        Vec4<float, float>::load(P + (long long)c * ld, a);
        const DF* vr = V + (long long)(idx ? idx[c] : base + c) * NCOL;
#pragma unroll
        for (int k = 0; k < NCOL; ++k) {
            const DF xv = vr[k];
#pragma unroll
            for (int r = 0; r < 4; ++r) df_fma(acc[k][r], a[r], xv);
        }
    }
}

template <int NCOL>
__global__ void __launch_bounds__(256) far_vt_df(OpView op, const DF* __restrict__ X, DF* __restrict__ T) {
    __shared__ DF part[NCOL][1024];
    const GWork w = op.sitems[blockIdx.x];
    const Group gr = op.groups[w.g];
    const int quads = (w.rows + 3) / 4;
    const int G = 256 / quads;
    const int q = threadIdx.x % quads, jg = threadIdx.x / quads;
    const long long ld = gr.ld;
    DF acc[NCOL][4];
#pragma unroll
    for (int c = 0; c < NCOL; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[c][r] = DF{0.0f, 0.0f};
    if (jg < G)
        stream_cols_df<NCOL>(static_cast<const float*>(op.far_pool) + gr.voff + w.r0 + 4 * q, ld, gr.n, jg, G,
                             nullptr, X, acc, gr.c0);
#pragma unroll
    for (int c = 0; c < NCOL; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) part[c][4 * threadIdx.x + r] = df_norm(acc[c][r]);
    __syncthreads();
    if ((int)threadIdx.x < w.rows) {
        const int rr = threadIdx.x;
#pragma unroll
        for (int c = 0; c < NCOL; ++c) {
            double sum = 0.0;
            for (int g = 0; g < G; ++g) {
                const DF d = part[c][4 * (g * quads) + rr];
                sum += (double)d.h + (double)d.l;
            }
            const float hi = __double2float_rn(sum);
            T[(long long)(gr.toff + w.r0 + rr) * NCOL + c] = DF{hi, __double2float_rn(sum - (double)hi)};
        }
    }
}

template <int NCOL>
__global__ void __launch_bounds__(256)
rows_df(OpView op, const DF* __restrict__ X, const DF* __restrict__ T, double* Y, int ldy, Epi epi) {
    __shared__ DF part[NCOL][1024];
    const Tile t = op.tiles[op.torder[blockIdx.x]];
    const int quads = t.ld / 4;
    const int G = 256 / quads;
    const int q = threadIdx.x % quads, g = threadIdx.x / quads;
    DF acc[NCOL][4];
#pragma unroll
    for (int c = 0; c < NCOL; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[c][r] = DF{0.0f, 0.0f};
    if (g < G) {
        stream_cols_df<NCOL>(static_cast<const float*>(op.near_pool) + t.noff + 4 * q, t.ld, t.kn, g, G,
                             op.xidx + t.ixn, X, acc);
        stream_cols_df<NCOL>(static_cast<const float*>(op.far_pool) + t.foff + 4 * q, t.ld, t.kf, g, G,
                             op.tidx + t.ixf, T, acc);
    }
#pragma unroll
    for (int c = 0; c < NCOL; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) part[c][4 * threadIdx.x + r] = df_norm(acc[c][r]);
    __syncthreads();
    if ((int)threadIdx.x < t.rows) {
        const int row = threadIdx.x;
#pragma unroll
        for (int c = 0; c < NCOL; ++c) {
            double sum = 0.0;
            for (int gg = 0; gg < G; ++gg) {
                const DF d = part[c][4 * (gg * quads) + row];
                sum += (double)d.h + (double)d.l;
            }
            epilogue<double>(epi, Y, ldy, t.r0 + row, c, sum);
        }
    }
}

// ---------------------------------------------------------------- many RHS
template <class AT> struct Chunk;
template <> struct Chunk<float> { static constexpr int KC = 32; };
template <> struct Chunk<double> { static constexpr int KC = 16; };
constexpr int kMaxCols = 96;    // right-hand sides per launch (multiple of 4)
constexpr int kStages = 3;
constexpr int kRPT = 8;         // panel rows per thread of the many-column GEMM (divides 64)

// Copy unit of the panel operand: 16 bytes (FP32, FP64) or 8 bytes (BF16,
// whose panel columns are only 8-byte aligned).
template <class S> struct AUnit { static constexpr int bytes = 16; };
template <> struct AUnit<__nv_bfloat16> { static constexpr int bytes = 8; };

// Dynamic shared memory of the panel GEMM: kStages x (A chunk: KC panel
// columns of up to 64 rows; B chunk: KC rows of 4 CQ columns).
template <class AS, class AT>
struct GemmLayout {
    static constexpr int KC = Chunk<AT>::KC;
    static constexpr size_t a_bytes = sizeof(AS) * KC * kTileRows;
    static __host__ __device__ size_t stage(int cq) { return (a_bytes + sizeof(AT) * KC * 4 * cq + 127) / 128 * 128; }
    static __host__ __device__ size_t bytes(int cq) { return kStages * stage(cq); }
};

// asynchronous global -> shared copies; a false predicate copies nothing and
// fills the destination with zeros
__device__ __forceinline__ void cp_async_16(void* sdst, const void* gsrc, bool pred) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gsrc), "r"(pred ? 16 : 0));
}
__device__ __forceinline__ void cp_async_8(void* sdst, const void* gsrc, bool pred) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gsrc), "r"(pred ? 8 : 0));
}
__device__ __forceinline__ void cp_async_4(void* sdst, const void* gsrc, bool pred) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gsrc), "r"(pred ? 4 : 0));
}
template <int B>
__device__ __forceinline__ void cp_async_n(void* d, const void* g, bool p) {
    if constexpr (B == 16) cp_async_16(d, g, p);
    else if constexpr (B == 8) cp_async_8(d, g, p);
    else cp_async_4(d, g, p);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Four consecutive accumulation-type values from shared memory.
template <class AT> struct Quad;
template <> struct Quad<float> {
    static __device__ __forceinline__ void load(const float* p, float v[4]) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
};
template <> struct Quad<double> {
    static __device__ __forceinline__ void load(const double* p, double v[4]) {
        const double2 a = reinterpret_cast<const double2*>(p)[0];
        const double2 b = reinterpret_cast<const double2*>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};

// acc(kRPT x 4 per thread) += A(rows x K) B(K x nc).  A: column-major
// panel (leading dimension lda, a chunk of rows_pad <= 64 rows, rows_pad a
// multiple of 4; rows up to the next multiple of kRPT are zero-filled);
// B(k, :) = row bsel(k) of the vector block Bv (leading dimension ldb).
// Thread (rg, cq) = (tid / CQ, tid % CQ) owns rows kRPT rg .. kRPT rg +
// kRPT - 1 and columns 4 cq .. 4 cq + 3; per k it reads kRPT / 4 quads of A
// and one quad of B from shared memory (lanes of a row group share the A
// quads) for 4 kRPT FMAs.
// Chunks of KC panel columns and the KC matching rows of B go through a
// kStages-deep cp.async ring; B rows move as 16-byte quads when VB (rows
// 16-byte aligned, padded to 4 CQ columns), else element by element with
// zero fill past nc.
template <class AS, class AT, bool VB, class BSel>
__device__ __forceinline__ void panel_gemm(AT (&acc)[kRPT][4], unsigned char* smem, const AS* __restrict__ A,
                                           long long lda, int rows_pad, int K, BSel bsel,
                                           const AT* __restrict__ Bv, int ldb, int nc, int CQ) {
    using L = GemmLayout<AS, AT>;
    constexpr int KC = L::KC;
    constexpr int AU = AUnit<AS>::bytes;
    constexpr int EPU = AU / (int)sizeof(AS);            // A elements per copy unit
    const int nchunks = (K + KC - 1) / KC;
    if (nchunks == 0) return;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int rg = tid / CQ, cq = tid - rg * CQ;
    const int rows_up = (rows_pad + kRPT - 1) / kRPT * kRPT;
    const bool active = rg < rows_up / kRPT;
    const int BS = 4 * CQ;                               // B row stride in shared memory
    const size_t stage = L::stage(CQ);
    const int upc = rows_up / EPU;                       // A copy units per panel column
    const int upv = rows_pad / EPU;                      // ... of which hold panel rows
    // A thread's copy units are the same in every chunk: unit u = tid + i nt
    // is panel column u / upc, piece u % upc of the A chunk, and row u / CQ,
    // quad u % CQ of the B chunk.  The divisions are done once here; the
    // chunk loop only steps through them.
    const int a_k0 = tid / upc, a_w0 = tid - a_k0 * upc;
    const int a_dk = nt / upc, a_dw = nt - a_dk * upc;
    const int a_units = KC * upc;
    // gathered B rows of this thread's copy units of the next chunk to
    // issue, loaded one chunk ahead so that the index loads do not stall
    // the copies (16-byte B rows only; at most KC kRPT / 64 units a thread)
    constexpr int kBU = (KC * kRPT + 63) / 64;
    int brow[kBU];
    int bkk[kBU], bq[kBU];
#pragma unroll
    for (int i = 0; i < kBU; ++i) {
        const int u = tid + i * nt;
        bkk[i] = u < KC * CQ ? u / CQ : KC;              // KC: no unit
        bq[i] = u - (u / CQ) * CQ;
    }
    auto load_rows = [&](int ch) {
        if constexpr (VB) {
            const int k0 = ch * KC;
#pragma unroll
            for (int i = 0; i < kBU; ++i) brow[i] = (bkk[i] < KC && k0 + bkk[i] < K) ? bsel(k0 + bkk[i]) : 0;
        }
    };
    auto issue = [&](int ch) {
        unsigned char* st = smem + (size_t)(ch % kStages) * stage;
        AS* As = reinterpret_cast<AS*>(st);
        AT* Bs = reinterpret_cast<AT*>(st + L::a_bytes);
        const int k0 = ch * KC;
        const AS* Ak = A + (long long)k0 * lda;
        for (int u = tid, kk = a_k0, w = a_w0; u < a_units; u += nt) {
            const bool ok = k0 + kk < K && w < upv;
            const AS* src = ok ? Ak + (long long)kk * lda + w * EPU : A;
            cp_async_n<AU>(As + kk * kTileRows + w * EPU, src, ok);
            kk += a_dk;
            w += a_dw;
            if (w >= upc) {
                w -= upc;
                ++kk;
            }
        }
        if constexpr (VB) {
#pragma unroll
            for (int i = 0; i < kBU; ++i) {
                if (bkk[i] >= KC) break;
                const bool ok = k0 + bkk[i] < K;
                const AT* src = ok ? Bv + (long long)brow[i] * ldb + 4 * bq[i] : Bv;
                cp_async_16(Bs + bkk[i] * BS + 4 * bq[i], src, ok);
            }
        } else {
            for (int u = tid; u < KC * BS; u += nt) {
                const int kk = u / BS, c = u - kk * BS;
                const bool ok = k0 + kk < K && c < nc;
                const AT* src = ok ? Bv + (long long)bsel(k0 + kk) * ldb + c : Bv;
                cp_async_n<(int)sizeof(AT)>(Bs + kk * BS + c, src, ok);
            }
        }
        cp_async_commit();
    };
    load_rows(0);
    issue(0);
    load_rows(1);
    if (nchunks > 1) issue(1);
    else cp_async_commit();
    load_rows(2);
    for (int ch = 0; ch < nchunks; ++ch) {
        cp_async_wait<kStages - 2>();
        __syncthreads();
        if (ch + 2 < nchunks) {
            issue(ch + 2);
            load_rows(ch + 3);
        } else {
            cp_async_commit();
        }
        if (active) {
            const unsigned char* st = smem + (size_t)(ch % kStages) * stage;
            const AS* As = reinterpret_cast<const AS*>(st);
            const AT* Bs = reinterpret_cast<const AT*>(st + L::a_bytes);
            // chunk entries past K were filled with zeros
#pragma unroll 8
            for (int kk = 0; kk < KC; ++kk) {
                AT a[kRPT], b[4];
#pragma unroll
                for (int h = 0; h < kRPT / 4; ++h) Vec4<AS, AT>::load(As + kk * kTileRows + rg * kRPT + 4 * h, a + 4 * h);
                Quad<AT>::load(Bs + kk * BS + 4 * cq, b);
#pragma unroll
                for (int r = 0; r < kRPT; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] += a[r] * b[c];
            }
        }
    }
    cp_async_wait<0>();
    __syncthreads();
}

struct AffineRows {
    int base;
    __device__ __forceinline__ int operator()(int k) const { return base + k; }
};
struct IndexRows {
    const int* idx;
    __device__ __forceinline__ int operator()(int k) const { return idx[k]; }
};

template <class FS, class AT, bool VB>
__global__ void __launch_bounds__(384)
far_vt_multi(OpView op, const AT* __restrict__ X, int ldx, AT* __restrict__ T, int ldt, int nc, int CQ) {
    extern __shared__ __align__(128) unsigned char dsm[];
    const GWork w = op.gwork[blockIdx.x];
    const Group gr = op.groups[w.g];
    const int rows_pad = (w.rows + 3) / 4 * 4;
    AT acc[kRPT][4] = {};
    panel_gemm<FS, AT, VB>(acc, dsm, static_cast<const FS*>(op.far_pool) + gr.voff + w.r0, gr.ld, rows_pad, gr.n,
                           AffineRows{gr.c0}, X, ldx, nc, CQ);
    const int rg = threadIdx.x / CQ, cq = threadIdx.x - rg * CQ;
#pragma unroll
    for (int r = 0; r < kRPT; ++r) {
        const int row = rg * kRPT + r;
        if (row >= w.rows) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int col = 4 * cq + c;
            if (col < nc) T[(long long)(gr.toff + w.r0 + row) * ldt + col] = acc[r][c];
        }
    }
}

template <class NS, class FS, class AT, bool VB>
__global__ void __launch_bounds__(384)
rows_multi(OpView op, const AT* __restrict__ X, int ldx, const AT* __restrict__ T, int ldt, void* Y, int ldy, int nc,
           int CQ, Epi epi) {
    extern __shared__ __align__(128) unsigned char dsm[];
    const Tile t = op.tiles[op.torder[blockIdx.x]];
    AT acc[kRPT][4] = {};
    panel_gemm<NS, AT, VB>(acc, dsm, static_cast<const NS*>(op.near_pool) + t.noff, t.ld, t.ld, t.kn,
                           IndexRows{op.xidx + t.ixn}, X, ldx, nc, CQ);
    // T rows are always padded to a multiple of 4 columns and 16-byte aligned
    panel_gemm<FS, AT, std::is_same<AT, float>::value>(acc, dsm, static_cast<const FS*>(op.far_pool) + t.foff, t.ld,
                                                       t.ld, t.kf, IndexRows{op.tidx + t.ixf}, T, ldt, nc, CQ);
    const int rg = threadIdx.x / CQ, cq = threadIdx.x - rg * CQ;
#pragma unroll
    for (int r = 0; r < kRPT; ++r) {
        const int row = rg * kRPT + r;
        if (row >= t.rows) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int col = 4 * cq + c;
            if (col < nc) epilogue<AT>(epi, Y, ldy, t.r0 + row, col, acc[r][c]);
        }
    }
}

// Threads of the panel GEMM for nc columns: 64 / kRPT row groups x
// ceil(nc / 4) column quads, rounded up to whole warps.
inline int gemm_threads(int cq) { return (64 / kRPT * cq + 31) / 32 * 32; }

template <class FS, class AT, bool VB>
void launch_far_vt(const OpView& op, const AT* X, int ldx, AT* T, int ldt, int nc, cudaStream_t s) {
    const int cq = (nc + 3) / 4;
    const size_t bytes = GemmLayout<FS, AT>::bytes(cq);
    static std::once_flag configured;
    std::call_once(configured, [&] {
        RAD_CUDA(cudaFuncSetAttribute(far_vt_multi<FS, AT, VB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)GemmLayout<FS, AT>::bytes(kMaxCols / 4)));
    });
    { ProfScope ps_("hmm_far_vt", s); far_vt_multi<FS, AT, VB><<<op.n_gwork, gemm_threads(cq), bytes, s>>>(op, X, ldx, T, ldt, nc, cq); }
    RAD_CHECK_LAUNCH();
}
template <class NS, class FS, class AT, bool VB>
void launch_rows(const OpView& op, const AT* X, int ldx, const AT* T, int ldt, void* Y, int ldy, int nc,
                 const Epi& epi, cudaStream_t s) {
    const int cq = (nc + 3) / 4;
    const size_t bytes = std::max(GemmLayout<NS, AT>::bytes(cq), GemmLayout<FS, AT>::bytes(cq));
    static std::once_flag configured;
    std::call_once(configured, [&] {
        const size_t mx = std::max(GemmLayout<NS, AT>::bytes(kMaxCols / 4), GemmLayout<FS, AT>::bytes(kMaxCols / 4));
        RAD_CUDA(cudaFuncSetAttribute(rows_multi<NS, FS, AT, VB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx));
    });
    { ProfScope ps_("hmm_rows", s); rows_multi<NS, FS, AT, VB><<<op.n_tiles, gemm_threads(cq), bytes, s>>>(op, X, ldx, T, ldt, Y, ldy, nc, cq, epi); }
    RAD_CHECK_LAUNCH();
}

// Grid of a grid-stride launch over `items` work items: one CTA per item, or
// the tuned persistent size.
inline unsigned grid_of(int tuned, int items) {
    return (unsigned)std::max(1, tuned > 0 ? std::min(tuned, items) : items);
}

template <class NS, class FS, class AT, int NCOL>
void launch_stream(const rad_htree* h, const OpView& op, const AT* X, int ldx, AT* T, int ldt, void* Y, int ldy,
                   const Epi& epi, cudaStream_t s) {
    if (op.n_gwork > 0) {
        { ProfScope ps_("hmv_far_vt", s); far_vt_stream<FS, AT, NCOL><<<grid_of(h->grid_a2, op.n_sitems), 256, 0, s>>>(op, X, ldx, T, ldt); }
        RAD_CHECK_LAUNCH();
    }
    { ProfScope ps_("hmv_rows", s); rows_stream<NS, FS, AT, NCOL><<<grid_of(h->grid_b2, op.n_tiles), 256, 0, s>>>(op, X, ldx, T, ldt, Y, ldy, epi); }
    RAD_CHECK_LAUNCH();
}

template <int NCOL>
void launch_df(const rad_htree* h, const OpView& op, const double* X, int ldx, double* Y, int ldy, int nrhs,
               const Epi& epi, double* T_ws, cudaStream_t s) {
    // the double-float copies of X and T share the T workspace
    const int n = (int)h->n;
    DF* Xd = reinterpret_cast<DF*>(T_ws);
    DF* Td = Xd + (size_t)n * NCOL;
    const long long cnt = (long long)n * nrhs;
    { ProfScope ps_("permute", s); to_df_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(X, ldx, n, NCOL, Xd); }
    RAD_CHECK_LAUNCH();
    if (op.n_gwork > 0) {
        { ProfScope ps_("hmv_far_vt", s); far_vt_df<NCOL><<<(unsigned)op.n_sitems, 256, 0, s>>>(op, Xd, Td); }
        RAD_CHECK_LAUNCH();
    }
    { ProfScope ps_("hmv_rows", s); rows_df<NCOL><<<op.n_tiles, 256, 0, s>>>(op, Xd, Td, Y, ldy, epi); }
    RAD_CHECK_LAUNCH();
}

template <class NS, class FS, class AT>
void apply_t(const rad_htree* h, const OpView& op, const AT* X, int ldx, void* Y, int ldy, int nrhs, const Epi& epi,
             AT* T, cudaStream_t s) {
    if (nrhs == 1) {
        AT* Yn = T + std::max(1, op.sum_rank);
        if constexpr (std::is_same<AT, float>::value && std::is_same<NS, float>::value) {
            if (h->one_col_path == 1 && h->hmv1_ok) {
                // the fused launch's two counters follow Yn, 16-byte aligned
                const uintptr_t c = (reinterpret_cast<uintptr_t>(Yn + h->n) + 15) & ~(uintptr_t)15;
                hmv1_product(h, X, T, Yn, reinterpret_cast<int*>(c), Y, epi, s);
                return;
            }
        }
        { ProfScope ps_("hmv_phase_a", s); single_phase_a<NS, FS, AT><<<grid_of(h->grid_a1, op.n_aitems), 256, 0, s>>>(op, X, T, Yn); }
        RAD_CHECK_LAUNCH();
        { ProfScope ps_("hmv_phase_b", s); single_phase_b<FS, AT><<<grid_of(h->grid_b1, op.n_tiles), 256, 0, s>>>(op, T, Yn, Y, epi); }
        RAD_CHECK_LAUNCH();
        return;
    }
    if (nrhs <= 4) {
        const int ldt = tree_ld(nrhs);
        switch (nrhs) {
            case 2: launch_stream<NS, FS, AT, 2>(h, op, X, ldx, T, ldt, Y, ldy, epi, s); break;
            case 3: launch_stream<NS, FS, AT, 3>(h, op, X, ldx, T, ldt, Y, ldy, epi, s); break;
            default: launch_stream<NS, FS, AT, 4>(h, op, X, ldx, T, ldt, Y, ldy, epi, s); break;
        }
        return;
    }
    const int ldt = tree_ld(nrhs);
    const int esz = epi.mode == kStore ? (int)sizeof(AT) : 8;
    // X rows move as 16-byte quads when they are FP32, 16-byte aligned and
    // padded to a multiple of 4 columns
    const bool vx = std::is_same<AT, float>::value && ldx % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
    for (int c0 = 0; c0 < nrhs; c0 += kMaxCols) {
        const int nc = std::min(kMaxCols, nrhs - c0);
        Epi e2 = epi;
        if (epi.mode != kStore) {
            e2.xin = epi.xin + c0;
            if (epi.b) e2.b = epi.b + c0;
        }
        const AT* Xc = X + c0;
        AT* Tc = T + c0;
        void* Yc = static_cast<char*>(Y) + (size_t)c0 * esz;
        if constexpr (std::is_same<AT, float>::value && std::is_same<NS, float>::value) {
            if (h->mm_path == 1 && h->tc_ready) {
                // tensor cores (BF16 x 3 split) for FP32 vectors; their
                // workspace follows the FP32 T block
                void* tws = reinterpret_cast<char*>(T) + sizeof(AT) * (size_t)std::max(1, op.sum_rank) * ldt;
                tc_product(h, op, Xc, ldx, Yc, ldy, nc, e2, tws, s);
                continue;
            }
        }
        if (vx) {
            if (op.n_gwork > 0) launch_far_vt<FS, AT, true>(op, Xc, ldx, Tc, ldt, nc, s);
            launch_rows<NS, FS, AT, true>(op, Xc, ldx, Tc, ldt, Yc, ldy, nc, e2, s);
        } else {
            if (op.n_gwork > 0) launch_far_vt<FS, AT, false>(op, Xc, ldx, Tc, ldt, nc, s);
            launch_rows<NS, FS, AT, false>(op, Xc, ldx, Tc, ldt, Yc, ldy, nc, e2, s);
        }
    }
}

// ---------------------------------------------------------------- permutation
template <class TI, class TO>
__global__ void gather_kernel(int n, int nrhs, const TI* __restrict__ x, long long ldx, const int* __restrict__ perm,
                              TO* __restrict__ X, int ldX) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * nrhs) return;
    const int p = (int)(e / nrhs), c = (int)(e - (long long)p * nrhs);
    X[(long long)p * ldX + c] = (TO)x[perm[p] + (long long)c * ldx];
}
template <class TI, class TO>
__global__ void scatter_kernel(int n, int nrhs, const TI* __restrict__ Y, int ldY, const int* __restrict__ perm,
                               TO* __restrict__ y, long long ldy) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * nrhs) return;
    const int p = (int)(e / nrhs), c = (int)(e - (long long)p * nrhs);
    y[perm[p] + (long long)c * ldy] = (TO)Y[(long long)p * ldY + c];
}

}  // namespace

size_t apply_workspace_bytes(const rad_htree* h, int nrhs) {
    const size_t esz = h->op_is_f64() ? 8 : 4;
    // T = V^T X, plus (one column) the dense-panel partial sums and 16
    // elements holding the fused launch's counters, plus the split vector
    // planes of the tensor-core path
    const size_t tc = nrhs >= 5 && h->mm_path == 1 && !h->op_is_f64() ? tc_workspace_bytes(h, nrhs) : 0;
    return esz * ((size_t)std::max(1, h->sum_rank) * (size_t)tree_ld(nrhs) + (nrhs == 1 ? (size_t)h->n + 16 : 0)) +
           tc;
}

void apply_tree(const rad_htree* h, const void* X, int ldx, void* Y, int ldy, int nrhs, const Epi& epi,
                void* T_ws, cudaStream_t s) {
    const OpView op = h->view();
    if (h->op_is_f64()) {
        apply_t<double, double, double>(h, op, static_cast<const double*>(X), ldx, Y, ldy, nrhs, epi,
                                        static_cast<double*>(T_ws), s);
    } else if (h->factor_dtype == RAD_F32) {
        apply_t<float, float, float>(h, op, static_cast<const float*>(X), ldx, Y, ldy, nrhs, epi,
                                     static_cast<float*>(T_ws), s);
    } else {
        apply_t<float, __nv_bfloat16, float>(h, op, static_cast<const float*>(X), ldx, Y, ldy, nrhs, epi,
                                             static_cast<float*>(T_ws), s);
    }
}

size_t apply_workspace_bytes_acc(const rad_htree* h, int nrhs) {
    const size_t gemm = sizeof(double) * (size_t)std::max(1, h->sum_rank) * (size_t)tree_ld(nrhs);
    const size_t df = sizeof(DF) * (size_t)4 * ((size_t)h->n + (size_t)std::max(1, h->sum_rank));
    return std::max(gemm, df);
}

void apply_tree_acc(const rad_htree* h, const double* X, int ldx, double* Y, int ldy, int nrhs, const Epi& epi,
                    double* T_ws, cudaStream_t s) {
    RAD_REQUIRE(h->has_accurate, RAD_EINVAL, "no accurate operator (compress with accurate_dtype = RAD_F32)");
    if (h->op_is_f64()) {
        apply_t<double, double, double>(h, h->view(), X, ldx, Y, ldy, nrhs, epi, T_ws, s);
        return;
    }
    OpView op = h->view();
    op.far_pool = h->accurate_far_pool();
    if (nrhs <= 4) {
        // FP64-grade accumulation on the FP32 pipe
        switch (nrhs) {
            case 1: launch_df<1>(h, op, X, ldx, Y, ldy, nrhs, epi, T_ws, s); break;
            case 2: launch_df<2>(h, op, X, ldx, Y, ldy, nrhs, epi, T_ws, s); break;
            case 3: launch_df<3>(h, op, X, ldx, Y, ldy, nrhs, epi, T_ws, s); break;
            default: launch_df<4>(h, op, X, ldx, Y, ldy, nrhs, epi, T_ws, s); break;
        }
        return;
    }
    apply_t<float, float, double>(h, op, X, ldx, Y, ldy, nrhs, epi, T_ws, s);
}

void gather_user_to_tree(const rad_htree* h, int dtype_in, const void* x, int64_t ldx, int nrhs, void* X, int ldX,
                         bool op64, cudaStream_t s) {
    const int n = (int)h->n;
    const long long tot = (long long)n * nrhs;
    const unsigned grid = (unsigned)((tot + 255) / 256);
    const int* perm = h->perm.as<int>();
    if (dtype_in == RAD_F64) {
        if (op64) { ProfScope ps_("permute", s); gather_kernel<double, double><<<grid, 256, 0, s>>>(n, nrhs, (const double*)x, ldx, perm, (double*)X, ldX); }
        else { ProfScope ps_("permute", s); gather_kernel<double, float><<<grid, 256, 0, s>>>(n, nrhs, (const double*)x, ldx, perm, (float*)X, ldX); }
    } else {
        if (op64) { ProfScope ps_("permute", s); gather_kernel<float, double><<<grid, 256, 0, s>>>(n, nrhs, (const float*)x, ldx, perm, (double*)X, ldX); }
        else { ProfScope ps_("permute", s); gather_kernel<float, float><<<grid, 256, 0, s>>>(n, nrhs, (const float*)x, ldx, perm, (float*)X, ldX); }
    }
    RAD_CHECK_LAUNCH();
}

void scatter_tree_to_user(const rad_htree* h, const void* Y, int ldY, int nrhs, bool op64, int dtype_out, void* y,
                          int64_t ldy, cudaStream_t s) {
    const int n = (int)h->n;
    const long long tot = (long long)n * nrhs;
    const unsigned grid = (unsigned)((tot + 255) / 256);
    const int* perm = h->perm.as<int>();
    if (dtype_out == RAD_F64) {
        if (op64) { ProfScope ps_("permute", s); scatter_kernel<double, double><<<grid, 256, 0, s>>>(n, nrhs, (const double*)Y, ldY, perm, (double*)y, ldy); }
        else { ProfScope ps_("permute", s); scatter_kernel<float, double><<<grid, 256, 0, s>>>(n, nrhs, (const float*)Y, ldY, perm, (double*)y, ldy); }
    } else {
        if (op64) { ProfScope ps_("permute", s); scatter_kernel<double, float><<<grid, 256, 0, s>>>(n, nrhs, (const double*)Y, ldY, perm, (float*)y, ldy); }
        else { ProfScope ps_("permute", s); scatter_kernel<float, float><<<grid, 256, 0, s>>>(n, nrhs, (const float*)Y, ldY, perm, (float*)y, ldy); }
    }
    RAD_CHECK_LAUNCH();
}


// ---------------------------------------------------------------- closed cavity
// §6 closed-cavity rows: s = F 1 with the stored operator, c = clamp(s, 0, 1),
// row i of F divided by c_i when c_i != 0.  The operator is stored by rows in
// the tile panels (dense panel and U panel; V is shared by all rows of a
// block), so the scaling multiplies the tile rows of both panels (and of the
// FP32 accurate copy of U when kept).
namespace {

template <class T>
__global__ void fill_kernel(T* x, long long cnt, T v) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < cnt) x[e] = v;
}

template <class T>
__global__ void row_scale_kernel(const T* __restrict__ sums, int n, double* __restrict__ s64,
                                 double* __restrict__ scale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double si = (double)sums[i];
    const double c = si < 0.0 ? 0.0 : (si > 1.0 ? 1.0 : si);
    s64[i] = si;
    scale[i] = c != 0.0 ? 1.0 / c : 1.0;
}

template <class S>
__global__ void __launch_bounds__(256)
scale_panel_kernel(const Tile* __restrict__ tiles, int far, const double* __restrict__ scale, S* pool) {
    const Tile t = tiles[blockIdx.x];
    const int k = far ? t.kf : t.kn;
    S* P = pool + (far ? t.foff : t.noff);
    const long long cnt = (long long)k * t.ld;
    for (long long e = threadIdx.x; e < cnt; e += 256) {
        const int r = (int)(e % t.ld);
        if (r < t.rows) P[e] = Store<S>::put((double)Store<S>::get(P[e]) * scale[t.r0 + r]);
    }
}

template <class S>
void scale_panels(const rad_htree* h, int far, const double* scale, void* pool, cudaStream_t s) {
    if (h->n_tiles == 0) return;
    { ProfScope ps_("close_cavity", s); scale_panel_kernel<S><<<h->n_tiles, 256, 0, s>>>(h->d_tiles.as<Tile>(), far, scale, static_cast<S*>(pool)); }
    RAD_CHECK_LAUNCH();
}

}  // namespace

void close_cavity(rad_htree* h, double* s_tree_out, cudaStream_t s) {
    RAD_REQUIRE(h->compressed, RAD_EINVAL, "handle is not compressed (call rad_compress_aca)");
    Scratch ws(s);
    const int n = (int)h->n;
    const unsigned g = (unsigned)((n + 255) / 256);
    double* S64 = s_tree_out;
    double* scale = ws.get_n<double>(n);
    const Epi st{kStore, nullptr, nullptr, nullptr, 0};
    if (h->op_is_f64() || h->has_accurate) {
        // FP64 operator, or the FP32 accurate copy with FP64-grade sums
        double* X = ws.get_n<double>(n);
        double* Y = ws.get_n<double>(n);
        fill_kernel<double><<<g, 256, 0, s>>>(X, n, 1.0);
        RAD_CHECK_LAUNCH();
        if (h->op_is_f64()) apply_tree(h, X, 1, Y, 1, 1, st, ws.get(apply_workspace_bytes(h, 1)), s);
        else apply_tree_acc(h, X, 1, Y, 1, 1, st, static_cast<double*>(ws.get(apply_workspace_bytes_acc(h, 1))), s);
        row_scale_kernel<double><<<g, 256, 0, s>>>(Y, n, S64, scale);
    } else {
        float* X = ws.get_n<float>(n);
        float* Y = ws.get_n<float>(n);
        fill_kernel<float><<<g, 256, 0, s>>>(X, n, 1.0f);
        RAD_CHECK_LAUNCH();
        apply_tree(h, X, 1, Y, 1, 1, st, ws.get(apply_workspace_bytes(h, 1)), s);
        row_scale_kernel<float><<<g, 256, 0, s>>>(Y, n, S64, scale);
    }
    RAD_CHECK_LAUNCH();
    if (h->near_dtype == RAD_F64) scale_panels<double>(h, 0, scale, h->near_pool.p, s);
    else scale_panels<float>(h, 0, scale, h->near_pool.p, s);
    if (h->factor_dtype == RAD_F64) scale_panels<double>(h, 1, scale, h->far_pool.p, s);
    else if (h->factor_dtype == RAD_F32) scale_panels<float>(h, 1, scale, h->far_pool.p, s);
    else scale_panels<__nv_bfloat16>(h, 1, scale, h->far_pool.p, s);
    if (h->far_pool_acc.p) scale_panels<float>(h, 1, scale, h->far_pool_acc.p, s);
    h->closed = 1;
}

// ---------------------------------------------------------------- autotuner
// Times the streaming products on this handle's operator for every
// candidate (far-field item rows x grid policy of each launch) and keeps the
// fastest.  The grid policy does not change results (every item is computed
// by one CTA in the same order); the item rows change the order of the sums
// over a column group's columns.
namespace {

template <class NS, class FS, class AT>
struct Tuner {
    rad_htree* h;
    cudaStream_t s;
    AT *X, *T, *Yn;
    void* Y;
    AT* X64;   // n x 64 block for the many-column product
    cudaEvent_t e0, e1;
    template <class F>
    float time(F&& launch) {
        launch();
        RAD_CHECK_LAUNCH();
        float best = 1e30f;
        for (int r = 0; r < 3; ++r) {
            RAD_CUDA(cudaEventRecord(e0, s));
            launch();
            RAD_CHECK_LAUNCH();
            RAD_CUDA(cudaEventRecord(e1, s));
            RAD_CUDA(cudaEventSynchronize(e1));
            float ms = 0.0f;
            RAD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            best = std::min(best, ms);
        }
        return best;
    }
    // best grid (0 = one CTA per item) and its time for one launch kind
    std::pair<int, float> pick(int kind, const std::vector<int>& grids) {
        const OpView op = h->view();
        const Epi epi{kStore, nullptr, nullptr, nullptr, 0};
        std::pair<int, float> best{0, 1e30f};
        for (int g : grids) {
            float t = 0.0f;
            if (kind == 0) t = time([&] { single_phase_a<NS, FS, AT><<<grid_of(g, op.n_aitems), 256, 0, s>>>(op, X, T, Yn); });
            if (kind == 1) t = time([&] { single_phase_b<FS, AT><<<grid_of(g, op.n_tiles), 256, 0, s>>>(op, T, Yn, Y, epi); });
            if (kind == 2 && op.n_sitems > 0)
                t = time([&] { far_vt_stream<FS, AT, 2><<<grid_of(g, op.n_sitems), 256, 0, s>>>(op, X, 2, T, 4); });
            if (kind == 3)
                t = time([&] { rows_stream<NS, FS, AT, 2><<<grid_of(g, op.n_tiles), 256, 0, s>>>(op, X, 2, T, 4, Y, 2, epi); });
            if (t < best.second) best = {g, t};
        }
        return best;
    }
    void run() {
        int sms = 0, dev = 0;
        RAD_CUDA(cudaGetDevice(&dev));
        RAD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const std::vector<int> grids{0, 2 * sms, 4 * sms, 8 * sms};
        const int rows_cand[3] = {64, 128, 256};
        float best_total = 1e30f;
        int best_rows = h->stream_rows, ga1 = 0, gb1 = 0, ga2 = 0, gb2 = 0;
        for (int rows : rows_cand) {
            build_stream_lists(h, rows, s);
            const auto a1 = pick(0, grids), b1 = pick(1, grids), a2 = pick(2, grids), b2 = pick(3, grids);
            const float total = a1.second + b1.second + a2.second + b2.second;
            if (total < best_total) {
                best_total = total;
                best_rows = rows;
                ga1 = a1.first;
                gb1 = b1.first;
                ga2 = a2.first;
                gb2 = b2.first;
            }
        }
        build_stream_lists(h, best_rows, s);
        h->grid_a1 = ga1;
        h->grid_b1 = gb1;
        h->grid_a2 = ga2;
        h->grid_b2 = gb2;
        // one column: the fused launch or the two tuned launches
        if constexpr (std::is_same<AT, float>::value && std::is_same<NS, float>::value) {
            if (h->hmv1_ok) {
                const Epi epi{kStore, nullptr, nullptr, nullptr, 0};
                float t1[2];
                for (int path = 0; path < 2; ++path) {
                    h->one_col_path = path;
                    t1[path] = time([&] { apply_t<NS, FS, AT>(h, h->view(), X, 1, Y, 1, 1, epi, T, s); });
                }
                h->one_col_path = t1[1] <= t1[0] ? 1 : 0;
            }
        }
        // many-column product: CUDA-core tiles or tensor cores, 64 columns
        if constexpr (std::is_same<AT, float>::value && std::is_same<NS, float>::value) {
            float best = 1e30f;
            int pick = 0;
            tc_build_images(h, s);
            for (int path = 0; path < 2; ++path) {
                h->mm_path = path;
                const float t = time([&] {
                    apply_t<NS, FS, AT>(h, h->view(), X64, 64, Y, 64, 64, Epi{kStore, nullptr, nullptr, nullptr, 0},
                                        T, s);
                });
                if (t < best) {
                    best = t;
                    pick = path;
                }
            }
            h->mm_path = pick;
            if (pick == 0) tc_drop_images(h, s);
        }
        h->tuned = 1;
    }
};

}  // namespace

void autotune(rad_htree* h, cudaStream_t s) {
    RAD_REQUIRE(h->compressed, RAD_EINVAL, "handle is not compressed (call rad_compress_aca)");
    drop_product_graph(h);
    Scratch ws(s);
    const int n = (int)h->n;
    const size_t esz = h->op_is_f64() ? 8 : 4;
    cudaEvent_t e0, e1;
    RAD_CUDA(cudaEventCreate(&e0));
    RAD_CUDA(cudaEventCreate(&e1));
    void* X = ws.get(esz * 2 * (size_t)n);
    void* Y = ws.get(8 * 64 * (size_t)n);
    const size_t tb = std::max({apply_workspace_bytes(h, 4) + esz * (size_t)n, apply_workspace_bytes(h, 64),
                                apply_workspace_bytes(h, 1)}) +
                      (h->op_is_f64() ? 0 : tc_workspace_bytes(h, 64));
    void* T = ws.get(tb);
    void* X64 = ws.get(esz * 64 * (size_t)n);
    RAD_CUDA(cudaMemsetAsync(X, 0, esz * 2 * (size_t)n, s));
    RAD_CUDA(cudaMemsetAsync(T, 0, tb, s));
    RAD_CUDA(cudaMemsetAsync(X64, 0, esz * 64 * (size_t)n, s));
    try {
        if (h->op_is_f64()) {
            Tuner<double, double, double> t{h, s, (double*)X, (double*)T, (double*)T + std::max(1, h->sum_rank) * 4, Y,
                                            (double*)X64, e0, e1};
            t.run();
        } else if (h->factor_dtype == RAD_F32) {
            Tuner<float, float, float> t{h, s, (float*)X, (float*)T, (float*)T + std::max(1, h->sum_rank) * 4, Y,
                                         (float*)X64, e0, e1};
            t.run();
        } else {
            Tuner<float, __nv_bfloat16, float> t{h, s, (float*)X, (float*)T, (float*)T + std::max(1, h->sum_rank) * 4,
                                                 Y, (float*)X64, e0, e1};
            t.run();
        }
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    RAD_CUDA(cudaStreamSynchronize(s));
}

}  // namespace rad
