// A4-A5: dense blocks (entries of Eq. 10) and cross approximation of the
// admissible blocks (§4.3, Eqs. 30-31), plus packing of the factors and the
// row-tile tables used by the matrix-vector product.
//
// Partial-pivot ACA runs one 256-thread CTA per admissible block with
// m + n > kWarpMaxMN and, in the same launch, persistent warps that take the
// other blocks one at a time (largest first) from a device counter.  Rows
// and columns of the block are evaluated on the fly from the tree-ordered
// facet geometry; the residual row/column are written straight into the
// block's slot of the U/V scratch (column-major, room for kmax columns);
// pivots come from warp-shuffle (or block-wide) argmax reductions
// (ties: lowest index); the Frobenius-norm estimate of the cross and the dot
// products accumulate in FP64 (or a two-sum FP32 pair where the tolerance
// allows FP32 arithmetic).
//
// Partial pivoting: first pivot row 0; column pivot = argmax |residual row|;
// a residual row whose largest modulus is <= max(1e-300, 1e-14 x largest
// pivot so far) is marked used and the lowest unused row is tried instead;
// next row = argmax |u_k| over unused rows; candidate stop when
// |u_k| |v_k| <= tol ||S_k||_F with
// ||S_k||^2 = ||S_{k-1}||^2 + 2 sum_{l<k} (u_k.u_l)(v_k.v_l) + |u_k|^2 |v_k|^2.
// Partial pivoting is the less reliable rule (§1), and that candidate stop
// can fire early, so this kernel (beyond the paper's plain rule) verifies it (at most kMaxChecks times per block) on
// m + n residual entries, one in every row and one in every column: sample
// s < m is (s, (s * 2654435761 + c * 40503 + 1) mod n), sample m + j is
// ((j * 2246822519 + c * 40503 + 3) mod m, j), c = checks so far; if
// (m n / (m + n)) sum r_s^2 > tol^2 ||S_k||^2 the iteration resumes from the
// row of the largest |r_s| (ties: lowest s).
// Full pivoting keeps the whole residual and stops when
// ||R_k||_F <= tol ||X||_F (Eq. 31 exactly).
// A block whose rank would exceed kmax = min(max_rank, m n / (m + n)) is
// stored dense.

#include <algorithm>
#include <climits>
#include <exception>
#include <memory>
#include <thread>
#include <cstring>
#include <numeric>

#include <mutex>

#include "rad_device.cuh"

namespace rad {

namespace {

struct AcaJob {
    int r0, c0, m, n, kmax, pad;
    long long offU, offV, offUsed;
};

constexpr int kAcaNT = 256;
// Blocks with m + n above this run on a whole CTA: one warp would take
// their ~m + n entries per step alone, and the largest of them would set
// the length of the launch.
constexpr int kWarpMaxMN = 768;

// position of verification sample s (< m + n) of check c
__device__ __forceinline__ void sample_pos(int s, int m, int n, int c, int& si, int& sj) {
    if (s < m) {
        si = s;
        sj = (int)(((unsigned long long)s * 2654435761ull + (unsigned long long)c * 40503ull + 1ull) %
                   (unsigned long long)n);
    } else {
        sj = s - m;
        si = (int)(((unsigned long long)sj * 2246822519ull + (unsigned long long)c * 40503ull + 3ull) %
                   (unsigned long long)m);
    }
}
constexpr int kMaxChecks = 4;

// Running sum of the stopping rule's ||S_k||^2.  With FP32 arithmetic it is
// kept as an unevaluated hi + lo pair updated by the error-free two-sum, so
// the accumulation keeps about twice FP32's precision without touching the
// narrow FP64 pipe; with FP64 arithmetic it is a plain double.
template <class CT> struct RunSum;
template <> struct RunSum<double> {
    double v = 0.0;
    __device__ __forceinline__ void add(double x) { v += x; }
    __device__ __forceinline__ double value() const { return v; }
};
template <> struct RunSum<float> {
    float h = 0.0f, l = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float s = __fadd_rn(h, x);
        const float bp = __fsub_rn(s, h);
        const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(x, bp));
        const float t = __fadd_rn(l, e);
        h = __fadd_rn(s, t);
        l = __fsub_rn(t, __fsub_rn(h, s));
    }
    __device__ __forceinline__ float value() const { return h; }
};
// Zero-row threshold floor (1e-300 in FP64; in FP32 only an exact zero
// is below it).
template <class CT> struct Tiny;
template <> struct Tiny<double> { static constexpr double v = 1e-300; };
template <> struct Tiny<float> { static constexpr float v = 0.0f; };


// lowest index i < m with used[i] == 0, or -1; all threads receive it
__device__ int lowest_unused(const unsigned char* used, int m, int* sm) {
    int best = 0x7fffffff;
    for (int i = threadIdx.x; i < m; i += kAcaNT)
        if (!used[i]) { best = i; break; }
    best = __reduce_min_sync(0xffffffffu, best);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sm[warp] = best;
    __syncthreads();
    if (warp == 0) {
        int t = lane < kAcaNT / 32 ? sm[lane] : 0x7fffffff;
        t = __reduce_min_sync(0xffffffffu, t);
        if (lane == 0) sm[kAcaNT / 32] = t;
    }
    __syncthreads();
    const int r = sm[kAcaNT / 32];
    __syncthreads();
    return r == 0x7fffffff ? -1 : r;
}

// For l < k: out[l] = sum_j a_j * B[l*ld + j] over this thread's j; plus
// out[k] = sum_j a_j^2.  Results land in red[0..k] for every thread.  Four
// products per pass over the thread's j (their loads in flight together),
// each summed over the warp by the same butterfly as warp_sum.
template <class CT>
__device__ void cross_dots(const CT* a, const CT* B, int len, long long ld, int k, CT (*part)[kMaxRank + 1],
                           CT* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int l0 = 0; l0 <= k; l0 += 4) {
        const int nq = min(4, k + 1 - l0);
        const CT* rows[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) rows[q] = (l0 + q < k) ? B + (long long)(l0 + q) * ld : a;
        CT t[4] = {CT(0), CT(0), CT(0), CT(0)};
        for (int j = threadIdx.x; j < len; j += kAcaNT) {
            const CT aj = a[j];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < nq) t[q] += aj * rows[q][j];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 4; ++q) t[q] += __shfl_xor_sync(0xffffffffu, t[q], o);
        if (lane == 0)
            for (int q = 0; q < nq; ++q) part[warp][l0 + q] = t[q];
    }
    __syncthreads();
    if ((int)threadIdx.x <= k) {
        CT s = 0;
        for (int w = 0; w < kAcaNT / 32; ++w) s += part[w][threadIdx.x];
        red[threadIdx.x] = s;
    }
    __syncthreads();
}

// Shared memory of one ACA CTA: the CTA-wide path and the per-warp path.
// All arithmetic runs in CT; the running ||S_k||^2 is a RunSum<CT>.
template <class CT>
struct AcaSmem {
    CT s_row[kMaxRank];
    CT part[kAcaNT / 32][kMaxRank + 1];
    CT s_cv[kMaxRank + 1];
    CT s_cu[kMaxRank + 1];
    ArgMaxT<CT> am_sm[kAcaNT / 32 + 1];
    int i_sm[kAcaNT / 32 + 1];
    CT red_sm[kAcaNT / 32 + 1];
    CT w_a[kAcaNT / 32][kMaxRank];       // per warp: pivot row/column of U, V
    CT w_c[kAcaNT / 32][kMaxRank];       // per warp: (v_k . v_l)
};

// One admissible block on a whole CTA (blocks with more than 1024 rows or
// 4096 columns).
template <class CT>
__device__ void aca_cta_block(const Geo& g, const AcaJob& jb, int bidx, CT* Upool, CT* Vpool,
                              unsigned char* used_pool, int* __restrict__ rank_out,
                              long long* __restrict__ evals_out, double tol, AcaSmem<CT>& sm) {
    CT* s_row = sm.s_row;
    CT (*part)[kMaxRank + 1] = sm.part;
    CT* s_cv = sm.s_cv;
    CT* s_cu = sm.s_cu;
    ArgMaxT<CT>* am_sm = sm.am_sm;
    int* i_sm = sm.i_sm;
    CT* red_sm = sm.red_sm;
    const int m = jb.m, n = jb.n, kmax = jb.kmax;
    CT* U = Upool + jb.offU;
    CT* V = Vpool + jb.offV;
    unsigned char* used = used_pool + jb.offUsed;

    int i = 0, k = 0, status = 0, checks = 0;  // status: 1 converged, 2 rank cap
    RunSum<CT> norm2;
    CT scale = 0;
    const CT tolsq = (CT)(tol * tol);
    long long evals = 0;
    for (int guard = 0; guard <= m + kmax + kMaxChecks + 2; ++guard) {
        if (k >= kmax) { status = 2; break; }
        // residual of pivot row i: X(i,:) - sum_l U(i,l) V(:,l)
        if ((int)threadIdx.x < k) s_row[threadIdx.x] = U[(long long)threadIdx.x * m + i];
        __syncthreads();
        CT* vk = V + (long long)k * n;
        ArgMaxT<CT> best{CT(-1), 0x7fffffff};
        for (int j = threadIdx.x; j < n; j += kAcaNT) {
            CT r = Entry<CT>::eval(g, jb.r0 + i, jb.c0 + j);
            for (int l = 0; l < k; ++l) r -= s_row[l] * V[(long long)l * n + j];
            vk[j] = r;
            best = am_better(best, ArgMaxT<CT>{fabs(r), j});
        }
        best = block_argmax<kAcaNT>(best, am_sm);
        evals += n;
        if (threadIdx.x == 0) used[i] = 1;
        __syncthreads();
        if (!(best.v > fmax(Tiny<CT>::v, CT(1e-14) * scale))) {
            const int nxt = lowest_unused(used, m, i_sm);
            if (nxt < 0) { status = 1; break; }
            i = nxt;
            continue;
        }
        scale = fmax(scale, best.v);
        const int jp = best.i;
        const CT piv = vk[jp];
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += kAcaNT) vk[j] = vk[j] / piv;
        // (v_k . v_l) for l < k and |v_k|^2; each thread reads its own j
        cross_dots<CT>(vk, V, n, n, k, part, s_cv);
        // residual of pivot column jp
        if ((int)threadIdx.x < k) s_row[threadIdx.x] = V[(long long)threadIdx.x * n + jp];
        __syncthreads();
        CT* uk = U + (long long)k * m;
        ArgMaxT<CT> bu{CT(-1), 0x7fffffff};
        for (int r = threadIdx.x; r < m; r += kAcaNT) {
            CT u = Entry<CT>::eval(g, jb.r0 + r, jb.c0 + jp);
            for (int l = 0; l < k; ++l) u -= s_row[l] * U[(long long)l * m + r];
            uk[r] = u;
            if (!used[r]) bu = am_better(bu, ArgMaxT<CT>{fabs(u), r});
        }
        evals += m;
        cross_dots<CT>(uk, U, m, m, k, part, s_cu);
        bu = block_argmax<kAcaNT>(bu, am_sm);
        CT cross = 0;
        for (int l = 0; l < k; ++l) cross += s_cu[l] * s_cv[l];
        const CT uu = s_cu[k], vv = s_cv[k];
        norm2.add(CT(2) * cross + uu * vv);
        ++k;
        // |u_k| |v_k| <= tol ||S_k||_F, compared squared
        if (uu * vv <= tolsq * fmax(norm2.value(), CT(0))) {
            if (checks >= kMaxChecks) { status = 1; break; }
            // verify the candidate stop on one residual entry per row and
            // one per column
            CT r2p = 0;
            ArgMaxT<CT> bsp{CT(-1), 0x7fffffff};
            for (int sidx = threadIdx.x; sidx < m + n; sidx += kAcaNT) {
                int si, sj;
                sample_pos(sidx, m, n, checks, si, sj);
                CT x = Entry<CT>::eval(g, jb.r0 + si, jb.c0 + sj);
                for (int l = 0; l < k; ++l) x -= U[(long long)l * m + si] * V[(long long)l * n + sj];
                r2p += x * x;
                bsp = am_better(bsp, ArgMaxT<CT>{fabs(x), sidx});
            }
            const CT r2 = block_sum<kAcaNT, CT>(r2p, red_sm);
            const ArgMaxT<CT> bs = block_argmax<kAcaNT>(bsp, am_sm);
            int wi, wj;
            sample_pos(bs.i, m, n, checks, wi, wj);
            ++checks;
            evals += m + n;
            if ((CT)m * (CT)n / CT(m + n) * r2 <= tolsq * fmax(norm2.value(), CT(0))) { status = 1; break; }
            if (used[wi]) {
                wi = lowest_unused(used, m, i_sm);
                if (wi < 0) { status = 1; break; }
            }
            i = wi;
            continue;
        }
        if (bu.v < CT(0)) { status = 1; break; }
        i = bu.i;
    }
    if (threadIdx.x == 0) {
        rank_out[bidx] = status == 1 ? k : -1;
        evals_out[bidx] = evals;
    }
}


// p[q] = sum_j a_j * B[(l0 + q) ld + j] over the warp (q < 4, l0 + q < k),
// with the four shuffle reductions interleaved.
template <class CT>
__device__ __forceinline__ void warp_dots4(const CT* a, const CT* B, int len, long long ld, int l0, int k,
                                           CT p[4]) {
    const int lane = threadIdx.x & 31;
    const int nq = min(4, k - l0);
    CT t[4] = {CT(0), CT(0), CT(0), CT(0)};
    for (int j = lane; j < len; j += 32) {
        const CT aj = a[j];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (q < nq) t[q] += aj * B[(long long)(l0 + q) * ld + j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < 4; ++q) t[q] += __shfl_xor_sync(0xffffffffu, t[q], o);
#pragma unroll
    for (int q = 0; q < 4; ++q) p[q] = t[q];
}

// One admissible block (m <= 1024 rows) on a single warp: no block
// barriers, shuffle reductions, and the used-row flags of rows lane + 32 t in
// bit t of a register.  Same pivoting, stopping and verification rules as
// the CTA path.
template <class CT>
__device__ void aca_warp_block(const Geo& g, const AcaJob& jb, int bidx, CT* Upool, CT* Vpool,
                               int* __restrict__ rank_out, long long* __restrict__ evals_out, double tol,
                               CT* s_a, CT* s_c) {
    const int lane = threadIdx.x & 31;
    const int m = jb.m, n = jb.n, kmax = jb.kmax;
    CT* U = Upool + jb.offU;
    CT* V = Vpool + jb.offV;
    unsigned used = 0u;
    int i = 0, k = 0, status = 0, checks = 0;
    RunSum<CT> norm2;
    CT scale = 0;
    const CT tolsq = (CT)(tol * tol);
    long long evals = 0;
    for (int guard = 0; guard <= m + kmax + kMaxChecks + 2; ++guard) {
        if (k >= kmax) { status = 2; break; }
        for (int l = lane; l < k; l += 32) s_a[l] = U[(long long)l * m + i];
        __syncwarp();
        CT* vk = V + (long long)k * n;
        ArgMaxT<CT> best{CT(-1), 0x7fffffff};
        for (int j = lane; j < n; j += 32) {
            CT r = Entry<CT>::eval(g, jb.r0 + i, jb.c0 + j);
            for (int l = 0; l < k; ++l) r -= s_a[l] * V[(long long)l * n + j];
            vk[j] = r;
            best = am_better(best, ArgMaxT<CT>{fabs(r), j});
        }
        best = warp_argmax(best);
        evals += n;
        if ((i & 31) == lane) used |= 1u << (i >> 5);
        if (!(best.v > fmax(Tiny<CT>::v, CT(1e-14) * scale))) {
            int cand = 0x7fffffff;
            for (int t = 0; t < 32 && lane + 32 * t < m; ++t)
                if (!((used >> t) & 1u)) { cand = lane + 32 * t; break; }
            cand = __reduce_min_sync(0xffffffffu, cand);
            if (cand == 0x7fffffff) { status = 1; break; }
            i = cand;
            __syncwarp();
            continue;
        }
        scale = fmax(scale, best.v);
        const int jp = best.i;
        __syncwarp();
        const CT piv = vk[jp];
        __syncwarp();
        CT vvp = 0;
        for (int j = lane; j < n; j += 32) {
            const CT v = vk[j] / piv;
            vk[j] = v;
            vvp += v * v;
        }
        const CT vv = warp_sum(vvp);
        for (int l0 = 0; l0 < k; l0 += 4) {
            CT p[4];
            warp_dots4<CT>(vk, V, n, n, l0, k, p);
            if (lane == 0)
                for (int q = 0; q < 4 && l0 + q < k; ++q) s_c[l0 + q] = p[q];
        }
        __syncwarp();
        for (int l = lane; l < k; l += 32) s_a[l] = V[(long long)l * n + jp];
        __syncwarp();
        CT* uk = U + (long long)k * m;
        ArgMaxT<CT> bu{CT(-1), 0x7fffffff};
        CT uup = 0;
        for (int r = lane; r < m; r += 32) {
            CT u = Entry<CT>::eval(g, jb.r0 + r, jb.c0 + jp);
            for (int l = 0; l < k; ++l) u -= s_a[l] * U[(long long)l * m + r];
            uk[r] = u;
            uup += u * u;
            if (!((used >> (r >> 5)) & 1u)) bu = am_better(bu, ArgMaxT<CT>{fabs(u), r});
        }
        const CT uu = warp_sum(uup);
        CT cross = 0;
        for (int l0 = 0; l0 < k; l0 += 4) {
            CT p[4];
            warp_dots4<CT>(uk, U, m, m, l0, k, p);
            for (int q = 0; q < 4 && l0 + q < k; ++q) cross += p[q] * s_c[l0 + q];
        }
        bu = warp_argmax(bu);
        evals += m;
        norm2.add(CT(2) * cross + uu * vv);
        ++k;
        // |u_k| |v_k| <= tol ||S_k||_F, compared squared
        if (uu * vv <= tolsq * fmax(norm2.value(), CT(0))) {
            if (checks >= kMaxChecks) { status = 1; break; }
            CT r2p = 0;
            ArgMaxT<CT> bs{CT(-1), 0x7fffffff};
            for (int sidx = lane; sidx < m + n; sidx += 32) {
                int si, sj;
                sample_pos(sidx, m, n, checks, si, sj);
                CT x = Entry<CT>::eval(g, jb.r0 + si, jb.c0 + sj);
                for (int l = 0; l < k; ++l) x -= U[(long long)l * m + si] * V[(long long)l * n + sj];
                r2p += x * x;
                bs = am_better(bs, ArgMaxT<CT>{fabs(x), sidx});
            }
            const CT r2 = warp_sum(r2p);
            bs = warp_argmax(bs);
            int wi, wj;
            sample_pos(bs.i, m, n, checks, wi, wj);
            ++checks;
            evals += m + n;
            if ((CT)m * (CT)n / CT(m + n) * r2 <= tolsq * fmax(norm2.value(), CT(0))) { status = 1; break; }
            const unsigned wused = __shfl_sync(0xffffffffu, (used >> (wi >> 5)) & 1u, wi & 31);
            if (wused) {
                int cand = 0x7fffffff;
                for (int t = 0; t < 32 && lane + 32 * t < m; ++t)
                    if (!((used >> t) & 1u)) { cand = lane + 32 * t; break; }
                cand = __reduce_min_sync(0xffffffffu, cand);
                if (cand == 0x7fffffff) { status = 1; break; }
                wi = cand;
            }
            i = wi;
            __syncwarp();
            continue;
        }
        if (bu.v < CT(0)) { status = 1; break; }
        i = bu.i;
        __syncwarp();
    }
    if (lane == 0) {
        rank_out[bidx] = status == 1 ? k : -1;
        evals_out[bidx] = evals;
    }
}

// Blocks [0, n_big) of the grid take one large block each (CTA path); the
// other CTAs are persistent: each warp takes the next block of the `small`
// list (largest first) from a device counter until the list is exhausted.
template <class CT>
__global__ void __launch_bounds__(kAcaNT, 4)
aca_partial_persistent(Geo g, const AcaJob* __restrict__ jobs, const int* __restrict__ big, int n_big,
                       const int* __restrict__ small, int n_small, int* __restrict__ next_small, CT* Upool,
                       CT* Vpool, unsigned char* used_pool, int* __restrict__ rank_out,
                       long long* __restrict__ evals_out, double tol) {
    __shared__ AcaSmem<CT> sm;
    if ((int)blockIdx.x < n_big) {
        const int bidx = big[blockIdx.x];
        const AcaJob jb = jobs[bidx];
        aca_cta_block<CT>(g, jb, bidx, Upool, Vpool, used_pool, rank_out, evals_out, tol, sm);
        return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        int w = 0;
        if (lane == 0) w = atomicAdd(next_small, 1);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= n_small) break;
        const int bidx = small[w];
        const AcaJob jb = jobs[bidx];
        aca_warp_block<CT>(g, jb, bidx, Upool, Vpool, rank_out, evals_out, tol, sm.w_a[warp], sm.w_c[warp]);
        __syncwarp();
    }
}

// Full pivoting: the residual R (m x n, column-major) lives in scratch.
template <class CT>
__global__ void __launch_bounds__(kAcaNT)
aca_full_kernel(Geo g, const AcaJob* __restrict__ jobs, const int* __restrict__ order, CT* Upool, CT* Vpool,
                CT* Rpool, const long long* __restrict__ offR, int* __restrict__ rank_out,
                long long* __restrict__ evals_out, double tol) {
    __shared__ double red[kAcaNT / 32 + 1];
    __shared__ ArgMax am_sm[kAcaNT / 32 + 1];
    const int bidx = order[blockIdx.x];
    const AcaJob jb = jobs[bidx];
    const int m = jb.m, n = jb.n, kmax = jb.kmax;
    const long long mn = (long long)m * n;
    CT* R = Rpool + offR[bidx];
    CT* U = Upool + jb.offU;
    CT* V = Vpool + jb.offV;
    double s = 0.0;
    for (long long e = threadIdx.x; e < mn; e += kAcaNT) {
        const int jj = (int)(e / m), ii = (int)(e - (long long)jj * m);
        const CT x = Entry<CT>::eval(g, jb.r0 + ii, jb.c0 + jj);
        R[e] = x;
        s += (double)x * (double)x;
    }
    const double normX2 = block_sum<kAcaNT, double>(s, red);
    double normR2 = normX2;
    int k = 0, status = 0;
    for (;;) {
        if (sqrt(normR2) <= tol * sqrt(normX2)) { status = 1; break; }
        if (k >= kmax) { status = 2; break; }
        // pivot: largest |R|, ties to the lowest (row, column) row-major
        ArgMax best{-1.0, 0x7fffffff};
        for (long long e = threadIdx.x; e < mn; e += kAcaNT) {
            const int jj = (int)(e / m), ii = (int)(e - (long long)jj * m);
            best = am_better(best, ArgMax{fabs((double)R[e]), ii * n + jj});
        }
        best = block_argmax<kAcaNT>(best, am_sm);
        const int ip = best.i / n, jp = best.i - ip * n;
        const CT piv = R[(long long)jp * m + ip];
        CT* uk = U + (long long)k * m;
        CT* vk = V + (long long)k * n;
        for (int r = threadIdx.x; r < m; r += kAcaNT) uk[r] = R[(long long)jp * m + r];
        for (int c = threadIdx.x; c < n; c += kAcaNT) vk[c] = R[(long long)c * m + ip] / piv;
        __syncthreads();
        s = 0.0;
        for (long long e = threadIdx.x; e < mn; e += kAcaNT) {
            const int jj = (int)(e / m), ii = (int)(e - (long long)jj * m);
            const CT x = R[e] - uk[ii] * vk[jj];
            R[e] = x;
            s += (double)x * (double)x;
        }
        normR2 = block_sum<kAcaNT, double>(s, red);
        ++k;
    }
    if (threadIdx.x == 0) {
        rank_out[bidx] = status == 1 ? k : -1;
        evals_out[bidx] = mn;
    }
}

// ------------------------------------------------------------ panel fill
// Dense pieces: columns [bc0, bc0 + ncols) of a dense block, restricted to
// the rows of tile `tile`, go to panel columns [col, col + ncols); rows of
// the panel beyond the tile's rows are zero.
struct DenseWork {
    int tile, bc0, ncols, col;
};
template <class S, class CT>
__global__ void __launch_bounds__(256)
dense_fill_kernel(Geo g, const Tile* __restrict__ tiles, const DenseWork* __restrict__ work, S* pool) {
    const DenseWork w = work[blockIdx.x];
    const Tile t = tiles[w.tile];
    S* P = pool + t.noff + (long long)w.col * t.ld;
    const int cnt = w.ncols * t.ld;
    for (int e = threadIdx.x; e < cnt; e += 256) {
        const int c = e / t.ld, i = e - c * t.ld;
        P[e] = i < t.rows ? Store<S>::put(Entry<CT>::eval(g, t.r0 + i, w.bc0 + c)) : Store<S>::put(CT(0));
    }
}

// Low-rank pieces: rows [ro, ro + tile rows) of U_b (ACA scratch, m x k
// column-major) go to low-rank panel columns [col, col + k).
struct UWork {
    int tile, ro, m, k, col, chunk;
    long long src;
};
// One warp per piece (eight per CTA): column l of the piece is rows
// ro .. ro + ld of U_b's column l (zeros past the tile's rows).
template <class CT, class S>
__global__ void __launch_bounds__(256)
u_fill_kernel(const Tile* __restrict__ tiles, const UWork* __restrict__ work, int nwork,
              const CT* const* __restrict__ Ubase, S* pool) {
    const int wi = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (wi >= nwork) return;
    const UWork w = work[wi];
    const CT* __restrict__ Us = Ubase[w.chunk];
    const Tile t = tiles[w.tile];
    S* P = pool + t.foff + (long long)w.col * t.ld;
    for (int l = 0; l < w.k; ++l) {
        const CT* src = Us + w.src + (long long)l * w.m + w.ro;
        S* dst = P + (long long)l * t.ld;
        for (int i = lane; i < t.ld; i += 32) dst[i] = i < t.rows ? Store<S>::put(src[i]) : Store<S>::put(CT(0));
    }
}

// V^T rows of block b (ACA scratch V_b, n x k column-major) go to rows
// [grow, grow + k) of its group's V panel.
struct VWork {
    int group, grow, n, k, chunk, pad;
    long long src;
};
template <class CT, class S>
__global__ void __launch_bounds__(256)
v_fill_kernel(const Group* __restrict__ groups, const VWork* __restrict__ work, const CT* const* __restrict__ Vbase,
              S* pool) {
    const VWork w = work[blockIdx.x];
    const CT* __restrict__ Vs = Vbase[w.chunk];
    const Group gr = groups[w.group];
    S* P = pool + gr.voff;
    const int cnt = w.n * w.k;
    for (int e = threadIdx.x; e < cnt; e += 256) {
        const int j = e / w.k, l = e - j * w.k;
        P[(long long)j * gr.ld + w.grow + l] = Store<S>::put(Vs[w.src + (long long)l * w.n + j]);
    }
}

// A caller's dense F (row-major n x n, FP64) as the dense panels of 64-row
// tiles.
__global__ void __launch_bounds__(256)
dense_from_matrix_kernel(int n, const Tile* __restrict__ tiles, const double* __restrict__ F, double* pool) {
    const Tile t = tiles[blockIdx.y];
    const long long cnt = (long long)n * t.ld;
    double* P = pool + t.noff;
    for (long long e = (long long)blockIdx.x * 256 + threadIdx.x; e < cnt; e += (long long)gridDim.x * 256) {
        const int c = (int)(e / t.ld), i = (int)(e - (long long)c * t.ld);
        P[e] = i < t.rows ? F[(long long)(t.r0 + i) * n + c] : 0.0;
    }
}

// Copies the first rank columns of every job's U and V scratch slots (column
// major, so m*k and n*k contiguous elements) to compact offsets.
template <class CT>
__global__ void __launch_bounds__(256)
compact_kernel(const AcaJob* __restrict__ jobs, const int* __restrict__ rank, const long long* __restrict__ cu,
               const long long* __restrict__ cv, const CT* __restrict__ Us, const CT* __restrict__ Vs, CT* Uc, CT* Vc) {
    const AcaJob j = jobs[blockIdx.x];
    const int k = rank[blockIdx.x];
    if (k <= 0) return;
    const long long nu = (long long)j.m * k, nv = (long long)j.n * k;
    for (long long e = threadIdx.x; e < nu; e += 256) Uc[cu[blockIdx.x] + e] = Us[j.offU + e];
    for (long long e = threadIdx.x; e < nv; e += 256) Vc[cv[blockIdx.x] + e] = Vs[j.offV + e];
}

// Indices 0..key.size()-1 ordered by descending key, ties in index order
// (two stable 16-bit counting passes; keys are clamped to 32 bits).
static std::vector<int> order_desc(const std::vector<long long>& key) {
    const size_t m = key.size();
    std::vector<int> a(m), b(m);
    std::vector<uint32_t> k(m);
    for (size_t i = 0; i < m; ++i) {
        a[i] = (int)i;
        k[i] = 0xffffffffu - (uint32_t)std::min<long long>(std::max<long long>(key[i], 0), 0xffffffffll);
    }
    // Large inputs: each pass counts per chunk of the current order on host
    // threads, takes offsets digit by digit and chunk by chunk (so equal
    // digits keep their order), and scatters per chunk: the same stable
    // passes as the sequential loop.
    const int P = m >= 200000 ? 16 : 1;
    if (P > 1) {
        std::vector<uint32_t> cnt((size_t)P * 65536);
        for (int pass = 0; pass < 2; ++pass) {
            const int sh = 16 * pass;
            std::fill(cnt.begin(), cnt.end(), 0u);
            parallel_parts(P, [&](int t) {
                uint32_t* c = &cnt[(size_t)t * 65536];
                for (size_t i = m * t / P, e = m * (t + 1) / P; i < e; ++i) ++c[(k[a[i]] >> sh) & 0xffff];
            });
            uint32_t run = 0;
            for (int d = 0; d < 65536; ++d)
                for (int t = 0; t < P; ++t) {
                    const uint32_t v = cnt[(size_t)t * 65536 + d];
                    cnt[(size_t)t * 65536 + d] = run;
                    run += v;
                }
            parallel_parts(P, [&](int t) {
                uint32_t* c = &cnt[(size_t)t * 65536];
                for (size_t i = m * t / P, e = m * (t + 1) / P; i < e; ++i) b[c[(k[a[i]] >> sh) & 0xffff]++] = a[i];
            });
            a.swap(b);
        }
        return a;
    }
    std::vector<int> cnt(65537);
    for (int pass = 0; pass < 2; ++pass) {
        const int sh = 16 * pass;
        std::fill(cnt.begin(), cnt.end(), 0);
        for (size_t i = 0; i < m; ++i) ++cnt[((k[a[i]] >> sh) & 0xffff) + 1];
        for (int d = 0; d < 65536; ++d) cnt[d + 1] += cnt[d];
        for (size_t i = 0; i < m; ++i) b[cnt[(k[a[i]] >> sh) & 0xffff]++] = a[i];
        a.swap(b);
    }
    return a;
}

// ------------------------------------------------------------ recompression
// §4.3 postprocessing of an ACA cross into standard form, with the rank
// truncated at a relative accuracy by the singular-value rule of §5.1:
// U = Q_U R_U and V = Q_V R_V (classical Gram-Schmidt applied twice),
// M = R_U R_V^T, one-sided Jacobi rotations on the columns of M accumulated
// in an orthogonal Z (M Z = W diag(s) at convergence), and the smallest r
// with sum_{i >= r} s_i^2 <= tol^2 sum_i s_i^2 is kept (s_i = norms of the
// columns of M Z in decreasing order, r >= 1):
// U <- Q_U (M Z)_r, V <- Q_V Z_r, in place in the ACA scratch.  Because Z is
// orthogonal, the dropped part has Frobenius norm exactly the norm of the
// dropped columns of M Z, converged or not.
constexpr int kRcMax = 64;     // crosses of higher rank keep their ACA form
constexpr int kRcRows = 64;    // row chunk of the final in-place product
constexpr int kRcSweeps = 10;

// shared memory of one cross of rank <= KM (leading dimension KM + 1)
template <class CT, int KM, int NT>
struct RcSmem {
    static constexpr int LD = KM + 1;
    CT R[2][KM * LD];          // R_U, R_V ([row][col], upper triangular)
    CT M[KM * LD];             // R_U R_V^T, rotated in place to M Z
    CT Z[KM * LD];             // accumulated rotations
    CT Qc[kRcRows * LD];       // row chunk of Q in the final product
    CT coef[KM];
    CT red[NT / 32 + 1];
    CT s2[KM];
    int pos[KM];               // column of M Z holding the r-th largest norm
    int keep;
    int rotated;
};

template <class CT> struct RcTol;
template <> struct RcTol<float> {
    static constexpr float eps = 1.1920929e-7f;
    static constexpr float orth = 1e-5f;     // Jacobi: columns count as orthogonal
};
template <> struct RcTol<double> {
    static constexpr double eps = 2.220446049250313e-16;
    static constexpr double orth = 1e-10;
};

// In-place QR of the len x k column-major A: A <- Q, R (row-major) upper
// triangular.  Each column loses its components along the previous ones
// twice (coefficients accumulated in R); what is left is normalised, or
// zeroed with R_cc = 0 when it is below 16 eps of the column.
template <class CT, int KM, int NT>
__device__ void rc_qr(CT* A, int len, int k, CT* R, RcSmem<CT, KM, NT>& S) {
    constexpr int LD = KM + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int e = threadIdx.x; e < KM * LD; e += NT) R[e] = CT(0);
    __syncthreads();
    for (int c = 0; c < k; ++c) {
        CT* a = A + (long long)c * len;
        for (int pass = 0; pass < 2 && c > 0; ++pass) {
            for (int q = warp; q < c; q += NT / 32) {
                const CT* aq = A + (long long)q * len;
                CT s = CT(0);
                for (int i = lane; i < len; i += 32) s += aq[i] * a[i];
                s = warp_sum(s);
                if (lane == 0) S.coef[q] = s;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < len; i += NT) {
                CT v = a[i];
                for (int q = 0; q < c; ++q) v -= A[(long long)q * len + i] * S.coef[q];
                a[i] = v;
            }
            if (threadIdx.x < c) R[threadIdx.x * LD + c] += S.coef[threadIdx.x];
            __syncthreads();
        }
        CT s = CT(0);
        for (int i = threadIdx.x; i < len; i += NT) s += a[i] * a[i];
        s = block_sum<NT>(s, S.red);
        CT orig = s;
        for (int q = 0; q < c; ++q) orig += R[q * LD + c] * R[q * LD + c];
        const bool dir = s > CT(0) && s > CT(256) * RcTol<CT>::eps * RcTol<CT>::eps * orig;
        const CT nrm = sqrt(s);
        const CT inv = dir ? CT(1) / nrm : CT(0);
        for (int i = threadIdx.x; i < len; i += NT) a[i] *= inv;
        if (threadIdx.x == 0) R[c * LD + c] = dir ? nrm : CT(0);
        __syncthreads();
    }
}

// One-sided Jacobi on the k x k matrix S.M, rotations accumulated in S.Z.
// Each sweep visits every column pair once in k - 1 rounds of disjoint pairs
// (round-robin: player 0 fixed, players 1 .. K-1 on a circle; an odd k adds
// an idle player); one warp per pair.  A pair (column norms^2 a, b,
// coupling g) is left alone when g is below orth sqrt(a b), or when
// rotating it would move a or b by less than `floor` (a thousandth of the
// truncation threshold tol^2 ||M||_F^2, divided by k): |g| <= floor or
// g^2 <= floor |a - b|.
template <class CT, int KM, int NT>
__device__ void rc_jacobi(int k, CT floor, RcSmem<CT, KM, NT>& S) {
    constexpr int LD = KM + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int K = k + (k & 1);
    for (int sweep = 0; sweep < kRcSweeps; ++sweep) {
        if (threadIdx.x == 0) S.rotated = 0;
        __syncthreads();
        for (int r = 0; r < K - 1; ++r) {
            for (int pr = warp; pr < K / 2; pr += NT / 32) {
                int p, q;
                if (pr == 0) {
                    p = 0;
                    q = r + 1;
                } else {
                    p = (r + pr) % (K - 1) + 1;
                    q = (r - pr + K - 1) % (K - 1) + 1;
                }
                if (p >= k || q >= k) continue;
                CT al = CT(0), be = CT(0), ga = CT(0);
                for (int i = lane; i < k; i += 32) {
                    const CT x = S.M[i * LD + p], y = S.M[i * LD + q];
                    al += x * x;
                    be += y * y;
                    ga += x * y;
                }
                // butterfly sums: every lane holds the same totals
                al = warp_sum(al);
                be = warp_sum(be);
                ga = warp_sum(ga);
                if (fabs(ga) <= floor || ga * ga <= floor * fabs(al - be) ||
                    fabs(ga) <= RcTol<CT>::orth * sqrt(al * be))
                    continue;
                const CT zeta = (be - al) / (CT(2) * ga);
                const CT t = (zeta >= CT(0) ? CT(1) : CT(-1)) / (fabs(zeta) + sqrt(CT(1) + zeta * zeta));
                const CT cs = CT(1) / sqrt(CT(1) + t * t), sn = cs * t;
                for (int i = lane; i < k; i += 32) {
                    const CT x = S.M[i * LD + p], y = S.M[i * LD + q];
                    S.M[i * LD + p] = cs * x - sn * y;
                    S.M[i * LD + q] = sn * x + cs * y;
                    const CT zx = S.Z[i * LD + p], zy = S.Z[i * LD + q];
                    S.Z[i * LD + p] = cs * zx - sn * zy;
                    S.Z[i * LD + q] = sn * zx + cs * zy;
                }
                if (lane == 0) S.rotated = 1;
            }
            __syncthreads();
        }
        const int any = S.rotated;
        __syncthreads();
        if (!any) break;
    }
}

// dst (len x keep, column-major) <- Q B_sel with Q = src (len x k,
// column-major) and B_sel = columns pos[0 .. keep) of the k x k matrix B,
// row chunk by row chunk (each chunk of Q is read into shared memory before
// any of its rows is written, so dst may be src).
template <class CT, int KM, int NT>
__device__ void rc_apply(const CT* src, CT* dst, int len, int k, int keep, const CT* B, RcSmem<CT, KM, NT>& S) {
    constexpr int LD = KM + 1;
    for (int i0 = 0; i0 < len; i0 += kRcRows) {
        const int rows = min(kRcRows, len - i0);
        for (int e = threadIdx.x; e < rows * k; e += NT) {
            const int c = e / rows, i = e - c * rows;
            S.Qc[i * LD + c] = src[(long long)c * len + i0 + i];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < rows * keep; e += NT) {
            const int r = e / rows, i = e - r * rows;
            const int col = S.pos[r];
            CT acc = CT(0);
            for (int c = 0; c < k; ++c) acc += S.Qc[i * LD + c] * B[c * LD + col];
            dst[(long long)r * len + i0 + i] = acc;
        }
        __syncthreads();
    }
}

// One CTA per listed ACA job (crosses of rank 2 .. KM); the rank is
// rewritten with the truncated one.  RES: the cross (m + n) x k is first
// copied into shared memory behind RcSmem and factorised there (one read
// and one write of global memory); otherwise it is factorised in place.
template <class CT, int KM, int NT, bool RES>
__global__ void __launch_bounds__(NT)
recompress_kernel(const AcaJob* __restrict__ jobs, const int* __restrict__ list, int* rank, CT* Us, CT* Vs,
                  double tol) {
    constexpr int LD = KM + 1;
    extern __shared__ __align__(16) unsigned char rc_smem[];
    RcSmem<CT, KM, NT>& S = *reinterpret_cast<RcSmem<CT, KM, NT>*>(rc_smem);
    const int b = list[blockIdx.x];
    const int k = rank[b];
    if (k < 2 || k > KM) return;
    const AcaJob j = jobs[b];
    CT* U = Us + j.offU;
    CT* V = Vs + j.offV;
    CT* qU = U;
    CT* qV = V;
    if constexpr (RES) {
        qU = reinterpret_cast<CT*>(rc_smem + sizeof(RcSmem<CT, KM, NT>));
        qV = qU + (long long)j.m * k;
        for (int e = threadIdx.x; e < j.m * k; e += NT) qU[e] = U[e];
        for (int e = threadIdx.x; e < j.n * k; e += NT) qV[e] = V[e];
        __syncthreads();
    }
    rc_qr(qU, j.m, k, S.R[0], S);
    rc_qr(qV, j.n, k, S.R[1], S);
    CT fro = CT(0);
    for (int e = threadIdx.x; e < k * k; e += NT) {
        const int a = e / k, c2 = e - a * k;
        CT s = CT(0);
        for (int c = 0; c < k; ++c) s += S.R[0][a * LD + c] * S.R[1][c2 * LD + c];
        S.M[a * LD + c2] = s;
        S.Z[a * LD + c2] = a == c2 ? CT(1) : CT(0);
        fro += s * s;
    }
    fro = block_sum<NT>(fro, S.red);
    rc_jacobi(k, CT(1e-3) * CT(tol) * CT(tol) * fro / CT(k), S);
    for (int c = threadIdx.x; c < k; c += NT) {
        CT s = CT(0);
        for (int i = 0; i < k; ++i) s += S.M[i * LD + c] * S.M[i * LD + c];
        S.s2[c] = s;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += NT) {
        int at = 0;
        for (int d = 0; d < k; ++d) at += (S.s2[d] > S.s2[c]) || (S.s2[d] == S.s2[c] && d < c);
        S.pos[at] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        CT total = CT(0);
        for (int r = 0; r < k; ++r) total += S.s2[S.pos[r]];
        int keep = 0;
        if (total > CT(0)) {
            const CT lim = CT(tol) * CT(tol) * total;
            CT tail = CT(0);
            keep = k;
            for (int r = k - 1; r >= 1; --r) {
                tail += S.s2[S.pos[r]];
                if (tail > lim) break;
                keep = r;
            }
        }
        S.keep = keep;
    }
    __syncthreads();
    const int keep = S.keep;
    rc_apply(qU, U, j.m, k, keep, S.M, S);
    rc_apply(qV, V, j.n, k, keep, S.Z, S);
    if (threadIdx.x == 0) rank[b] = keep;
}

// res_elems > 0: resident variant with room for that many cross elements
template <class CT, int KM, int NT, bool RES>
void launch_recompress(const std::vector<int>& list, long long res_elems, const AcaJob* d_jobs, int* d_rank,
                       CT* Us, CT* Vs, double tol, Scratch& ws, cudaStream_t s) {
    if (list.empty()) return;
    int* d_list = ws.get_n<int>(list.size());
    h2d(d_list, list, s);
    const size_t bytes = sizeof(RcSmem<CT, KM, NT>) + (RES ? (size_t)res_elems * sizeof(CT) : 0);
    // the attribute is set once, to the largest size a launch can ask for
    // (the 48 KiB tier), so that concurrent compressions on other host
    // threads never see it lowered between their setting and their launch
    static std::once_flag configured;
    std::call_once(configured, [] {
        RAD_CUDA(cudaFuncSetAttribute(recompress_kernel<CT, KM, NT, RES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(RcSmem<CT, KM, NT>) + (RES ? (size_t)(48 << 10) : 0))));
    });
    recompress_kernel<CT, KM, NT, RES><<<(unsigned)list.size(), NT, bytes, s>>>(d_jobs, d_list, d_rank, Us, Vs,
                                                                                 tol);
    RAD_CHECK_LAUNCH();
}

// Recompression of every cross of rank 2..64 (ranks on the host, updated
// on return): by rank class (16 / 32 / 64) and by whether the cross fits
// in shared memory (up to 16 KiB, up to 48 KiB, in place otherwise),
// largest work first within a launch.
template <class CT>
void recompress_all(const std::vector<AcaJob>& jobs, std::vector<int>& ranks, const AcaJob* d_jobs, int* d_rank,
                    CT* Us, CT* Vs, double tol, Scratch& ws, cudaStream_t s) {
    const int nj = (int)jobs.size();
    std::vector<long long> wk(nj);
    for (int b = 0; b < nj; ++b) wk[b] = (long long)(jobs[b].m + jobs[b].n) * ranks[b] * ranks[b];
    constexpr long long kTier[2] = {16 << 10, 48 << 10};
    std::vector<int> lists[3][3];        // [rank class][tier 0, tier 1, in place]
    long long need[3][2] = {};
    for (int b : order_desc(wk)) {
        const int k = ranks[b];
        if (k < 2 || k > kRcMax) continue;
        const int kc = k <= 16 ? 0 : k <= 32 ? 1 : 2;
        const long long el = (long long)(jobs[b].m + jobs[b].n) * k;
        const long long by = el * (long long)sizeof(CT);
        const int t = by <= kTier[0] ? 0 : by <= kTier[1] ? 1 : 2;
        lists[kc][t].push_back(b);
        if (t < 2) need[kc][t] = std::max(need[kc][t], el);
    }
    ProfScope ps_("aca_recompress", s);
    for (int t = 2; t >= 0; --t) {
        if (t == 2) {
            launch_recompress<CT, 16, 256, false>(lists[0][2], 0, d_jobs, d_rank, Us, Vs, tol, ws, s);
            launch_recompress<CT, 32, 256, false>(lists[1][2], 0, d_jobs, d_rank, Us, Vs, tol, ws, s);
            launch_recompress<CT, 64, 256, false>(lists[2][2], 0, d_jobs, d_rank, Us, Vs, tol, ws, s);
        } else {
            launch_recompress<CT, 16, 128, true>(lists[0][t], need[0][t], d_jobs, d_rank, Us, Vs, tol, ws, s);
            launch_recompress<CT, 32, 128, true>(lists[1][t], need[1][t], d_jobs, d_rank, Us, Vs, tol, ws, s);
            launch_recompress<CT, 64, 128, true>(lists[2][t], need[2][t], d_jobs, d_rank, Us, Vs, tol, ws, s);
        }
    }
    RAD_CUDA(cudaMemcpyAsync(ranks.data(), d_rank, sizeof(int) * nj, cudaMemcpyDeviceToHost, s));
    RAD_CUDA(cudaStreamSynchronize(s));
}

template <class CT>
void launch_aca(rad_htree* h, const rad_aca_params* p, const std::vector<AcaJob>& jobs, std::vector<int>& ranks,
                std::vector<long long>& evals, std::vector<std::vector<double>>* unused, Scratch& ws,
                CT*& Us, CT*& Vs, cudaStream_t s) {
    (void)unused;
    auto hs_prep = std::make_unique<HostScope>("host_aca_prep");
    const int nj = (int)jobs.size();
    long long su = 0, sv = 0, sused = 0;
    for (auto& j : jobs) {
        su = std::max(su, j.offU + (long long)j.m * j.kmax);
        sv = std::max(sv, j.offV + (long long)j.n * j.kmax);
        sused = std::max(sused, j.offUsed + j.m);
    }
    Us = ws.get_n<CT>(std::max<long long>(su, 1));
    Vs = ws.get_n<CT>(std::max<long long>(sv, 1));
    AcaJob* d_jobs = ws.get_n<AcaJob>(nj);
    h2d(d_jobs, jobs, s);
    // schedule the largest blocks first
    std::vector<long long> wkey(nj);
    for (int b = 0; b < nj; ++b) wkey[b] = (long long)(jobs[b].m + jobs[b].n) * std::max(1, jobs[b].kmax);
    const std::vector<int> order = order_desc(wkey);
    int* d_order = ws.get_n<int>(nj);
    h2d(d_order, order, s);
    int* d_rank = ws.get_n<int>(nj);
    long long* d_evals = ws.get_n<long long>(nj);
    const Geo g = geo_view(h->geo.as<double>(), h->geo32.as<float>(), h->n);
    hs_prep.reset();
    if (p->pivoting == RAD_ACA_FULL) {
        std::vector<long long> offR(nj);
        long long sr = 0;
        for (int b = 0; b < nj; ++b) {
            offR[b] = sr;
            sr += round_up((long long)jobs[b].m * jobs[b].n, 8);
        }
        RAD_REQUIRE(sr * (long long)sizeof(CT) <= (8ll << 30), RAD_ELIMIT,
                    "full-pivot ACA needs more than 8 GiB of residual storage; use partial pivoting");
        CT* R = ws.get_n<CT>(std::max<long long>(sr, 1));
        long long* d_offR = ws.get_n<long long>(nj);
        h2d(d_offR, offR, s);
        { ProfScope ps_("aca_full", s); aca_full_kernel<CT><<<nj, kAcaNT, 0, s>>>(g, d_jobs, d_order, Us, Vs, R, d_offR, d_rank, d_evals, p->tol); }
    } else {
        unsigned char* used = ws.get_n<unsigned char>(std::max<long long>(sused, 1));
        RAD_CUDA(cudaMemsetAsync(used, 0, std::max<long long>(sused, 1), s));
        std::vector<int> big, small;
        for (int b : order) {
            if (jobs[b].m + jobs[b].n <= kWarpMaxMN) small.push_back(b);
            else big.push_back(b);
        }
        int* d_big = ws.get_n<int>(std::max<size_t>(1, big.size()));
        int* d_small = ws.get_n<int>(std::max<size_t>(1, small.size()));
        h2d(d_big, big, s);
        h2d(d_small, small, s);
        const int nb = (int)big.size(), nsm = (int)small.size();
        int* d_next = ws.get_n<int>(1);
        RAD_CUDA(cudaMemsetAsync(d_next, 0, sizeof(int), s));
        static int persistent = 0;   // resident CTAs of the persistent kernel (one query per type)
        static std::once_flag once;
        std::call_once(once, [&] {
            int dev = 0, sms = 0, per = 0;
            RAD_CUDA(cudaGetDevice(&dev));
            RAD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            RAD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, aca_partial_persistent<CT>, kAcaNT, 0));
            persistent = std::max(1, per) * sms;
        });
        const int grid = nb + std::min(persistent, std::max(1, (nsm + kAcaNT / 32 - 1) / (kAcaNT / 32)));
        { ProfScope ps_("aca_partial", s); aca_partial_persistent<CT><<<grid, kAcaNT, 0, s>>>(g, d_jobs, d_big, nb, d_small, nsm, d_next, Us, Vs, used, d_rank, d_evals, p->tol); }
    }
    RAD_CHECK_LAUNCH();
    ranks.resize(nj);
    evals.resize(nj);
    RAD_CUDA(cudaMemcpyAsync(ranks.data(), d_rank, sizeof(int) * nj, cudaMemcpyDeviceToHost, s));
    RAD_CUDA(cudaMemcpyAsync(evals.data(), d_evals, sizeof(long long) * nj, cudaMemcpyDeviceToHost, s));
    RAD_CUDA(cudaStreamSynchronize(s));
    if (p->recompress_tol > 0.0) recompress_all<CT>(jobs, ranks, d_jobs, d_rank, Us, Vs, p->recompress_tol, ws, s);
}

// Row tiles: leaf clusters (or [0, n) for a dense-wrapped matrix) cut into
// pieces of at most 64 rows.
static void make_tiles(rad_htree* h, std::vector<Tile>& tiles, std::vector<int>& tile_at) {
    const int n = (int)h->n;
    std::vector<std::pair<int, int>> leaves;
    if (h->from_dense) {
        leaves.push_back({0, n});
    } else {
        for (auto& nd : h->nodes)
            if (nd.leaf) leaves.push_back({nd.begin, nd.end});
        std::sort(leaves.begin(), leaves.end());
    }
    tiles.clear();
    tile_at.assign(n + 1, -1);
    for (auto& lf : leaves)
        for (int r = lf.first; r < lf.second; r += kTileRows) {
            tile_at[r] = (int)tiles.size();
            Tile t{};
            t.r0 = r;
            t.rows = std::min(kTileRows, lf.second - r);
            t.ld = (int)round_up(t.rows, 4);
            tiles.push_back(t);
        }
}

// Tiles covering rows [r0, r1) of a block (block rows are cluster ranges,
// which are unions of consecutive tiles).
template <class F>
static void for_tiles(const std::vector<Tile>& tiles, const std::vector<int>& tile_at, int r0, int r1, F&& f) {
    int r = r0;
    while (r < r1) {
        const int t = tile_at[r];
        RAD_REQUIRE(t >= 0, RAD_ECUDA, "internal: block rows do not align with row tiles");
        f(t);
        r += tiles[t].rows;
    }
}

// A run of consecutive gather indices: out[dst + i] = start + i, i < count.
// Every tile's gather list (near: X rows of its dense blocks; far: T rows of
// its low-rank blocks) is a concatenation of such runs.
struct IdxRun {
    int tile, col, start, count;
};
__global__ void __launch_bounds__(256)
fill_runs_kernel(const IdxRun* __restrict__ runs, int nruns, const Tile* __restrict__ tiles, int far, int* out) {
    const int r = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (r >= nruns) return;
    const IdxRun u = runs[r];
    const Tile t = tiles[u.tile];
    int* o = out + (far ? t.ixf : t.ixn) + u.col;
    for (int i = threadIdx.x & 31; i < u.count; i += 32) o[i] = u.start + i;
}

}  // namespace

// Work lists of the streaming (1-4 column) products for far-field items of
// at most `rows` rows: sitems (heaviest first) and the phase-A order that
// mixes them with the tiles' dense panels.
void build_stream_lists(rad_htree* h, int rows, cudaStream_t s) {
    const auto& G = h->groups_h;
    std::vector<GWork> w;
    for (int g = 0; g < (int)G.size(); ++g)
        for (int r = 0; r < G[g].M; r += rows) w.push_back(GWork{g, r, std::min(rows, G[g].M - r), 0});
    std::vector<long long> key(w.size());
    for (size_t i = 0; i < w.size(); ++i) key[i] = (long long)w[i].rows * G[w[i].g].n;
    std::vector<GWork> sitems(w.size());
    {
        const std::vector<int> ord = order_desc(key);
        for (size_t i = 0; i < w.size(); ++i) sitems[i] = w[ord[i]];
    }
    std::vector<long long> akey;
    std::vector<int> acode;
    for (size_t i = 0; i < sitems.size(); ++i) {
        akey.push_back((long long)sitems[i].rows * G[sitems[i].g].n);
        acode.push_back((int)i);
    }
    for (size_t t = 0; t < h->tiles_h.size(); ++t) {
        akey.push_back((long long)h->tiles_h[t].ld * h->tiles_h[t].kn);
        acode.push_back(-(int)t - 1);
    }
    std::vector<int> aorder(acode.size());
    {
        const std::vector<int> o = order_desc(akey);
        for (size_t i = 0; i < o.size(); ++i) aorder[i] = acode[o[i]];
    }
    h->stream_rows = rows;
    h->n_sitems = (int)sitems.size();
    h->n_aitems = (int)aorder.size();
    h->d_sitems.alloc(sizeof(GWork) * std::max<size_t>(1, sitems.size()), s);
    h->d_aorder.alloc(sizeof(int) * std::max<size_t>(1, aorder.size()), s);
    h2d(h->d_sitems.as<GWork>(), sitems, s);
    h2d(h->d_aorder.as<int>(), aorder, s);
}

namespace {

// SMs of the current device (one query per process)
static int sm_count() {
    static const int n = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            (void)cudaGetLastError();
            return 1;
        }
        return std::max(1, v);
    }();
    return n;
}

// Heaviest-first order re-dealt in snake order over L slots (the SMs that
// the first wave of one-CTA-per-item launches spreads over): positions
// 0..L-1 take items 0..L-1, positions L..2L-1 take items 2L-1..L, and so on,
// so that every slot's items add up to about the same work.
static std::vector<int> snake_order(const std::vector<int>& heavy_first, int L) {
    const size_t n = heavy_first.size();
    std::vector<int> out(n);
    for (size_t i = 0; i < n; ++i) {
        const size_t round = i / L, pos = i % L;
        const size_t src = round * L + ((round & 1) ? std::min<size_t>(L, n - round * L) - 1 - pos : pos);
        out[i] = heavy_first[src];
    }
    return out;
}

static void upload_operator(rad_htree* h, const HVec<IdxRun>& near_runs, const HVec<IdxRun>& far_runs,
                            cudaStream_t s) {
    long long nx = 0, nf = 0;
    for (auto& t : h->tiles_h) {
        t.ixn = (int)nx;
        t.ixf = (int)nf;
        nx += t.kn;
        nf += t.kf;
    }
    RAD_REQUIRE(nx < INT_MAX && nf < INT_MAX, RAD_ELIMIT, "gather lists exceed 2^31 entries");
    // Work lists, heaviest item first so that the long items start in the
    // first wave and the short ones fill the tail (longest-processing-time
    // order); ties keep the natural order.
    const auto& G = h->groups_h;
    auto split_groups = [&](int rows_per_item) {
        std::vector<GWork> w;
        for (int g = 0; g < (int)G.size(); ++g)
            for (int r = 0; r < G[g].M; r += rows_per_item)
                w.push_back(GWork{g, r, std::min(rows_per_item, G[g].M - r), 0});
        std::vector<long long> key(w.size());
        for (size_t i = 0; i < w.size(); ++i) key[i] = (long long)w[i].rows * G[w[i].g].n;
        std::vector<GWork> sorted(w.size());
        const std::vector<int> ord = order_desc(key);
        for (size_t i = 0; i < w.size(); ++i) sorted[i] = w[ord[i]];
        w.swap(sorted);
        return w;
    };
    std::vector<GWork> gwork = split_groups(kTileRows);
    {
        // one CTA per item, dealt across the SMs in snake order
        const std::vector<int> ident_order = [&] {
            std::vector<int> v(gwork.size());
            std::iota(v.begin(), v.end(), 0);
            return v;
        }();
        const std::vector<int> so = snake_order(ident_order, sm_count());
        std::vector<GWork> g2(gwork.size());
        for (size_t i = 0; i < so.size(); ++i) g2[i] = gwork[so[i]];
        gwork.swap(g2);
    }
    std::vector<long long> tkey(h->tiles_h.size());
    for (size_t t = 0; t < tkey.size(); ++t) {
        const Tile& tl = h->tiles_h[t];
        tkey[t] = (long long)tl.ld * (tl.kn + tl.kf);
    }
    const std::vector<int> torder = snake_order(order_desc(tkey), sm_count());
    std::vector<long long> fkey(h->tiles_h.size());
    for (size_t t = 0; t < fkey.size(); ++t) fkey[t] = (long long)h->tiles_h[t].ld * h->tiles_h[t].kf;
    const std::vector<int> forder = order_desc(fkey);
    h->n_tiles = (int)h->tiles_h.size();
    h->n_gwork = (int)gwork.size();
    h->gwork_h = gwork;
    h->d_torder.alloc(sizeof(int) * std::max<size_t>(1, torder.size()), s);
    h->d_forder.alloc(sizeof(int) * std::max<size_t>(1, forder.size()), s);
    h2d(h->d_torder.as<int>(), torder, s);
    h2d(h->d_forder.as<int>(), forder, s);
    build_stream_lists(h, h->stream_rows, s);
    h->d_tiles.alloc(sizeof(Tile) * std::max<size_t>(1, h->tiles_h.size()), s);
    // 4 ints of slack after each list: the fused one-column product copies
    // index slices in whole 16-byte words
    h->d_xidx.alloc(sizeof(int) * (std::max<long long>(1, nx) + 4), s);
    h->d_tidx.alloc(sizeof(int) * (std::max<long long>(1, nf) + 4), s);
    h->d_gwork.alloc(sizeof(GWork) * std::max<size_t>(1, gwork.size()), s);
    h->d_groups.alloc(sizeof(Group) * std::max<size_t>(1, h->groups_h.size()), s);
    h2d(h->d_tiles.as<Tile>(), h->tiles_h, s);
    h2d(h->d_gwork.as<GWork>(), gwork, s);
    h2d(h->d_groups.as<Group>(), h->groups_h, s);
    Scratch ws(s);
    const HVec<IdxRun>* lists[2] = {&near_runs, &far_runs};
    int* outs[2] = {h->d_xidx.as<int>(), h->d_tidx.as<int>()};
    for (int f = 0; f < 2; ++f) {
        const HVec<IdxRun>& rl = *lists[f];
        if (rl.empty()) continue;
        IdxRun* d = ws.get_n<IdxRun>(rl.size());
        h2d(d, rl, s);
        { ProfScope ps_("gather_lists", s); fill_runs_kernel<<<(unsigned)((rl.size() + 7) / 8), 256, 0, s>>>(d, (int)rl.size(), h->d_tiles.as<Tile>(), f, outs[f]); }
        RAD_CHECK_LAUNCH();
    }
    hmv1_plan(h, s);
}

template <class S, class CT>
static void launch_dense_fill(rad_htree* h, const HVec<DenseWork>& work, cudaStream_t s) {
    if (work.empty()) return;
    Scratch ws(s);
    DenseWork* d_work = ws.get_n<DenseWork>(work.size());
    h2d(d_work, work, s);
    const Geo g = geo_view(h->geo.as<double>(), h->geo32.as<float>(), h->n);
    { ProfScope ps_("near_assemble", s); dense_fill_kernel<S, CT><<<(unsigned)work.size(), 256, 0, s>>>(g, h->d_tiles.as<Tile>(), d_work, h->near_pool.as<S>()); }
    RAD_CHECK_LAUNCH();
}

template <class CT, class S>
static void launch_factor_fill(rad_htree* h, const HVec<UWork>& uw, const HVec<VWork>& vw,
                               const CT* const* Ubase, const CT* const* Vbase, cudaStream_t s, void* pool = nullptr) {
    S* dst = static_cast<S*>(pool ? pool : h->far_pool.p);
    Scratch ws(s);
    if (!uw.empty()) {
        UWork* d = ws.get_n<UWork>(uw.size());
        h2d(d, uw, s);
        { ProfScope ps_("aca_pack", s); u_fill_kernel<CT, S><<<(unsigned)((uw.size() + 7) / 8), 256, 0, s>>>(h->d_tiles.as<Tile>(), d, (int)uw.size(), Ubase, dst); }
        RAD_CHECK_LAUNCH();
    }
    if (!vw.empty()) {
        VWork* d = ws.get_n<VWork>(vw.size());
        h2d(d, vw, s);
        { ProfScope ps_("aca_pack", s); v_fill_kernel<CT, S><<<(unsigned)vw.size(), 256, 0, s>>>(h->d_groups.as<Group>(), d, Vbase, dst); }
        RAD_CHECK_LAUNCH();
    }
}

template <class CT>
void compress_t(rad_htree* h, const rad_aca_params* p, cudaStream_t s) {
    Scratch ws(s);
    // admissible blocks -> ACA jobs
    auto hs_jobs = std::make_unique<HostScope>("host_aca_jobs");
    std::vector<int> adm;
    for (int b = 0; b < (int)h->blocks.size(); ++b)
        if (h->blocks[b].admissible) adm.push_back(b);
    // jobs with their scratch offsets (running sums over the admissible
    // blocks in order), in parallel parts for large lists
    std::vector<AcaJob> jobs(adm.size());
    long long ou = 0, ov = 0, oused = 0;
    {
        const int64_t na = (int64_t)adm.size();
        const int P = na >= 8000 ? 16 : 1;
        std::vector<long long> su(P + 1, 0), sv(P + 1, 0), ss(P + 1, 0);
        auto kmax_of = [&](int m, int n) {
            const long long brk = (long long)m * n / (m + n);
            return (int)std::min<long long>({(long long)p->max_rank, brk, (long long)kMaxRank});
        };
        parallel_parts(P, [&](int q) {
            for (int64_t a = na * q / P, e = na * (q + 1) / P; a < e; ++a) {
                const BlockH& bk = h->blocks[adm[a]];
                const int m = bk.r1 - bk.r0, n = bk.c1 - bk.c0, kmax = kmax_of(m, n);
                su[q + 1] += round_up((long long)m * kmax, 8);
                sv[q + 1] += round_up((long long)n * kmax, 8);
                ss[q + 1] += round_up(m, 16);
            }
        });
        for (int q = 0; q < P; ++q) {
            su[q + 1] += su[q];
            sv[q + 1] += sv[q];
            ss[q + 1] += ss[q];
        }
        parallel_parts(P, [&](int q) {
            long long u = su[q], v = sv[q], us = ss[q];
            for (int64_t a = na * q / P, e = na * (q + 1) / P; a < e; ++a) {
                const BlockH& bk = h->blocks[adm[a]];
                const int m = bk.r1 - bk.r0, n = bk.c1 - bk.c0, kmax = kmax_of(m, n);
                jobs[a] = AcaJob{bk.r0, bk.c0, m, n, kmax, 0, u, v, us};
                u += round_up((long long)m * kmax, 8);
                v += round_up((long long)n * kmax, 8);
                us += round_up(m, 16);
            }
        });
        ou = su[P];
        ov = sv[P];
        oused = ss[P];
    }
    hs_jobs.reset();
    // ACA scratch holds kmax columns per block.  When that exceeds the
    // budget (large batches), the jobs run in chunks, and after each chunk
    // the first rank columns are compacted and the scratch is released.
    size_t free_b = 0, total_b = 0;
    RAD_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const long long budget =
        p->scratch_mib > 0 ? (long long)p->scratch_mib << 20
                           : std::max<long long>(1ll << 30, std::min<long long>((long long)(0.3 * (double)free_b), 48ll << 30));
    std::vector<int> ranks(jobs.size(), 0);
    std::vector<long long> evals(jobs.size(), 0);
    std::vector<long long> src_u(jobs.size(), 0), src_v(jobs.size(), 0);
    std::vector<int> job_chunk(jobs.size(), 0);
    std::vector<const CT*> ubase, vbase;
    if (!jobs.empty()) {
        HostScope hs_("host_aca_launch_wait");
        if ((ou + ov) * (long long)sizeof(CT) <= budget) {
            CT* Us = nullptr;
            CT* Vs = nullptr;
            launch_aca<CT>(h, p, jobs, ranks, evals, nullptr, ws, Us, Vs, s);
            for (size_t j = 0; j < jobs.size(); ++j) {
                src_u[j] = jobs[j].offU;
                src_v[j] = jobs[j].offV;
            }
            ubase.push_back(Us);
            vbase.push_back(Vs);
        } else {
            size_t j0 = 0;
            while (j0 < jobs.size()) {
                // jobs [j0, j1): scratch within the budget (at least one job)
                size_t j1 = j0;
                long long sz = 0;
                while (j1 < jobs.size()) {
                    const long long add = round_up((long long)jobs[j1].m * jobs[j1].kmax, 8) +
                                          round_up((long long)jobs[j1].n * jobs[j1].kmax, 8);
                    if (j1 > j0 && (sz + add) * (long long)sizeof(CT) > budget) break;
                    sz += add;
                    ++j1;
                }
                std::vector<AcaJob> cj(jobs.begin() + j0, jobs.begin() + j1);
                const long long bu = cj.front().offU, bv = cj.front().offV, bs = cj.front().offUsed;
                for (auto& j : cj) {
                    j.offU -= bu;
                    j.offV -= bv;
                    j.offUsed -= bs;
                }
                std::vector<int> cr;
                std::vector<long long> ce, cu(cj.size()), cv(cj.size());
                Scratch cws(s);
                CT* Us = nullptr;
                CT* Vs = nullptr;
                launch_aca<CT>(h, p, cj, cr, ce, nullptr, cws, Us, Vs, s);
                HostScope hs_cp("host_aca_compact_prep");
                long long tu = 0, tv = 0;
                for (size_t q = 0; q < cj.size(); ++q) {
                    cu[q] = tu;
                    cv[q] = tv;
                    const int k = std::max(cr[q], 0);
                    tu += (long long)cj[q].m * k;
                    tv += (long long)cj[q].n * k;
                }
                CT* Uc = ws.get_n<CT>(std::max<long long>(tu, 1));
                CT* Vc = ws.get_n<CT>(std::max<long long>(tv, 1));
                AcaJob* d_cj = cws.get_n<AcaJob>(cj.size());
                int* d_cr = cws.get_n<int>(cj.size());
                long long* d_cu = cws.get_n<long long>(cj.size());
                long long* d_cv = cws.get_n<long long>(cj.size());
                h2d(d_cj, cj, s);
                h2d(d_cr, cr, s);
                h2d(d_cu, cu, s);
                h2d(d_cv, cv, s);
                { ProfScope ps_("aca_compact", s); compact_kernel<CT><<<(unsigned)cj.size(), 256, 0, s>>>(d_cj, d_cr, d_cu, d_cv, Us, Vs, Uc, Vc); }
                RAD_CHECK_LAUNCH();
                for (size_t q = 0; q < cj.size(); ++q) {
                    ranks[j0 + q] = cr[q];
                    evals[j0 + q] = ce[q];
                    src_u[j0 + q] = cu[q];
                    src_v[j0 + q] = cv[q];
                    job_chunk[j0 + q] = (int)ubase.size();
                }
                ubase.push_back(Uc);
                vbase.push_back(Vc);
                j0 = j1;
            }
        }
    }
    const CT** d_ubase = ws.get_n<const CT*>(std::max<size_t>(1, ubase.size()));
    const CT** d_vbase = ws.get_n<const CT*>(std::max<size_t>(1, vbase.size()));
    if (!ubase.empty()) {
        RAD_CUDA(cudaMemcpyAsync(d_ubase, ubase.data(), sizeof(CT*) * ubase.size(), cudaMemcpyHostToDevice, s));
        RAD_CUDA(cudaMemcpyAsync(d_vbase, vbase.data(), sizeof(CT*) * vbase.size(), cudaMemcpyHostToDevice, s));
    }
    auto hs_plan = std::make_unique<HostScope>("host_plan");
    std::vector<int> job_of(h->blocks.size(), -1);
    h->aca_entries = 0;
    for (auto e : evals) h->aca_entries += e;

    // ---- storage plan: row tiles, column groups, panels
    std::vector<int> tile_at;
    make_tiles(h, h->tiles_h, tile_at);
    std::vector<Tile>& tiles = h->tiles_h;
    h->near_pieces.clear();
    h->far_pieces.clear();
    h->groups_h.clear();
    int64_t fallback = 0;
    // row ranges of the parallel plan (below): cut at tile starts
    const int nb = (int)h->blocks.size();
    const int parts = nb >= 20000 ? 16 : nb >= 8000 ? 8 : 1;
    std::vector<int> cut(parts + 1, 0);
    cut[parts] = (int)h->n;
    for (int q = 1; q < parts; ++q) {
        int r = (int)((long long)h->n * q / parts);
        while (r < (int)h->n && tile_at[r] < 0) ++r;
        cut[q] = std::max(cut[q - 1], r);
    }
    std::vector<std::vector<int>> part_blocks(parts), part_cross(parts);
    // one pass over the blocks: ACA job and rank, column group of the
    // low-rank blocks (k > 0, groups in order of first use), row range
    std::vector<int> group_of_node(h->nodes.size(), -1);
    size_t next_adm = 0;
    for (int b = 0; b < nb; ++b) {
        BlockH& bk = h->blocks[b];
        if (next_adm < adm.size() && adm[next_adm] == b) {
            job_of[b] = (int)next_adm;
            bk.rank = ranks[next_adm];
            ++next_adm;
        }
        {
            const int q = (int)(std::upper_bound(cut.begin(), cut.end(), bk.r0) - cut.begin()) - 1;
            if (bk.r1 > cut[q + 1]) {
                for (int q2 = q; q2 < parts && cut[q2] < bk.r1; ++q2) part_cross[q2].push_back(b);
            } else {
                part_blocks[q].push_back(b);
            }
        }
        bk.group = -1;
        bk.grow = 0;
        if (!bk.admissible) {
            bk.rank = -1;
            continue;
        }
        if (bk.rank < 0) {
            ++fallback;
            continue;
        }
        if (bk.rank == 0) continue;
        int& gid = group_of_node[bk.col_node];
        if (gid < 0) {
            gid = (int)h->groups_h.size();
            h->groups_h.push_back(Group{bk.c0, bk.c1 - bk.c0, 0, 0, 0, 0, 0});
        }
        bk.group = gid;
        bk.grow = h->groups_h[gid].M;
        h->groups_h[gid].M += bk.rank;
    }
    int toff = 0;
    for (auto& gr : h->groups_h) {
        gr.ld = (int)round_up(gr.M, 4);
        gr.toff = toff;
        toff += gr.M;
    }
    h->sum_rank = toff;
    // Per-tile panel columns, gather runs and fill work.  Large plans are
    // split into row ranges (8 from 8,000 blocks, 16 from 20,000) cut at
    // tile starts and built by threads (each range owns its tiles); the
    // pieces of blocks whose rows cross a cut come first in each range.
    // The layout is deterministic for a given block list (the part count
    // depends only on the block count, not on the machine).
    struct PlanPart {
        std::vector<DenseWork> dwork;
        std::vector<UWork> uwork;
        std::vector<VWork> vwork;
        std::vector<IdxRun> near_runs, far_runs;
        std::vector<Piece> near_pieces, far_pieces;
        int64_t near_e = 0, far_u = 0, far_v = 0;
        int maxk = 0;
    };
    // block b's pieces in the tiles of rows [lo, hi); the per-block items
    // (entry counts, the V^T fill) only for its owner part
    auto plan_block = [&](int b, PlanPart& o, int lo, int hi, bool owner) {
        const BlockH& bk = h->blocks[b];
        const int m = bk.r1 - bk.r0, n = bk.c1 - bk.c0;
        const int r0 = std::max(bk.r0, lo), r1 = std::min(bk.r1, hi);
        if (bk.rank < 0) {
            if (owner) o.near_e += (long long)m * n;
            for_tiles(tiles, tile_at, r0, r1, [&](int t) {
                o.near_pieces.push_back(Piece{b, t, tiles[t].kn});
                for (int c0 = 0; c0 < n; c0 += 64)
                    o.dwork.push_back(DenseWork{t, bk.c0 + c0, std::min(64, n - c0), tiles[t].kn + c0});
                o.near_runs.push_back(IdxRun{t, tiles[t].kn, bk.c0, n});
                tiles[t].kn += n;
            });
        } else if (bk.rank > 0) {
            const int k = bk.rank;
            const int jb = job_of[b];
            const Group& gr = h->groups_h[bk.group];
            if (owner) {
                o.maxk = std::max(o.maxk, k);
                o.far_u += (long long)k * m;
                o.far_v += (long long)k * n;
            }
            for_tiles(tiles, tile_at, r0, r1, [&](int t) {
                o.far_pieces.push_back(Piece{b, t, tiles[t].kf});
                o.uwork.push_back(UWork{t, tiles[t].r0 - bk.r0, m, k, tiles[t].kf, job_chunk[jb], src_u[jb]});
                o.far_runs.push_back(IdxRun{t, tiles[t].kf, gr.toff + bk.grow, k});
                tiles[t].kf += k;
            });
            if (owner) o.vwork.push_back(VWork{bk.group, bk.grow, n, k, job_chunk[jb], 0, src_v[jb]});
        }
    };
    // range q plans first the pieces of the blocks that cross into it from
    // other ranges (in block order), then its own blocks: per tile, the
    // same column order as one sequential pass over crossing blocks first
    std::vector<PlanPart> pp(parts);
    auto hs_parts = std::make_unique<HostScope>("host_plan_parts");
    parallel_parts(parts, [&](int q) {
        for (int b : part_cross[q]) {
            const BlockH& bk = h->blocks[b];
            plan_block(b, pp[q], cut[q], cut[q + 1], bk.r0 >= cut[q] && bk.r0 < cut[q + 1]);
        }
        for (int b : part_blocks[q]) plan_block(b, pp[q], cut[q], cut[q + 1], true);
    });
    hs_parts.reset();
    auto hs_merge = std::make_unique<HostScope>("host_plan_merge");
    // concatenation of the parts' lists in part order (copies in parallel)
    HVec<DenseWork> dwork;
    HVec<UWork> uwork;
    HVec<VWork> vwork;
    HVec<IdxRun> near_runs, far_runs;
    int64_t near_e = 0, far_u = 0, far_v = 0;
    int maxk = 0;
    {
        const int np = (int)pp.size();
        std::vector<size_t> od(np + 1, 0), ou_(np + 1, 0), ov_(np + 1, 0), onr(np + 1, 0), ofr(np + 1, 0),
            opn(np + 1, 0), opf(np + 1, 0);
        for (int q = 0; q < np; ++q) {
            const PlanPart& o = pp[q];
            od[q + 1] = od[q] + o.dwork.size();
            ou_[q + 1] = ou_[q] + o.uwork.size();
            ov_[q + 1] = ov_[q] + o.vwork.size();
            onr[q + 1] = onr[q] + o.near_runs.size();
            ofr[q + 1] = ofr[q] + o.far_runs.size();
            opn[q + 1] = opn[q] + o.near_pieces.size();
            opf[q + 1] = opf[q] + o.far_pieces.size();
            near_e += o.near_e; far_u += o.far_u; far_v += o.far_v;
            maxk = std::max(maxk, o.maxk);
        }
        dwork.resize(od[np]); uwork.resize(ou_[np]); vwork.resize(ov_[np]);
        near_runs.resize(onr[np]); far_runs.resize(ofr[np]);
        h->near_pieces.resize(opn[np]);
        h->far_pieces.resize(opf[np]);
        const bool par = nb >= 8000;
        parallel_parts(par ? np : 1, [&](int q0) {
            for (int q = (par ? q0 : 0); q < (par ? q0 + 1 : np); ++q) {
                const PlanPart& o = pp[q];
                std::copy(o.dwork.begin(), o.dwork.end(), dwork.begin() + od[q]);
                std::copy(o.uwork.begin(), o.uwork.end(), uwork.begin() + ou_[q]);
                std::copy(o.vwork.begin(), o.vwork.end(), vwork.begin() + ov_[q]);
                std::copy(o.near_runs.begin(), o.near_runs.end(), near_runs.begin() + onr[q]);
                std::copy(o.far_runs.begin(), o.far_runs.end(), far_runs.begin() + ofr[q]);
                std::copy(o.near_pieces.begin(), o.near_pieces.end(), h->near_pieces.begin() + opn[q]);
                std::copy(o.far_pieces.begin(), o.far_pieces.end(), h->far_pieces.begin() + opf[q]);
            }
        });
    }
    hs_merge.reset();
    long long noff = 0, foff = 0;
    for (auto& t : tiles) {
        t.noff = noff;
        noff += round_up((long long)t.ld * t.kn, 16);
        t.foff = foff;
        foff += round_up((long long)t.ld * t.kf, 16);
    }
    for (auto& gr : h->groups_h) {
        gr.voff = foff;
        foff += round_up((long long)gr.ld * gr.n, 16);
    }
    h->stored_near = noff;
    h->stored_far = foff;
    hs_plan.reset();
    auto hs_up = std::make_unique<HostScope>("host_alloc_upload_fill");
    const int ns = dtype_size(h->near_dtype);
    const int fs = dtype_size(h->factor_dtype);
    h->near_pool.alloc((size_t)std::max<long long>(noff, 16) * ns, s);
    h->far_pool.alloc((size_t)std::max<long long>(foff, 16) * fs, s);
    RAD_CUDA(cudaMemsetAsync(h->far_pool.p, 0, h->far_pool.bytes, s));
    upload_operator(h, near_runs, far_runs, s);
    if (h->near_dtype == RAD_F64) launch_dense_fill<double, double>(h, dwork, s);
    else launch_dense_fill<float, float>(h, dwork, s);
    if (h->factor_dtype == RAD_F64) launch_factor_fill<CT, double>(h, uwork, vwork, d_ubase, d_vbase, s);
    else if (h->factor_dtype == RAD_F32) launch_factor_fill<CT, float>(h, uwork, vwork, d_ubase, d_vbase, s);
    else launch_factor_fill<CT, __nv_bfloat16>(h, uwork, vwork, d_ubase, d_vbase, s);
    // accurate operator for mixed-precision refinement: FP32 factors
    h->far_pool_acc.release(s);
    h->has_accurate = false;
    if (p->accurate_dtype == RAD_F32) {
        if (h->factor_dtype == RAD_BF16) {
            h->far_pool_acc.alloc((size_t)std::max<long long>(foff, 16) * sizeof(float), s);
            RAD_CUDA(cudaMemsetAsync(h->far_pool_acc.p, 0, h->far_pool_acc.bytes, s));
            launch_factor_fill<CT, float>(h, uwork, vwork, d_ubase, d_vbase, s, h->far_pool_acc.p);
        }
        h->has_accurate = true;
    }
    if (h->factor_dtype == RAD_F64) h->has_accurate = true;
    h->n_dense_fallback = fallback;
    h->max_rank_used = maxk;
    h->near_entries = near_e;
    h->far_u_entries = far_u;
    h->far_v_entries = far_v;
    h->far_entries = far_u + far_v;
    // K-groups of the tensor-core path, counted now so that its images can be
    // built at the first many-column product without another synchronisation
    if (h->mm_path == 1) tc_count_async(h, s);
    hs_up.reset();
    HostScope hs_sync("host_compress_final_wait");
    RAD_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

void compress(rad_htree* h, const rad_aca_params* p, cudaStream_t s) {
    RAD_REQUIRE(p != nullptr, RAD_EINVAL, "null aca params");
    RAD_REQUIRE(p->tol >= 0.0 && p->tol == p->tol, RAD_EINVAL, "tol must be >= 0");
    RAD_REQUIRE(p->max_rank >= 0 && p->max_rank <= kMaxRank, RAD_EINVAL, "max_rank must be in [0, 128]");
    RAD_REQUIRE(p->pivoting == RAD_ACA_PARTIAL || p->pivoting == RAD_ACA_FULL, RAD_EINVAL, "bad pivoting");
    RAD_REQUIRE(p->near_dtype == RAD_F64 || p->near_dtype == RAD_F32, RAD_EINVAL, "near_dtype must be F64 or F32");
    RAD_REQUIRE(p->factor_dtype == RAD_F64 || p->factor_dtype == RAD_F32 || p->factor_dtype == RAD_BF16,
                RAD_EINVAL, "bad factor_dtype");
    RAD_REQUIRE((p->near_dtype == RAD_F64) == (p->factor_dtype == RAD_F64), RAD_EINVAL,
                "near_dtype F64 requires factor_dtype F64 and vice versa");
    RAD_REQUIRE(p->accurate_dtype == -1 || p->accurate_dtype == RAD_F32, RAD_EINVAL,
                "accurate_dtype must be -1 or RAD_F32");
    RAD_REQUIRE(p->scratch_mib >= 0, RAD_EINVAL, "scratch_mib must be >= 0");
    RAD_REQUIRE(p->recompress_tol >= 0.0 && p->recompress_tol < 1.0, RAD_EINVAL,
                "recompress_tol must be in [0, 1)");
    RAD_REQUIRE(!h->from_dense, RAD_EINVAL, "a dense-wrapped handle cannot be recompressed");
    drop_product_graph(h);
    h->stream_rows = kStreamRows;
    h->grid_a1 = h->grid_b1 = h->grid_a2 = h->grid_b2 = 0;
    h->tuned = 0;
    h->mm_path = p->near_dtype == RAD_F64 ? 0 : 1;   // tensor cores for FP32 / BF16 operators
    h->one_col_path = 1;
    tc_drop_images(h, s);
    h->tc_cnt_h.clear();
    h->closed = 0;
    h->compressed = false;
    h->factor_dtype = p->factor_dtype;
    h->near_dtype = p->near_dtype;
    h->tol = p->tol;
    h->pivoting = p->pivoting;
    // ACA arithmetic: FP64 for the FP64 path and for tolerances below 1e-6
    // (near FP32 resolution); FP32 otherwise (hi/lo centroid differences,
    // two-sum running norm).
    StageScope stage;
    if (p->near_dtype == RAD_F64 || p->tol < 1e-6) compress_t<double>(h, p, s);
    else compress_t<float>(h, p, s);
    h->compressed = true;
}

void load_dense_operator(rad_htree* h, const double* F_dev, cudaStream_t s) {
    const int n = (int)h->n;
    h->near_dtype = RAD_F64;
    h->factor_dtype = RAD_F64;
    h->blocks.assign(1, BlockH{0, 0, 0, n, 0, n, 0, -1, -1, 0});
    std::vector<int> tile_at;
    make_tiles(h, h->tiles_h, tile_at);
    HVec<IdxRun> near_runs, far_runs;
    h->near_pieces.clear();
    h->far_pieces.clear();
    h->groups_h.clear();
    long long noff = 0;
    for (size_t t = 0; t < h->tiles_h.size(); ++t) {
        Tile& tl = h->tiles_h[t];
        tl.kn = n;
        tl.noff = noff;
        tl.foff = 0;
        noff += round_up((long long)tl.ld * n, 16);
        h->near_pieces.push_back(Piece{0, (int)t, 0});
        near_runs.push_back(IdxRun{(int)t, 0, 0, n});
    }
    h->sum_rank = 0;
    h->stored_near = noff;
    h->stored_far = 0;
    h->near_pool.alloc(sizeof(double) * (size_t)std::max<long long>(noff, 16), s);
    h->far_pool.alloc(16 * sizeof(double), s);
    upload_operator(h, near_runs, far_runs, s);
    dim3 grid((unsigned)std::min<long long>(1024, ((long long)n * 64 + 255) / 256), (unsigned)h->tiles_h.size());
    { ProfScope ps_("dense_load", s); dense_from_matrix_kernel<<<grid, 256, 0, s>>>(n, h->d_tiles.as<Tile>(), F_dev, h->near_pool.as<double>()); }
    RAD_CHECK_LAUNCH();
    h->near_entries = (long long)n * n;
    h->far_entries = h->far_u_entries = h->far_v_entries = 0;
    h->has_accurate = true;
    RAD_CUDA(cudaStreamSynchronize(s));
    h->compressed = true;
}

static void to_double(const void* src, int dt, size_t cnt, std::vector<double>& out) {
    out.resize(cnt);
    if (dt == RAD_F64) {
        std::memcpy(out.data(), src, cnt * 8);
    } else if (dt == RAD_F32) {
        const float* f = static_cast<const float*>(src);
        for (size_t i = 0; i < cnt; ++i) out[i] = f[i];
    } else {
        const uint16_t* b = static_cast<const uint16_t*>(src);
        for (size_t i = 0; i < cnt; ++i) {
            uint32_t bits = (uint32_t)b[i] << 16;
            float f;
            std::memcpy(&f, &bits, 4);
            out[i] = f;
        }
    }
}

void export_block(const rad_htree* h, int64_t b, double* D, double* U, double* V) {
    RAD_REQUIRE(h->compressed, RAD_EINVAL, "handle is not compressed");
    RAD_REQUIRE(b >= 0 && b < (int64_t)h->blocks.size(), RAD_EINVAL, "block index out of range");
    const BlockH& bk = h->blocks[b];
    const int m = bk.r1 - bk.r0, n = bk.c1 - bk.c0;
    std::vector<unsigned char> raw;
    std::vector<double> cm;
    auto fetch = [&](const void* pool, int dt, long long off, size_t cnt) {
        const int sz = dtype_size(dt);
        raw.resize(cnt * sz);
        RAD_CUDA(cudaMemcpy(raw.data(), static_cast<const char*>(pool) + off * sz, raw.size(),
                            cudaMemcpyDeviceToHost));
        to_double(raw.data(), dt, cnt, cm);
    };
    if (bk.rank < 0) {
        if (!D) return;
        for (const Piece& pc : h->near_pieces) {
            if (pc.block != b) continue;
            const Tile& t = h->tiles_h[pc.tile];
            fetch(h->near_pool.p, h->near_dtype, t.noff + (long long)pc.col * t.ld, (size_t)n * t.ld);
            for (int i = 0; i < t.rows; ++i)
                for (int c = 0; c < n; ++c) D[(size_t)(t.r0 - bk.r0 + i) * n + c] = cm[(size_t)c * t.ld + i];
        }
        return;
    }
    const int k = bk.rank;
    if (k == 0) return;
    if (U)
        for (const Piece& pc : h->far_pieces) {
            if (pc.block != b) continue;
            const Tile& t = h->tiles_h[pc.tile];
            fetch(h->far_pool.p, h->factor_dtype, t.foff + (long long)pc.col * t.ld, (size_t)k * t.ld);
            for (int i = 0; i < t.rows; ++i)
                for (int l = 0; l < k; ++l) U[(size_t)(t.r0 - bk.r0 + i) * k + l] = cm[(size_t)l * t.ld + i];
        }
    if (V) {
        const Group& gr = h->groups_h[bk.group];
        fetch(h->far_pool.p, h->factor_dtype, gr.voff, (size_t)gr.ld * gr.n);
        for (int j = 0; j < n; ++j)
            for (int l = 0; l < k; ++l) V[(size_t)j * k + l] = cm[(size_t)j * gr.ld + bk.grow + l];
    }
}

}  // namespace rad
