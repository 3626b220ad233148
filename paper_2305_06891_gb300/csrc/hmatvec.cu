// A6: the block low-rank matrix-vector product y = F x of §5.2, in tree
// order, in two phases:
//   phase 1  t_b = V_b^T x_tau           for every low-rank block b
//   phase 2  y_rho = sum_near D x_tau + sum_far U t_b   per row tile rho
// Phase 2 gives every row tile (a leaf cluster, <= 64 rows) to one CTA, which
// owns its output rows: no atomics, a fixed summation order, deterministic.
//
// Dense blocks and U, V are stored column-major, so a tile's rows of a block
// are one contiguous run per column: with one thread per row, each warp
// load is 32 consecutive elements (fully coalesced streaming from HBM).
//
// One right-hand side: phase 1 is one warp per row of V^T (lanes over the
// block's columns, shuffle reduction); phase 2 spreads a tile's blocks over
// the CTA's warps and reduces the partial rows through shared memory in a
// fixed order.
// Many right-hand sides: both phases are small gathered GEMMs; A (block
// rows) and B (rows of X or T) are staged through shared memory in K-chunks
// and every thread accumulates a 4 x RN register tile (FP32 or FP64 FFMA).
//
// Epilogues fuse the reflection operator of Eq. (11):
//   kReflect: w = xin - (1 - eps) o (F x)
//   kResid:   r = b - (xin - (1 - eps) o (F x))

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
template <class FS, class AT>
__global__ void __launch_bounds__(256) phase1_single(OpView op, const AT* __restrict__ X, AT* __restrict__ T) {
    const int w = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= op.sum_rank) return;
    const int b = op.trow_block[w];
    const FarDesc f = op.fd[b];
    const int l = w - f.toff;
    const FS* v = static_cast<const FS*>(op.far_pool) + f.offV + (long long)l * f.n;
    const AT* x = X + f.c0;
    AT a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    int j = lane;
    for (; j + 96 < f.n; j += 128) {
        a0 += (AT)Store<FS>::get(v[j]) * x[j];
        a1 += (AT)Store<FS>::get(v[j + 32]) * x[j + 32];
        a2 += (AT)Store<FS>::get(v[j + 64]) * x[j + 64];
        a3 += (AT)Store<FS>::get(v[j + 96]) * x[j + 96];
    }
    for (; j < f.n; j += 32) a0 += (AT)Store<FS>::get(v[j]) * x[j];
    AT acc = warp_sum((a0 + a1) + (a2 + a3));
    if (lane == 0) T[w] = acc;
}

template <class NS, class FS, class AT>
__global__ void __launch_bounds__(256)
phase2_single(OpView op, const AT* __restrict__ X, const AT* __restrict__ T, void* Y, Epi epi) {
    __shared__ AT part[8][kTileRows];
    const TileDesc t = op.tiles[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nh = (t.rows + 31) >> 5;
    const int hh = warp % nh, g = warp / nh, ng = 8 / nh;
    const int row = hh * 32 + lane;
    const bool active = row < t.rows;
    AT acc = 0;
    for (int e = t.e0 + g; e < t.e1; e += ng) {
        const int2 en = op.entries[e];
        if (en.x & kFarBit) {
            const FarDesc f = op.fd[en.x & 0x7fffffff];
            if (active) {
                const FS* U = static_cast<const FS*>(op.far_pool) + f.offU + en.y + row;
                const AT* tb = T + f.toff;
                AT s0 = 0, s1 = 0;
                int l = 0;
                for (; l + 1 < f.k; l += 2) {
                    s0 += (AT)Store<FS>::get(U[(long long)l * f.m]) * tb[l];
                    s1 += (AT)Store<FS>::get(U[(long long)(l + 1) * f.m]) * tb[l + 1];
                }
                if (l < f.k) s0 += (AT)Store<FS>::get(U[(long long)l * f.m]) * tb[l];
                acc += s0 + s1;
            }
        } else {
            const NearDesc d = op.nd[en.x];
            if (active) {
                const NS* D = static_cast<const NS*>(op.near_pool) + d.off + en.y + row;
                const AT* x = X + d.c0;
                const long long m = d.m;
                AT s0 = 0, s1 = 0, s2 = 0, s3 = 0;
                int j = 0;
                for (; j + 3 < d.n; j += 4) {
                    s0 += (AT)Store<NS>::get(D[(long long)j * m]) * x[j];
                    s1 += (AT)Store<NS>::get(D[(long long)(j + 1) * m]) * x[j + 1];
                    s2 += (AT)Store<NS>::get(D[(long long)(j + 2) * m]) * x[j + 2];
                    s3 += (AT)Store<NS>::get(D[(long long)(j + 3) * m]) * x[j + 3];
                }
                for (; j < d.n; ++j) s0 += (AT)Store<NS>::get(D[(long long)j * m]) * x[j];
                acc += (s0 + s1) + (s2 + s3);
            }
        }
    }
    if (active) part[g][row] = acc;
    __syncthreads();
    if ((int)threadIdx.x < t.rows) {
        const int r = threadIdx.x;
        AT s = 0;
        for (int q = 0; q < ng; ++q) s += part[q][r];
        epilogue<AT>(epi, Y, 1, t.r0 + r, 0, s);
    }
}

// ---------------------------------------------------------------- many RHS
constexpr int kKC = 16;

template <class AT, int RN>
struct MicroTile {
    AT acc[4][RN];
    __device__ void zero() {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < RN; ++q) acc[r][q] = 0;
    }
};

// Accumulate C(64 x NC) += A(rows x K) B(K x nc) through shared memory.
//   A(i, k) = Aptr[k * a_ld + i]  (a_colmajor) or Aptr[i * a_ld + k]
//   B(k, c) = Bptr[k * ldb + c]
template <class AS, class AT, int RN>
__device__ __forceinline__ void gemm_tile(MicroTile<AT, RN>& mt, AT (*As)[kTileRows + 4], AT (*Bs)[16 * RN + 4],
                                          const AS* Aptr, long long a_ld, bool a_colmajor, int rows, int K,
                                          const AT* Bptr, long long ldb, int nc) {
    constexpr int NC = 16 * RN;
    const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
    for (int k0 = 0; k0 < K; k0 += kKC) {
        if (a_colmajor) {
            for (int q = threadIdx.x; q < kKC * kTileRows; q += 256) {
                const int kk = q / kTileRows, i = q - kk * kTileRows;
                AT v = 0;
                if (i < rows && k0 + kk < K) v = (AT)Store<AS>::get(Aptr[(long long)(k0 + kk) * a_ld + i]);
                As[kk][i] = v;
            }
        } else {
            for (int q = threadIdx.x; q < kKC * kTileRows; q += 256) {
                const int i = q / kKC, kk = q - i * kKC;
                AT v = 0;
                if (i < rows && k0 + kk < K) v = (AT)Store<AS>::get(Aptr[(long long)i * a_ld + k0 + kk]);
                As[kk][i] = v;
            }
        }
        for (int q = threadIdx.x; q < kKC * NC; q += 256) {
            const int kk = q / NC, c = q - kk * NC;
            AT v = 0;
            if (c < nc && k0 + kk < K) v = Bptr[(long long)(k0 + kk) * ldb + c];
            Bs[kk][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kKC; ++kk) {
            AT a[4], b[RN];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][tr * 4 + r];
#pragma unroll
            for (int q = 0; q < RN; ++q) b[q] = Bs[kk][tc + 16 * q];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < RN; ++q) mt.acc[r][q] += a[r] * b[q];
        }
        __syncthreads();
    }
}

template <class FS, class AT, int RN>
__global__ void __launch_bounds__(256)
phase1_multi(OpView op, const AT* __restrict__ X, int ldx, AT* __restrict__ T, int ldt, int nc) {
    __shared__ AT As[kKC][kTileRows + 4];
    __shared__ AT Bs[kKC][16 * RN + 4];
    const FarDesc f = op.fd[op.far_nz[blockIdx.x]];
    const FS* V = static_cast<const FS*>(op.far_pool) + f.offV;
    const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
    for (int l0 = 0; l0 < f.k; l0 += kTileRows) {
        MicroTile<AT, RN> mt;
        mt.zero();
        gemm_tile<FS, AT, RN>(mt, As, Bs, V + (long long)l0 * f.n, f.n, false, min(kTileRows, f.k - l0), f.n,
                              X + (long long)f.c0 * ldx, ldx, nc);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int l = l0 + tr * 4 + r;
            if (l >= f.k) continue;
#pragma unroll
            for (int q = 0; q < RN; ++q) {
                const int c = tc + 16 * q;
                if (c < nc) T[(long long)(f.toff + l) * ldt + c] = mt.acc[r][q];
            }
        }
    }
}

template <class NS, class FS, class AT, int RN>
__global__ void __launch_bounds__(256)
phase2_multi(OpView op, const AT* __restrict__ X, int ldx, const AT* __restrict__ T, int ldt, void* Y, int ldy,
             int nc, Epi epi) {
    __shared__ AT As[kKC][kTileRows + 4];
    __shared__ AT Bs[kKC][16 * RN + 4];
    const TileDesc t = op.tiles[blockIdx.x];
    MicroTile<AT, RN> mt;
    mt.zero();
    for (int e = t.e0; e < t.e1; ++e) {
        const int2 en = op.entries[e];
        if (en.x & kFarBit) {
            const FarDesc f = op.fd[en.x & 0x7fffffff];
            const FS* U = static_cast<const FS*>(op.far_pool) + f.offU + en.y;
            gemm_tile<FS, AT, RN>(mt, As, Bs, U, f.m, true, t.rows, f.k, T + (long long)f.toff * ldt, ldt, nc);
        } else {
            const NearDesc d = op.nd[en.x];
            const NS* D = static_cast<const NS*>(op.near_pool) + d.off + en.y;
            gemm_tile<NS, AT, RN>(mt, As, Bs, D, d.m, true, t.rows, d.n, X + (long long)d.c0 * ldx, ldx, nc);
        }
    }
    const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int row = tr * 4 + r;
        if (row >= t.rows) continue;
#pragma unroll
        for (int q = 0; q < RN; ++q) {
            const int c = tc + 16 * q;
            if (c < nc) epilogue<AT>(epi, Y, ldy, t.r0 + row, c, mt.acc[r][q]);
        }
    }
}

template <class NS, class FS, class AT, int RN>
void launch_multi(const rad_htree* h, const AT* X, int ldx, AT* T, int ldt, void* Y, int ldy, int nc,
                  const Epi& epi, cudaStream_t s) {
    const OpView op = h->view();
    if (op.n_far_nz > 0) {
        { ProfScope ps_("hmm_far_vt", s); phase1_multi<FS, AT, RN><<<op.n_far_nz, 256, 0, s>>>(op, X, ldx, T, ldt, nc); }
        RAD_CHECK_LAUNCH();
    }
    { ProfScope ps_("hmm_rows", s); phase2_multi<NS, FS, AT, RN><<<op.n_tiles, 256, 0, s>>>(op, X, ldx, T, ldt, Y, ldy, nc, epi); }
    RAD_CHECK_LAUNCH();
}

template <class NS, class FS, class AT>
void apply_t(const rad_htree* h, const AT* X, int ldx, void* Y, int ldy, int nrhs, const Epi& epi, AT* T,
             cudaStream_t s) {
    const OpView op = h->view();
    if (nrhs == 1) {
        if (op.sum_rank > 0) {
            { ProfScope ps_("hmv_far_vt", s); phase1_single<FS, AT><<<(op.sum_rank + 7) / 8, 256, 0, s>>>(op, X, T); }
            RAD_CHECK_LAUNCH();
        }
        { ProfScope ps_("hmv_rows", s); phase2_single<NS, FS, AT><<<op.n_tiles, 256, 0, s>>>(op, X, T, Y, epi); }
        RAD_CHECK_LAUNCH();
        return;
    }
    const int esz = epi.mode == kStore ? (int)sizeof(AT) : 8;
    for (int c0 = 0; c0 < nrhs; c0 += 128) {
        const int nc = std::min(128, nrhs - c0);
        Epi e2 = epi;
        if (epi.mode != kStore) {
            e2.xin = epi.xin + c0;
            if (epi.b) e2.b = epi.b + c0;
        }
        const AT* Xc = X + c0;
        AT* Tc = T + c0;
        void* Yc = static_cast<char*>(Y) + (size_t)c0 * esz;
        const int rn = (nc + 15) / 16;
        switch (rn) {
            case 1: launch_multi<NS, FS, AT, 1>(h, Xc, ldx, Tc, nrhs, Yc, ldy, nc, e2, s); break;
            case 2: launch_multi<NS, FS, AT, 2>(h, Xc, ldx, Tc, nrhs, Yc, ldy, nc, e2, s); break;
            case 3: launch_multi<NS, FS, AT, 3>(h, Xc, ldx, Tc, nrhs, Yc, ldy, nc, e2, s); break;
            case 4: launch_multi<NS, FS, AT, 4>(h, Xc, ldx, Tc, nrhs, Yc, ldy, nc, e2, s); break;
            case 5: launch_multi<NS, FS, AT, 5>(h, Xc, ldx, Tc, nrhs, Yc, ldy, nc, e2, s); break;
            case 6: launch_multi<NS, FS, AT, 6>(h, Xc, ldx, Tc, nrhs, Yc, ldy, nc, e2, s); break;
            case 7: launch_multi<NS, FS, AT, 7>(h, Xc, ldx, Tc, nrhs, Yc, ldy, nc, e2, s); break;
            default: launch_multi<NS, FS, AT, 8>(h, Xc, ldx, Tc, nrhs, Yc, ldy, nc, e2, s); break;
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
    return esz * (size_t)std::max(1, h->sum_rank) * (size_t)nrhs;
}

void apply_tree(const rad_htree* h, const void* X, int ldx, void* Y, int ldy, int nrhs, const Epi& epi,
                void* T_ws, cudaStream_t s) {
    if (h->op_is_f64()) {
        apply_t<double, double, double>(h, static_cast<const double*>(X), ldx, Y, ldy, nrhs, epi,
                                        static_cast<double*>(T_ws), s);
    } else if (h->factor_dtype == RAD_F32) {
        apply_t<float, float, float>(h, static_cast<const float*>(X), ldx, Y, ldy, nrhs, epi,
                                     static_cast<float*>(T_ws), s);
    } else {
        apply_t<float, __nv_bfloat16, float>(h, static_cast<const float*>(X), ldx, Y, ldy, nrhs, epi,
                                             static_cast<float*>(T_ws), s);
    }
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

}  // namespace rad
