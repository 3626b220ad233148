// Hierarchical block LU of the reflection matrix C = I - diag(1 - eps) F
// (§5.1) and the forward and backward substitution with its factors (§5.2),
// on the GPU.
//
// The factorisation keeps the paper's block structure (the leaves of the
// handle's block tree, Algorithm 2) and follows its definition: the block
// products and substitutions are formed, then brought back into the block
// format with the ranks of the admissible leaves truncated at eps_rel.
//   1. C is expanded once into a dense working matrix M (tree order,
//      column-major) from the handle's stored operator F~ (dense blocks, and
//      U V^T of the low-rank blocks): M = I - diag(1 - eps) F~; every
//      admissible leaf of M is then truncated.
//   2. Recursion on the diagonal cluster pairs (tau, tau).  A leaf pair gets
//      a dense LU without pivoting (C is strictly diagonally dominant by rows
//      for the cavities of this library: max(1 - eps) < 1 and row sums of F
//      near 1).  A pair with children tau1, tau2 is a 2 x 2 block matrix:
//      its upper-left block is factorised first (recursively), the two
//      off-diagonal blocks become L21 = M21 U11^-1 and U12 = L11^-1 M12 by
//      triangular solves, the lower-right block is replaced by its Schur
//      complement M22 - L21 U12 and factorised (recursively).  After each of
//      the three updates every admissible leaf of the updated region is
//      truncated, and the block in M is replaced by its truncation so that
//      later steps use the truncated values.
//   3. The factors are then taken from M into compact storage: dense leaves
//      (a diagonal leaf holds its unit-lower L and upper U together) and the
//      low-rank leaves from their last truncation.  M is released.
//
// Truncation of a block X (m x n) at eps: cross approximation with full
// pivoting (Eq. 30) until ||X - U V^T||_F <= (eps / 2) ||X||_F, then QR of
// both factors (classical Gram-Schmidt, twice), the SVD of R_U R_V^T by
// one-sided Jacobi rotations, and the smallest rank whose dropped singular
// values have sqrt(sum s_i^2) <= (eps / 2) ||U V^T||_F (so that the block
// moves by at most about eps ||X||_F).  A block whose
// cross would need more than kcap = min(64, m n / (m + n)) terms stays dense.
//
// Substitutions (§5.2), forward L y = b then backward U x = y, follow the
// block structure: a triangular solve in every diagonal leaf, and between
// them one product per off-diagonal region with all its leaves (D x for a
// dense leaf, U (V^T x) for a low-rank one).
//
// Arithmetic is FP64 for an FP64 operator and FP32 otherwise (the factors
// are an approximation at eps_rel; the FP32 version serves eps_rel >= 1e-5
// and preconditioning).

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <unordered_map>
#include <vector>

#include "rad_device.cuh"

namespace rad {

namespace {

constexpr int kHluMaxLeaf = 128;   // diagonal leaves factorised in shared memory
constexpr int kHluMaxRank = 64;    // rank capacity of a truncated leaf

template <class T> __device__ __forceinline__ T eps_mach();
template <> __device__ __forceinline__ double eps_mach<double>() { return 2.220446049250313e-16; }
template <> __device__ __forceinline__ float eps_mach<float>() { return 1.1920929e-7f; }

// ------------------------------------------------------------ expansion of F~
// Dense piece of a row tile: M[r0 + i, c0 + j] = D[i + j ld] (i < rows, j < n).
struct ExpandDense {
    int r0, rows, c0, n, ld, pad;
    long long src;
};
// Low-rank piece: M[r0 + i, c0 + j] = sum_l U[uoff + i + l uld] V[voff + l + j vld].
struct ExpandLowRank {
    int r0, rows, c0, n, k, uld, vld, pad;
    long long uoff, voff;
};

template <class T, class S>
__global__ void __launch_bounds__(256) hlu_expand_dense_kernel(T* __restrict__ M, long long ldm,
                                                               const ExpandDense* __restrict__ jobs,
                                                               const S* __restrict__ pool) {
    const ExpandDense jb = jobs[blockIdx.x];
    const long long total = (long long)jb.rows * jb.n;
    for (long long e = threadIdx.x; e < total; e += blockDim.x) {
        const int i = (int)(e % jb.rows), j = (int)(e / jb.rows);
        M[(jb.r0 + i) + (long long)(jb.c0 + j) * ldm] = (T)Store<S>::get(pool[jb.src + i + (long long)j * jb.ld]);
    }
}

template <class T, class S>
__global__ void __launch_bounds__(256) hlu_expand_lowrank_kernel(T* __restrict__ M, long long ldm,
                                                                 const ExpandLowRank* __restrict__ jobs,
                                                                 const S* __restrict__ pool) {
    const ExpandLowRank jb = jobs[blockIdx.x];
    const long long total = (long long)jb.rows * jb.n;
    for (long long e = threadIdx.x; e < total; e += blockDim.x) {
        const int i = (int)(e % jb.rows), j = (int)(e / jb.rows);
        T acc = 0;
        for (int l = 0; l < jb.k; ++l)
            acc += (T)Store<S>::get(pool[jb.uoff + i + (long long)l * jb.uld]) *
                   (T)Store<S>::get(pool[jb.voff + l + (long long)j * jb.vld]);
        M[(jb.r0 + i) + (long long)(jb.c0 + j) * ldm] = acc;
    }
}

// M := I - diag(1 - eps) M  (rows in tree order); `segrow` (may be null)
// gives every row's cavity: entries between different cavities stay zero.
template <class T>
__global__ void hlu_reflection_kernel(T* __restrict__ M, int n, const double* __restrict__ eps_t) {
    const long long total = (long long)n * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), j = (int)(e / n);
        const double v = (double)M[e];
        M[e] = (T)((i == j ? 1.0 : 0.0) - (1.0 - eps_t[i]) * v);
    }
}

// ------------------------------------------------------------ dense kernels
// LU without pivoting of the m x m diagonal block at (r0, r0) of M, in place
// (unit lower L below the diagonal, U on and above).  A zero pivot sets bit 1
// of *err (the factors then hold inf/nan; the host reports it).
template <class T>
__global__ void __launch_bounds__(256) hlu_lu_leaf_kernel(T* __restrict__ M, long long ldm, int r0, int m,
                                                          int* __restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    T* A = reinterpret_cast<T*>(smem_raw);
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e % m, j = e / m;
        A[e] = M[(r0 + i) + (long long)(r0 + j) * ldm];
    }
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        const T piv = A[k + k * m];
        if (threadIdx.x == 0 && piv == T(0)) atomicOr(err, 1);
        for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) A[i + k * m] /= piv;
        __syncthreads();
        const int rem = m - k - 1;
        for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
            const int i = k + 1 + e % rem, j = k + 1 + e / rem;
            A[i + j * m] -= A[i + k * m] * A[k + j * m];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e % m, j = e / m;
        M[(r0 + i) + (long long)(r0 + j) * ldm] = A[e];
    }
}

// Triangular solves with an m x m triangle Tr (column-major, leading dim
// ldt, m <= 128) on nc right-hand sides X(l, c) = X[l rs + c cs], l < m:
//   kLowerUnit: X := L^-1 X,   L the unit lower triangle of Tr
//   kUpperT:    X := U^-T X,   U the upper triangle of Tr (so X^T := X^T U^-1)
//   kUpper:     X := U^-1 X
// One warp per right-hand side: lane j holds rows j, j + 32, j + 64, j + 96
// in registers; each eliminated value is broadcast by a shuffle, so there is
// no barrier and no shared memory.
enum TrsmMode { kLowerUnit = 0, kUpperT = 1, kUpper = 2 };
template <class T, int MODE>
__global__ void __launch_bounds__(256) hlu_trsm_kernel(const T* __restrict__ Tr, long long ldt, int m,
                                                       T* __restrict__ X, long long rs, long long cs, int nc) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (c >= nc) return;                       // whole warps leave together
    T* x = X + (long long)c * cs;
    T v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int l = lane + 32 * q;
        v[q] = l < m ? x[(long long)l * rs] : T(0);
    }
    if (MODE == kUpper) {
#pragma unroll
        for (int q = 3; q >= 0; --q) {
            for (int kk = 31; kk >= 0; --kk) {
                const int k = 32 * q + kk;
                if (k >= m) continue;
                if (lane == kk) v[q] /= Tr[k + (long long)k * ldt];
                const T xk = __shfl_sync(0xffffffffu, v[q], kk);
#pragma unroll
                for (int p = 0; p <= q; ++p) {
                    const int i = lane + 32 * p;
                    if (i < k) v[p] -= Tr[i + (long long)k * ldt] * xk;
                }
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            for (int kk = 0; kk < 32; ++kk) {
                const int k = 32 * q + kk;
                if (k >= m) break;
                if (MODE == kUpperT && lane == kk) v[q] /= Tr[k + (long long)k * ldt];
                const T xk = __shfl_sync(0xffffffffu, v[q], kk);
#pragma unroll
                for (int p = q; p < 4; ++p) {
                    const int i = lane + 32 * p;
                    if (i > k && i < m)
                        v[p] -= (MODE == kLowerUnit ? Tr[i + (long long)k * ldt] : Tr[k + (long long)i * ldt]) * xk;
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int l = lane + 32 * q;
        if (l < m) x[(long long)l * rs] = v[q];
    }
}

// C -= A B, column-major: C m x n (ldc), A m x k (lda), B k x n (ldb).
// 64 x 64 output tile per CTA, 4 x 4 per thread, k in chunks of 16 through
// shared memory.
template <class T>
__global__ void __launch_bounds__(256) hlu_gemm_kernel(int m, int n, int k, const T* __restrict__ A, long long lda,
                                                       const T* __restrict__ B, long long ldb, T* __restrict__ C,
                                                       long long ldc) {
    __shared__ T As[16][64 + 1];
    __shared__ T Bs[16][64 + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0;
    for (int kk = 0; kk < k; kk += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int r = e % 64, q = e / 64;   // A(i0 + r, kk + q)
            As[q][r] = (i0 + r < m && kk + q < k) ? A[(i0 + r) + (long long)(kk + q) * lda] : T(0);
            const int q2 = e % 16, c = e / 16;  // B(kk + q2, j0 + c)
            Bs[q2][c] = (kk + q2 < k && j0 + c < n) ? B[(kk + q2) + (long long)(j0 + c) * ldb] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            T a[4], b[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                a[t] = As[q][tx + 16 * t];
                b[t] = Bs[q][ty + 16 * t];
            }
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int t = 0; t < 4; ++t) acc[s][t] += a[s] * b[t];
        }
        __syncthreads();
    }
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int i = i0 + tx + 16 * s, j = j0 + ty + 16 * t;
            if (i < m && j < n) C[i + (long long)j * ldc] -= acc[s][t];
        }
}

// ------------------------------------------------------------ truncation
struct TruncJob {
    long long moff;      // block's first entry in M (row r0, column c0)
    long long uoff, voff;  // slots: U m x 2 kcap, V n x 2 kcap (column-major)
    int m, n, kcap, leaf;
};

template <class T>
__device__ __forceinline__ T block_sum256(T v, T* red) {
    return block_sum<256, T>(v, red);
}

// One CTA (256 threads) per admissible leaf; see the file comment.
// rank[leaf] receives the stored rank, or -1 when the block stays dense.
template <class T>
__global__ void __launch_bounds__(256) hlu_truncate_kernel(T* __restrict__ M, long long ldm,
                                                           const TruncJob* __restrict__ jobs, T* __restrict__ slots,
                                                           double tol, int* __restrict__ rank) {
    extern __shared__ unsigned char smem_raw[];
    const TruncJob jb = jobs[blockIdx.x];
    const int m = jb.m, n = jb.n, kc = jb.kcap;
    T* X = M + jb.moff;
    T* U = slots + jb.uoff;   // m x 2kc
    T* V = slots + jb.voff;   // n x 2kc
    T* Ru = reinterpret_cast<T*>(smem_raw);   // kc x kc
    T* Rv = Ru + kc * kc;
    T* Mk = Rv + kc * kc;                     // R_U R_V^T, then M Z
    T* Z = Mk + kc * kc;
    __shared__ T red[16];
    __shared__ ArgMaxT<T> ared[16];
    __shared__ int s_i, s_j, s_k, s_rank, s_rot;
    __shared__ T s_piv, s_norm2;
    __shared__ int perm[kHluMaxRank];
    __shared__ T sval[kHluMaxRank];
    const long long mn = (long long)m * n;
    const int tid = threadIdx.x;

    // ||X||_F^2 and the first pivot
    T nx2 = 0;
    ArgMaxT<T> am{T(-1), 0x7fffffff};
    for (long long e = tid; e < mn; e += 256) {
        const int i = (int)(e % m), j = (int)(e / m);
        const T x = X[i + (long long)j * ldm];
        nx2 += x * x;
        const int flat = i * n + j;   // row-major index: ties to the lowest (row, column)
        am = am_better(am, ArgMaxT<T>{fabs(x), flat});
    }
    nx2 = block_sum256(nx2, red);
    am = block_argmax<256, T>(am, ared);
    if (nx2 == T(0)) {
        if (tid == 0) rank[jb.leaf] = 0;
        return;
    }
    const T d2 = (T)(0.25 * tol * tol) * nx2;     // (eps / 2)^2 ||X||^2
    T r2 = nx2;
    int k = 0;
    for (;;) {
        if (r2 <= d2) break;
        if (k >= kc) break;
        if (tid == 0) {
            s_i = am.i / n;
            s_j = am.i % n;
            s_piv = X[s_i + (long long)s_j * ldm];
        }
        __syncthreads();
        const int pi = s_i, pj = s_j;
        const T piv = s_piv;
        if (piv == T(0)) break;
        for (int i = tid; i < m; i += 256) U[i + (long long)k * m] = X[i + (long long)pj * ldm];
        for (int j = tid; j < n; j += 256) V[j + (long long)k * n] = X[pi + (long long)j * ldm] / piv;
        __syncthreads();
        // R -= u v^T, with the norm and the next pivot in the same pass
        T s2 = 0;
        ArgMaxT<T> a2{T(-1), 0x7fffffff};
        const T* uk = U + (long long)k * m;
        const T* vk = V + (long long)k * n;
        for (long long e = tid; e < mn; e += 256) {
            const int i = (int)(e % m), j = (int)(e / m);
            T& x = X[i + (long long)j * ldm];
            x -= uk[i] * vk[j];
            s2 += x * x;
            a2 = am_better(a2, ArgMaxT<T>{fabs(x), i * n + j});
        }
        r2 = block_sum256(s2, red);
        am = block_argmax<256, T>(a2, ared);
        ++k;
    }
    if (r2 > d2) {
        // no cross within kcap terms: put the block back (residual + cross)
        for (long long e = tid; e < mn; e += 256) {
            const int i = (int)(e % m), j = (int)(e / m);
            T s = 0;
            for (int l = 0; l < k; ++l) s += U[i + (long long)l * m] * V[j + (long long)l * n];
            X[i + (long long)j * ldm] += s;
        }
        if (tid == 0) rank[jb.leaf] = -1;
        return;
    }
    if (k == 0) {
        if (tid == 0) rank[jb.leaf] = 0;
        for (long long e = tid; e < mn; e += 256) X[(e % m) + (e / m) * ldm] = 0;
        return;
    }
    // QR of U and V (classical Gram-Schmidt, twice); R in shared memory
    for (int side = 0; side < 2; ++side) {
        T* Q = side == 0 ? U : V;
        T* R = side == 0 ? Ru : Rv;
        const int rows = side == 0 ? m : n;
        for (int e = tid; e < kc * kc; e += 256) R[e] = 0;
        __syncthreads();
        for (int j = 0; j < k; ++j) {
            T* qj = Q + (long long)j * rows;
            T n0 = 0;
            for (int i = tid; i < rows; i += 256) n0 += qj[i] * qj[i];
            n0 = block_sum256(n0, red);
            for (int pass = 0; pass < 2; ++pass) {
                // r_l = q_l . q_j for l < j, one warp per l
                const int warp = tid / 32, lane = tid % 32;
                for (int l = warp; l < j; l += 8) {
                    const T* ql = Q + (long long)l * rows;
                    T s = 0;
                    for (int i = lane; i < rows; i += 32) s += ql[i] * qj[i];
                    s = warp_sum(s);
                    if (lane == 0) Mk[l] = s;   // Mk as scratch for the coefficients
                }
                __syncthreads();
                for (int i = tid; i < rows; i += 256) {
                    T s = 0;
                    for (int l = 0; l < j; ++l) s += Q[i + (long long)l * rows] * Mk[l];
                    qj[i] -= s;
                }
                if (tid < j) R[tid + j * kc] += Mk[tid];
                __syncthreads();
            }
            T nn = 0;
            for (int i = tid; i < rows; i += 256) nn += qj[i] * qj[i];
            nn = block_sum256(nn, red);
            const T nrm = sqrt(nn);
            const bool dep = !(nrm > T(16) * eps_mach<T>() * sqrt(n0)) || nrm == T(0);
            const T inv = dep ? T(0) : T(1) / nrm;
            for (int i = tid; i < rows; i += 256) qj[i] *= inv;
            if (tid == 0) R[j + j * kc] = dep ? T(0) : nrm;
            __syncthreads();
        }
    }
    // Mk = R_U R_V^T (k x k), Z = I
    for (int e = tid; e < k * k; e += 256) {
        const int i = e % k, j = e / k;
        T s = 0;
        for (int l = 0; l < k; ++l) s += Ru[i + l * kc] * Rv[j + l * kc];
        Mk[i + j * kc] = s;
        Z[i + j * kc] = i == j ? T(1) : T(0);
    }
    __syncthreads();
    // one-sided Jacobi on the columns of Mk (rotations accumulated in Z)
    for (int sweep = 0; sweep < 40; ++sweep) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        const int kk = k + (k & 1);   // round-robin over an even count
        for (int round = 0; round < kk - 1; ++round) {
            const int warp = tid / 32, lane = tid % 32;
            for (int pr = warp; pr < kk / 2; pr += 8) {
                // pair pr of this round (circle method: index kk - 1 fixed,
                // the others rotate; every pair meets once per sweep)
                const int a = (round + pr) % (kk - 1);
                const int b = pr == 0 ? kk - 1 : (round + kk - 1 - pr) % (kk - 1);
                if (a >= k || b >= k) continue;
                T al = 0, be = 0, ga = 0;
                for (int i = lane; i < k; i += 32) {
                    const T x = Mk[i + a * kc], y = Mk[i + b * kc];
                    al += x * x;
                    be += y * y;
                    ga += x * y;
                }
                al = warp_sum(al);
                be = warp_sum(be);
                ga = warp_sum(ga);
                if (!(fabs(ga) > T(8) * eps_mach<T>() * sqrt(al * be))) continue;
                const T zeta = (be - al) / (T(2) * ga);
                const T t = (zeta >= 0 ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
                const T c = T(1) / sqrt(T(1) + t * t), s = c * t;
                for (int i = lane; i < k; i += 32) {
                    const T x = Mk[i + a * kc], y = Mk[i + b * kc];
                    Mk[i + a * kc] = c * x - s * y;
                    Mk[i + b * kc] = s * x + c * y;
                    const T zx = Z[i + a * kc], zy = Z[i + b * kc];
                    Z[i + a * kc] = c * zx - s * zy;
                    Z[i + b * kc] = s * zx + c * zy;
                }
                if (lane == 0) atomicAdd(&s_rot, 1);
            }
            __syncthreads();
        }
        if (s_rot == 0) break;
        __syncthreads();
    }
    // singular values (column norms of Mk Z), sorted, and the rank
    for (int j = tid; j < k; j += 256) {
        T s = 0;
        for (int i = 0; i < k; ++i) s += Mk[i + j * kc] * Mk[i + j * kc];
        sval[j] = s;   // squared
    }
    __syncthreads();
    if (tid == 0) {
        T total = 0;
        for (int j = 0; j < k; ++j) {
            perm[j] = j;
            total += sval[j];
        }
        for (int a = 0; a < k; ++a)   // selection sort, descending (ties: lower index)
            for (int b = a + 1; b < k; ++b)
                if (sval[perm[b]] > sval[perm[a]]) {
                    const int t = perm[a];
                    perm[a] = perm[b];
                    perm[b] = t;
                }
        const T lim = (T)(0.25 * tol * tol) * total;     // (eps / 2)^2 ||U V^T||^2
        T tail = 0;
        int r = k;
        while (r > 1 && tail + sval[perm[r - 1]] <= lim) {
            tail += sval[perm[r - 1]];
            --r;
        }
        s_rank = total > T(0) ? r : 0;
        s_norm2 = total;
    }
    __syncthreads();
    const int r = s_rank;
    // U' = Q_U (Mk Z)_r -> columns kc.. of U;  V' = Q_V Z_r -> columns kc.. of V
    for (int i = tid; i < m; i += 256)
        for (int j = 0; j < r; ++j) {
            T s = 0;
            for (int l = 0; l < k; ++l) s += U[i + (long long)l * m] * Mk[l + perm[j] * kc];
            U[i + (long long)(kc + j) * m] = s;
        }
    for (int i = tid; i < n; i += 256)
        for (int j = 0; j < r; ++j) {
            T s = 0;
            for (int l = 0; l < k; ++l) s += V[i + (long long)l * n] * Z[l + perm[j] * kc];
            V[i + (long long)(kc + j) * n] = s;
        }
    __syncthreads();
    for (int i = tid; i < m; i += 256)
        for (int j = 0; j < r; ++j) U[i + (long long)j * m] = U[i + (long long)(kc + j) * m];
    for (int i = tid; i < n; i += 256)
        for (int j = 0; j < r; ++j) V[i + (long long)j * n] = V[i + (long long)(kc + j) * n];
    __syncthreads();
    // the block becomes its truncation
    for (long long e = tid; e < mn; e += 256) {
        const int i = (int)(e % m), j = (int)(e / m);
        T s = 0;
        for (int l = 0; l < r; ++l) s += U[i + (long long)l * m] * V[j + (long long)l * n];
        X[i + (long long)j * ldm] = s;
    }
    if (tid == 0) rank[jb.leaf] = r;
}

// ------------------------------------------------------------ extraction
struct CopyJob {
    long long src, dst;   // src in M (ld ldm) or in the slots (ld m); dst in a pool (ld m)
    int m, n, from_slots, pad;
};
template <class T>
__global__ void __launch_bounds__(256) hlu_copy_kernel(const T* __restrict__ M, long long ldm,
                                                       const T* __restrict__ slots, const CopyJob* __restrict__ jobs,
                                                       T* __restrict__ pool) {
    const CopyJob jb = jobs[blockIdx.x];
    const long long total = (long long)jb.m * jb.n;
    for (long long e = threadIdx.x; e < total; e += blockDim.x) {
        const int i = (int)(e % jb.m), j = (int)(e / jb.m);
        pool[jb.dst + e] = jb.from_slots ? slots[jb.src + e] : M[jb.src + i + (long long)j * ldm];
    }
}

// ------------------------------------------------------------ substitution
// Vectors: tree order, row-major n x nc (ld nc), type T.
// Phase 1 of a region product: t_b = V_b^T x[cols of b] for its low-rank
// leaves (k x nc each, at toff nc in the workspace).
struct RegLR {
    long long voff;   // V of the leaf (n x k, column-major)
    int c0, n, k, toff;
};
template <class T>
__global__ void __launch_bounds__(256) hlu_region_vt_kernel(const RegLR* __restrict__ jobs, const T* __restrict__ up,
                                                            const T* __restrict__ x, int nc, T* __restrict__ t) {
    const RegLR jb = jobs[blockIdx.x];
    if (nc >= 32) {
        // a thread per output (l, c), c fastest: coalesced reads of x rows
        for (int e = threadIdx.x; e < jb.k * nc; e += blockDim.x) {
            const int l = e / nc, c = e % nc;
            const T* v = up + jb.voff + (long long)l * jb.n;
            T s = 0;
            for (int j = 0; j < jb.n; ++j) s += v[j] * x[(long long)(jb.c0 + j) * nc + c];
            t[(long long)jb.toff * nc + e] = s;
        }
        return;
    }
    // few right-hand sides: a warp per output, lanes along the dot product
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int e = warp; e < jb.k * nc; e += 8) {
        const int l = e / nc, c = e % nc;
        const T* v = up + jb.voff + (long long)l * jb.n;
        T s = 0;
        for (int j = lane; j < jb.n; j += 32) s += v[j] * x[(long long)(jb.c0 + j) * nc + c];
        s = warp_sum(s);
        if (lane == 0) t[(long long)jb.toff * nc + e] = s;
    }
}
// Phase 2: one CTA per row segment (a leaf cluster of the region's rows);
// y[rows] -= sum over the leaves covering them of D x or U t.
struct RegRow {
    int r0, rows, p0, p1;   // pieces [p0, p1)
};
struct RegPiece {
    long long off;   // dense: D + (row offset in the leaf); low-rank: U + row offset
    int ld;          // leading dimension (the leaf's rows)
    int lowrank;     // 1: U t, 0: D x
    int c0, n;       // dense: columns; low-rank: n unused
    int k, toff;     // low-rank: rank and workspace offset
};
template <class T>
__global__ void __launch_bounds__(256) hlu_region_rows_kernel(const RegRow* __restrict__ segs,
                                                              const RegPiece* __restrict__ pieces,
                                                              const T* __restrict__ dp, const T* __restrict__ up,
                                                              const T* __restrict__ t, T* __restrict__ y, int nc) {
    const RegRow sg = segs[blockIdx.x];
    for (int e = threadIdx.x; e < sg.rows * nc; e += blockDim.x) {
        const int i = e / nc, c = e % nc;
        T s = 0;
        for (int p = sg.p0; p < sg.p1; ++p) {
            const RegPiece pc = pieces[p];
            if (pc.lowrank) {
                const T* u = up + pc.off + i;
                for (int l = 0; l < pc.k; ++l) s += u[(long long)l * pc.ld] * t[(long long)(pc.toff + l) * nc + c];
            } else {
                const T* d = dp + pc.off + i;
                for (int j = 0; j < pc.n; ++j) s += d[(long long)j * pc.ld] * y[(long long)(pc.c0 + j) * nc + c];
            }
        }
        y[(long long)(sg.r0 + i) * nc + c] -= s;
    }
}

template <class T>
__global__ void hlu_cast_kernel(const double* __restrict__ a, T* __restrict__ b, long long cnt) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < cnt) b[e] = (T)a[e];
}
template <class T>
__global__ void hlu_uncast_kernel(const T* __restrict__ a, double* __restrict__ b, long long cnt) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < cnt) b[e] = (double)a[e];
}

inline unsigned grid_of(long long cnt, int bs = 256) { return (unsigned)std::max<long long>(1, (cnt + bs - 1) / bs); }

}  // namespace
}  // namespace rad

// ------------------------------------------------------------ the factor object
struct rad_hlu {
    ~rad_hlu() { (void)cudaDeviceSynchronize(); }
    const rad_htree* h = nullptr;
    int n = 0;
    bool f64 = true;
    double tol = 0.0;
    int device = 0;
    struct Leaf {
        int r0, r1, c0, c1, adm;
        int rank = -1;                 // -1: dense
        long long doff = -1;           // dense pool offset (column-major, ld = rows)
        long long uoff = -1, voff = -1;  // low-rank pool offsets (U rows x rank, V cols x rank)
    };
    std::vector<Leaf> leaves;
    rad::DevBuf dpool, upool;          // factor storage (T)
    // solve schedule
    struct Op {
        int kind;       // 0 leaf forward, 1 leaf backward, 2 region product
        int r0, m;      // leaf: rows; region: segment range [r0, r0 + m) of d_segs
        long long doff; // leaf: diagonal block in dpool
        int lr0, lr1;   // region: low-rank jobs [lr0, lr1)
    };
    std::vector<Op> fwd, bwd;
    rad::DevBuf d_lr, d_segs, d_pieces;
    int sum_rank_t = 0;                // rows of the t workspace (per column)
    // statistics
    long long dense_entries = 0, lowrank_entries = 0;
    int max_rank = 0, n_lowrank = 0, n_fallback = 0;
    double factor_ms = 0.0;
};

namespace rad {
namespace {

struct HluStructure {
    const rad_htree* h;
    std::unordered_map<long long, int> leaf_of;   // (row node, col node) -> block
    long long key(int a, int b) const { return (long long)a * 1000003LL + b; }
    explicit HluStructure(const rad_htree* hh) : h(hh) {
        leaf_of.reserve(h->blocks.size() * 2);
        for (size_t b = 0; b < h->blocks.size(); ++b) leaf_of[key(h->blocks[b].row_node, h->blocks[b].col_node)] = (int)b;
    }
    // leaves of the region (sigma, rho), in a fixed (recursive) order
    void collect(int s, int r, std::vector<int>& out) const {
        auto it = leaf_of.find(key(s, r));
        if (it != leaf_of.end()) {
            out.push_back(it->second);
            return;
        }
        const NodeShape& a = h->nodes[s];
        const NodeShape& b = h->nodes[r];
        RAD_REQUIRE(!a.leaf && !b.leaf, RAD_ECUDA, "block tree does not cover a cluster pair");
        for (int x : {a.child0, a.child1})
            for (int y : {b.child0, b.child1}) collect(x, y, out);
    }
};

template <class T>
struct HluBuilder {
    rad_hlu* lu;
    const rad_htree* h;
    const HluStructure& st;
    cudaStream_t s;
    int n;
    T* M = nullptr;
    T* slots = nullptr;
    int* d_rank = nullptr;
    int* d_err = nullptr;
    std::vector<long long> slot_u, slot_v;   // per leaf (admissible), -1 otherwise
    std::vector<int> kcap;
    // truncation job lists per region, uploaded once
    std::vector<TruncJob> tjobs;
    std::unordered_map<long long, std::pair<int, int>> region_jobs;   // (s, r) -> [j0, j1)
    TruncJob* d_tjobs = nullptr;

    size_t trunc_smem(int kc) const { return (size_t)4 * kc * kc * sizeof(T); }

    void trsm(int mode, const T* Tr, long long ldt, int m, T* X, long long rs, long long cs, int nc) {
        if (nc <= 0 || m <= 0) return;
        const unsigned grid = (unsigned)((nc + 7) / 8);
        ProfScope ps_("hlu_trsm", s);
        if (mode == kLowerUnit) hlu_trsm_kernel<T, kLowerUnit><<<grid, 256, 0, s>>>(Tr, ldt, m, X, rs, cs, nc);
        else if (mode == kUpperT) hlu_trsm_kernel<T, kUpperT><<<grid, 256, 0, s>>>(Tr, ldt, m, X, rs, cs, nc);
        else hlu_trsm_kernel<T, kUpper><<<grid, 256, 0, s>>>(Tr, ldt, m, X, rs, cs, nc);
        RAD_CHECK_LAUNCH();
    }
    void gemm(int m, int nn, int k, const T* A, long long lda, const T* B, long long ldb, T* C, long long ldc) {
        if (m <= 0 || nn <= 0 || k <= 0) return;
        dim3 grid((unsigned)((m + 63) / 64), (unsigned)((nn + 63) / 64));
        ProfScope ps_("hlu_gemm", s);
        hlu_gemm_kernel<T><<<grid, 256, 0, s>>>(m, nn, k, A, lda, B, ldb, C, ldc);
        RAD_CHECK_LAUNCH();
    }
    T* at(int i, int j) const { return M + i + (long long)j * n; }

    // M[tau, cols] := L_tau^-1 M[tau, cols]
    void trsm_left(int tau, int c0, int c1) {
        const NodeShape& t = h->nodes[tau];
        if (t.leaf) {
            trsm(kLowerUnit, at(t.begin, t.begin), n, t.end - t.begin, at(t.begin, c0), 1, n, c1 - c0);
            return;
        }
        const NodeShape& a = h->nodes[t.child0];
        const NodeShape& b = h->nodes[t.child1];
        trsm_left(t.child0, c0, c1);
        gemm(b.end - b.begin, c1 - c0, a.end - a.begin, at(b.begin, a.begin), n, at(a.begin, c0), n, at(b.begin, c0), n);
        trsm_left(t.child1, c0, c1);
    }
    // M[rows, tau] := M[rows, tau] U_tau^-1
    void trsm_right(int tau, int r0, int r1) {
        const NodeShape& t = h->nodes[tau];
        if (t.leaf) {
            // X^T := U^-T X^T: the rows of M[rows, tau] are the right-hand sides
            trsm(kUpperT, at(t.begin, t.begin), n, t.end - t.begin, at(r0, t.begin), n, 1, r1 - r0);
            return;
        }
        const NodeShape& a = h->nodes[t.child0];
        const NodeShape& b = h->nodes[t.child1];
        trsm_right(t.child0, r0, r1);
        gemm(r1 - r0, b.end - b.begin, a.end - a.begin, at(r0, a.begin), n, at(a.begin, b.begin), n, at(r0, b.begin), n);
        trsm_right(t.child1, r0, r1);
    }
    void truncate_region(int sg, int rh) {
        if (lu->tol <= 0.0) return;
        auto it = region_jobs.find(st.key(sg, rh));
        if (it == region_jobs.end() || it->second.first == it->second.second) return;
        const int j0 = it->second.first, cnt = it->second.second - j0;
        ProfScope ps_("hlu_truncate", s);
        hlu_truncate_kernel<T><<<cnt, 256, trunc_smem(kHluMaxRank), s>>>(M, n, d_tjobs + j0, slots, lu->tol, d_rank);
        RAD_CHECK_LAUNCH();
    }
    void factor(int tau) {
        const NodeShape& t = h->nodes[tau];
        if (t.leaf) {
            const int m = t.end - t.begin;
            ProfScope ps_("hlu_lu_leaf", s);
            hlu_lu_leaf_kernel<T><<<1, 256, (size_t)m * m * sizeof(T), s>>>(M, n, t.begin, m, d_err);
            RAD_CHECK_LAUNCH();
            return;
        }
        const int c1 = t.child0, c2 = t.child1;
        const NodeShape& a = h->nodes[c1];
        const NodeShape& b = h->nodes[c2];
        factor(c1);
        trsm_left(c1, b.begin, b.end);
        truncate_region(c1, c2);
        trsm_right(c1, b.begin, b.end);
        truncate_region(c2, c1);
        gemm(b.end - b.begin, b.end - b.begin, a.end - a.begin, at(b.begin, a.begin), n, at(a.begin, b.begin), n,
             at(b.begin, b.begin), n);
        truncate_region(c2, c2);
        factor(c2);
    }
    // region truncation job lists: the three regions of every non-leaf
    // diagonal pair, and the whole diagonal pair of every root
    void plan_region(int sg, int rh) {
        std::vector<int> lv;
        st.collect(sg, rh, lv);
        const int j0 = (int)tjobs.size();
        for (int b : lv) {
            if (slot_u[b] < 0) continue;
            const BlockH& bk = h->blocks[b];
            TruncJob jb;
            jb.moff = bk.r0 + (long long)bk.c0 * n;
            jb.uoff = slot_u[b];
            jb.voff = slot_v[b];
            jb.m = bk.r1 - bk.r0;
            jb.n = bk.c1 - bk.c0;
            jb.kcap = kcap[b];
            jb.leaf = b;
            tjobs.push_back(jb);
        }
        region_jobs[st.key(sg, rh)] = {j0, (int)tjobs.size()};
    }
    void plan_node(int tau) {
        const NodeShape& t = h->nodes[tau];
        if (t.leaf) return;
        plan_region(t.child0, t.child1);
        plan_region(t.child1, t.child0);
        plan_region(t.child1, t.child1);
        plan_node(t.child0);
        plan_node(t.child1);
    }
};

std::vector<int> roots_of(const rad_htree* h) {
    std::vector<int> r;
    for (size_t q = 0; q < h->nodes.size(); ++q)
        if (h->nodes[q].level == 0) r.push_back((int)q);
    return r;
}

template <class T, class S>
void expand_operator(const rad_htree* h, T* M, const void* far_pool_v, Scratch& ws, cudaStream_t s) {
    const int n = (int)h->n;
    std::vector<ExpandDense> dj;
    std::vector<ExpandLowRank> lj;
    for (const Piece& pc : h->near_pieces) {
        const BlockH& bk = h->blocks[pc.block];
        const Tile& t = h->tiles_h[pc.tile];
        dj.push_back(ExpandDense{t.r0, t.rows, bk.c0, bk.c1 - bk.c0, t.ld, 0, t.noff + (long long)pc.col * t.ld});
    }
    for (const Piece& pc : h->far_pieces) {
        const BlockH& bk = h->blocks[pc.block];
        if (bk.rank <= 0) continue;
        const Tile& t = h->tiles_h[pc.tile];
        const Group& g = h->groups_h[bk.group];
        lj.push_back(ExpandLowRank{t.r0, t.rows, bk.c0, bk.c1 - bk.c0, bk.rank, t.ld, g.ld, 0,
                                   t.foff + (long long)pc.col * t.ld, g.voff + bk.grow});
    }
    if (!dj.empty()) {
        ExpandDense* d = ws.get_n<ExpandDense>(dj.size());
        RAD_CUDA(cudaMemcpyAsync(d, dj.data(), sizeof(ExpandDense) * dj.size(), cudaMemcpyHostToDevice, s));
        ProfScope ps_("hlu_expand", s);
        if (h->near_dtype == RAD_F64)
            hlu_expand_dense_kernel<T, double><<<(unsigned)dj.size(), 256, 0, s>>>(M, n, d, (const double*)h->near_pool.p);
        else
            hlu_expand_dense_kernel<T, float><<<(unsigned)dj.size(), 256, 0, s>>>(M, n, d, (const float*)h->near_pool.p);
        RAD_CHECK_LAUNCH();
    }
    if (!lj.empty()) {
        ExpandLowRank* d = ws.get_n<ExpandLowRank>(lj.size());
        RAD_CUDA(cudaMemcpyAsync(d, lj.data(), sizeof(ExpandLowRank) * lj.size(), cudaMemcpyHostToDevice, s));
        ProfScope ps_("hlu_expand", s);
        hlu_expand_lowrank_kernel<T, S><<<(unsigned)lj.size(), 256, 0, s>>>(M, n, d, (const S*)far_pool_v);
        RAD_CHECK_LAUNCH();
    }
    RAD_CUDA(cudaStreamSynchronize(s));   // the host job lists go out of scope
}

template <class T>
void set_smem_limits() {
    static bool done = false;   // per process and type; the attribute is per function
    if (done) return;
    const int big = 200 * 1024;
    RAD_CUDA(cudaFuncSetAttribute(hlu_lu_leaf_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    RAD_CUDA(cudaFuncSetAttribute(hlu_truncate_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    done = true;
}

template <class T>
void build_solve_schedule(rad_hlu* lu, const HluStructure& st, Scratch& ws, cudaStream_t s) {
    const rad_htree* h = lu->h;
    std::vector<RegLR> lr;
    std::vector<RegRow> segs;
    std::vector<RegPiece> pieces;
    int toff = 0;
    // one region product y[rows sg] -= A(sg, rh) x[rh]
    auto region = [&](int sg, int rh) -> rad_hlu::Op {
        std::vector<int> lv;
        st.collect(sg, rh, lv);
        rad_hlu::Op op{2, (int)segs.size(), 0, 0, (int)lr.size(), 0};
        std::unordered_map<int, int> t_of;
        for (int b : lv) {
            const rad_hlu::Leaf& L = lu->leaves[b];
            if (L.rank > 0) {
                t_of[b] = toff;
                lr.push_back(RegLR{L.voff, L.c0, L.c1 - L.c0, L.rank, toff});
                toff += L.rank;
            }
        }
        op.lr1 = (int)lr.size();
        // row segments: the leaf clusters below sg
        std::vector<int> stack{sg};
        std::vector<int> leafc;
        while (!stack.empty()) {
            const int q = stack.back();
            stack.pop_back();
            const NodeShape& nd = h->nodes[q];
            if (nd.leaf) leafc.push_back(q);
            else {
                stack.push_back(nd.child1);
                stack.push_back(nd.child0);
            }
        }
        for (int q : leafc) {
            const NodeShape& nd = h->nodes[q];
            RegRow sgm{nd.begin, nd.end - nd.begin, (int)pieces.size(), 0};
            for (int b : lv) {
                const rad_hlu::Leaf& L = lu->leaves[b];
                if (L.r0 > nd.begin || L.r1 < nd.end || L.rank == 0) continue;
                RegPiece pc;
                pc.ld = L.r1 - L.r0;
                if (L.rank > 0) {
                    pc.lowrank = 1;
                    pc.off = L.uoff + (nd.begin - L.r0);
                    pc.k = L.rank;
                    pc.toff = t_of[b];
                    pc.c0 = L.c0;
                    pc.n = 0;
                } else {
                    pc.lowrank = 0;
                    pc.off = L.doff + (nd.begin - L.r0);
                    pc.c0 = L.c0;
                    pc.n = L.c1 - L.c0;
                    pc.k = 0;
                    pc.toff = 0;
                }
                pieces.push_back(pc);
            }
            sgm.p1 = (int)pieces.size();
            segs.push_back(sgm);
        }
        op.m = (int)segs.size() - op.r0;
        return op;
    };
    auto diag_leaf = [&](int q) -> long long {
        const NodeShape& nd = h->nodes[q];
        auto it = st.leaf_of.find(st.key(q, q));
        RAD_REQUIRE(it != st.leaf_of.end(), RAD_ECUDA, "diagonal leaf missing");
        (void)nd;
        return lu->leaves[it->second].doff;
    };
    std::function<void(int)> fwd = [&](int q) {
        const NodeShape& nd = h->nodes[q];
        if (nd.leaf) {
            lu->fwd.push_back(rad_hlu::Op{0, nd.begin, nd.end - nd.begin, diag_leaf(q), 0, 0});
            return;
        }
        fwd(nd.child0);
        lu->fwd.push_back(region(nd.child1, nd.child0));
        fwd(nd.child1);
    };
    std::function<void(int)> bwd = [&](int q) {
        const NodeShape& nd = h->nodes[q];
        if (nd.leaf) {
            lu->bwd.push_back(rad_hlu::Op{1, nd.begin, nd.end - nd.begin, diag_leaf(q), 0, 0});
            return;
        }
        bwd(nd.child1);
        lu->bwd.push_back(region(nd.child0, nd.child1));
        bwd(nd.child0);
    };
    for (int r : roots_of(h)) {
        fwd(r);
        bwd(r);
    }
    lu->sum_rank_t = std::max(1, toff);
    lu->d_lr.alloc(sizeof(RegLR) * std::max<size_t>(1, lr.size()), s);
    lu->d_segs.alloc(sizeof(RegRow) * std::max<size_t>(1, segs.size()), s);
    lu->d_pieces.alloc(sizeof(RegPiece) * std::max<size_t>(1, pieces.size()), s);
    if (!lr.empty()) RAD_CUDA(cudaMemcpyAsync(lu->d_lr.p, lr.data(), sizeof(RegLR) * lr.size(), cudaMemcpyHostToDevice, s));
    if (!segs.empty())
        RAD_CUDA(cudaMemcpyAsync(lu->d_segs.p, segs.data(), sizeof(RegRow) * segs.size(), cudaMemcpyHostToDevice, s));
    if (!pieces.empty())
        RAD_CUDA(cudaMemcpyAsync(lu->d_pieces.p, pieces.data(), sizeof(RegPiece) * pieces.size(),
                                 cudaMemcpyHostToDevice, s));
    RAD_CUDA(cudaStreamSynchronize(s));
    (void)ws;
}

template <class T>
void factor_t(rad_hlu* lu, const double* eps_dev, cudaStream_t s) {
    const rad_htree* h = lu->h;
    const int n = lu->n;
    set_smem_limits<T>();
    HluStructure st(h);
    Scratch ws(s);
    // eps in tree order
    double* eps_t = ws.get_n<double>(n);
    gather_user_to_tree(h, RAD_F64, eps_dev, n, 1, eps_t, 1, true, s);
    HluBuilder<T> B{lu, h, st, s, n};
    B.M = static_cast<T*>(ws.get(sizeof(T) * (size_t)n * n));
    RAD_CUDA(cudaMemsetAsync(B.M, 0, sizeof(T) * (size_t)n * n, s));
    // F~ from the stored operator (FP32 accurate factors when the fast ones are BF16)
    {
        HostScope hs_("host_hlu_expand");
        if (h->op_is_f64()) {
            expand_operator<T, double>(h, B.M, h->far_pool.p, ws, s);
        } else if (h->factor_dtype == RAD_F32 || h->far_pool_acc.p) {
            expand_operator<T, float>(h, B.M, h->accurate_far_pool(), ws, s);
        } else {
            expand_operator<T, __nv_bfloat16>(h, B.M, h->far_pool.p, ws, s);
        }
    }
    {
        ProfScope ps_("hlu_expand", s);
        hlu_reflection_kernel<T><<<grid_of((long long)n * n), 256, 0, s>>>(B.M, n, eps_t);
    }
    RAD_CHECK_LAUNCH();
    // truncation slots of the admissible leaves
    const size_t nb = h->blocks.size();
    B.slot_u.assign(nb, -1);
    B.slot_v.assign(nb, -1);
    B.kcap.assign(nb, 0);
    long long off = 0;
    for (size_t b = 0; b < nb; ++b) {
        const BlockH& bk = h->blocks[b];
        if (!bk.admissible || lu->tol <= 0.0) continue;
        const int m = bk.r1 - bk.r0, nn = bk.c1 - bk.c0;
        const int kc = std::max(1, std::min<int>(kHluMaxRank, (int)((long long)m * nn / (m + nn))));
        B.kcap[b] = kc;
        B.slot_u[b] = off;
        off += (long long)m * 2 * kc;
        B.slot_v[b] = off;
        off += (long long)nn * 2 * kc;
    }
    B.slots = static_cast<T*>(ws.get(sizeof(T) * (size_t)std::max<long long>(off, 16)));
    B.d_rank = ws.get_n<int>(std::max<size_t>(1, nb));
    B.d_err = ws.get_n<int>(1);
    RAD_CUDA(cudaMemsetAsync(B.d_rank, 0xff, sizeof(int) * std::max<size_t>(1, nb), s));   // -1: dense
    RAD_CUDA(cudaMemsetAsync(B.d_err, 0, sizeof(int), s));
    const std::vector<int> roots = roots_of(h);
    for (int r : roots) {
        B.plan_region(r, r);
        B.plan_node(r);
    }
    if (!B.tjobs.empty()) {
        B.d_tjobs = ws.get_n<TruncJob>(B.tjobs.size());
        RAD_CUDA(cudaMemcpyAsync(B.d_tjobs, B.tjobs.data(), sizeof(TruncJob) * B.tjobs.size(), cudaMemcpyHostToDevice, s));
    }
    // the admissible leaves of C, then the recursion
    {
        HostScope hs_("host_hlu_factor");
        for (int r : roots) B.truncate_region(r, r);
        for (int r : roots) B.factor(r);
    }
    // ranks and the zero-pivot flag
    std::vector<int> rk(std::max<size_t>(1, nb));
    int err = 0;
    RAD_CUDA(cudaMemcpyAsync(rk.data(), B.d_rank, sizeof(int) * rk.size(), cudaMemcpyDeviceToHost, s));
    RAD_CUDA(cudaMemcpyAsync(&err, B.d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    RAD_CUDA(cudaStreamSynchronize(s));
    RAD_REQUIRE(err == 0, RAD_EINVAL, "zero pivot in the block LU (the reflection matrix is not diagonally dominant)");
    // compact factor storage
    lu->leaves.resize(nb);
    long long dsz = 0, usz = 0;
    std::vector<CopyJob> dj, uj;
    for (size_t b = 0; b < nb; ++b) {
        const BlockH& bk = h->blocks[b];
        rad_hlu::Leaf& L = lu->leaves[b];
        L.r0 = bk.r0;
        L.r1 = bk.r1;
        L.c0 = bk.c0;
        L.c1 = bk.c1;
        L.adm = bk.admissible;
        const int m = bk.r1 - bk.r0, nn = bk.c1 - bk.c0;
        L.rank = B.slot_u[b] >= 0 ? rk[b] : -1;
        if (L.rank < 0) {
            L.doff = dsz;
            dj.push_back(CopyJob{bk.r0 + (long long)bk.c0 * n, dsz, m, nn, 0, 0});
            dsz += (long long)m * nn;
            lu->dense_entries += (long long)m * nn;
            if (bk.admissible && lu->tol > 0.0) ++lu->n_fallback;
        } else {
            L.uoff = usz;
            if (L.rank > 0) uj.push_back(CopyJob{B.slot_u[b], usz, m, L.rank, 1, 0});
            usz += (long long)m * L.rank;
            L.voff = usz;
            if (L.rank > 0) uj.push_back(CopyJob{B.slot_v[b], usz, nn, L.rank, 1, 0});
            usz += (long long)nn * L.rank;
            lu->lowrank_entries += (long long)L.rank * (m + nn);
            lu->max_rank = std::max(lu->max_rank, L.rank);
            ++lu->n_lowrank;
        }
    }
    lu->dpool.alloc(sizeof(T) * (size_t)std::max<long long>(dsz, 16), s);
    lu->upool.alloc(sizeof(T) * (size_t)std::max<long long>(usz, 16), s);
    for (int pass = 0; pass < 2; ++pass) {
        std::vector<CopyJob>& jv = pass == 0 ? dj : uj;
        if (jv.empty()) continue;
        CopyJob* d = ws.get_n<CopyJob>(jv.size());
        RAD_CUDA(cudaMemcpyAsync(d, jv.data(), sizeof(CopyJob) * jv.size(), cudaMemcpyHostToDevice, s));
        ProfScope ps_("hlu_extract", s);
        hlu_copy_kernel<T><<<(unsigned)jv.size(), 256, 0, s>>>(B.M, n, B.slots, d, pass == 0 ? lu->dpool.as<T>()
                                                                                              : lu->upool.as<T>());
        RAD_CHECK_LAUNCH();
    }
    RAD_CUDA(cudaStreamSynchronize(s));
    build_solve_schedule<T>(lu, st, ws, s);
}

// forward and backward substitution on tree-order row-major vectors (T)
template <class T>
void substitute_t(const rad_hlu* lu, T* X, int nc, T* tws, cudaStream_t s) {
    const T* dp = lu->dpool.as<T>();
    const T* up = lu->upool.as<T>();
    for (int pass = 0; pass < 2; ++pass) {
        const std::vector<rad_hlu::Op>& ops = pass == 0 ? lu->fwd : lu->bwd;
        for (const rad_hlu::Op& op : ops) {
            if (op.kind == 0 || op.kind == 1) {
                const int m = op.m;
                const unsigned grid = (unsigned)((nc + 7) / 8);
                ProfScope ps_("hlu_solve_leaf", s);
                if (op.kind == 0)
                    hlu_trsm_kernel<T, kLowerUnit><<<grid, 256, 0, s>>>(dp + op.doff, m, m, X + (long long)op.r0 * nc,
                                                                        nc, 1, nc);
                else
                    hlu_trsm_kernel<T, kUpper><<<grid, 256, 0, s>>>(dp + op.doff, m, m, X + (long long)op.r0 * nc, nc,
                                                                    1, nc);
                RAD_CHECK_LAUNCH();
            } else {
                if (op.lr1 > op.lr0) {
                    ProfScope ps_("hlu_solve_region", s);
                    hlu_region_vt_kernel<T><<<op.lr1 - op.lr0, 256, 0, s>>>(
                        lu->d_lr.as<RegLR>() + op.lr0, up, X, nc, tws);
                    RAD_CHECK_LAUNCH();
                }
                if (op.m > 0) {
                    ProfScope ps_("hlu_solve_region", s);
                    hlu_region_rows_kernel<T><<<op.m, 256, 0, s>>>(lu->d_segs.as<RegRow>() + op.r0,
                                                                   lu->d_pieces.as<RegPiece>(), dp, up, tws, X, nc);
                    RAD_CHECK_LAUNCH();
                }
            }
        }
    }
}

}  // namespace

// x = U^-1 L^-1 b on tree-order FP64 row-major vectors (n x nc), in place.
void hlu_apply_tree(const rad_hlu* lu, double* X, int nc, cudaStream_t s) {
    Scratch ws(s);
    const long long cnt = (long long)lu->n * nc;
    if (lu->f64) {
        double* tws = ws.get_n<double>((size_t)lu->sum_rank_t * nc);
        substitute_t<double>(lu, X, nc, tws, s);
        return;
    }
    float* X32 = ws.get_n<float>(cnt);
    float* tws = ws.get_n<float>((size_t)lu->sum_rank_t * nc);
    { ProfScope ps_("hlu_convert", s); hlu_cast_kernel<float><<<grid_of(cnt), 256, 0, s>>>(X, X32, cnt); }
    RAD_CHECK_LAUNCH();
    substitute_t<float>(lu, X32, nc, tws, s);
    { ProfScope ps_("hlu_convert", s); hlu_uncast_kernel<float><<<grid_of(cnt), 256, 0, s>>>(X32, X, cnt); }
    RAD_CHECK_LAUNCH();
}

const rad_htree* hlu_handle(const rad_hlu* lu) { return lu->h; }

}  // namespace rad

using namespace rad;

extern "C" {

int rad_hlu_factor(const rad_htree* h, const double* eps, const rad_hlu_params* p, void* stream, rad_hlu** out) {
    NvtxRange nv_(__func__);
    try {
        RAD_REQUIRE(h != nullptr && eps != nullptr && p != nullptr && out != nullptr, RAD_EINVAL, "null argument");
        *out = nullptr;
        RAD_REQUIRE(h->compressed, RAD_EINVAL, "handle is not compressed (call rad_compress_aca)");
        RAD_REQUIRE(!h->from_dense, RAD_EINVAL, "the H-LU needs a block tree (not a single dense block)");
        RAD_REQUIRE(std::isfinite(p->tol) && p->tol >= 0.0 && p->tol < 1.0, RAD_EINVAL, "tol must be in [0, 1)");
        RAD_REQUIRE(h->n <= 46340, RAD_ELIMIT, "the H-LU works on a dense n x n matrix: n must be <= 46340");
        for (const NodeShape& nd : h->nodes)
            RAD_REQUIRE(!nd.leaf || nd.end - nd.begin <= kHluMaxLeaf, RAD_ELIMIT, "leaf clusters above 128 facets");
        AllocScope as(h->alloc);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        auto lu = std::make_unique<rad_hlu>();
        lu->h = h;
        lu->n = (int)h->n;
        lu->f64 = h->op_is_f64();
        lu->tol = p->tol;
        RAD_CUDA(cudaGetDevice(&lu->device));
        Scratch ws(s);
        const double* epsd = to_device_t(eps, (size_t)h->n, ws);
        {
            // the emissivities define C: reject what the solves reject
            std::vector<double> he(h->n);
            RAD_CUDA(cudaMemcpyAsync(he.data(), epsd, sizeof(double) * h->n, cudaMemcpyDeviceToHost, s));
            RAD_CUDA(cudaStreamSynchronize(s));
            for (double e : he) RAD_REQUIRE(std::isfinite(e) && e > 0.0 && e <= 1.0, RAD_EINVAL,
                                            "every emissivity must be finite and in (0, 1]");
        }
        const auto t0 = std::chrono::steady_clock::now();
        if (lu->f64) factor_t<double>(lu.get(), epsd, s);
        else factor_t<float>(lu.get(), epsd, s);
        lu->factor_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        check_bounds_after_call();
        *out = lu.release();
        return RAD_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.code;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return RAD_ECUDA;
    }
}

int rad_hlu_solve(const rad_hlu* lu, const double* B, int64_t ldB, int64_t nrhs, double* X, int64_t ldX,
                  void* stream) {
    NvtxRange nv_(__func__);
    try {
        RAD_REQUIRE(lu != nullptr && B != nullptr && X != nullptr, RAD_EINVAL, "null argument");
        RAD_REQUIRE(nrhs >= 1 && nrhs <= 4096, RAD_EINVAL, "nrhs must be in [1, 4096]");
        RAD_REQUIRE(ldB >= lu->n && ldX >= lu->n, RAD_EINVAL, "leading dimension smaller than n");
        const rad_htree* h = lu->h;
        AllocScope as(h->alloc);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const int n = lu->n, nr = (int)nrhs;
        Scratch ws(s);
        const bool bdev = is_device_ptr(B), xdev = is_device_ptr(X);
        const double* Bd = B;
        int64_t ldb = ldB;
        if (!bdev) {
            double* d = ws.get_n<double>((size_t)n * nr);
            RAD_CUDA(cudaMemcpy2DAsync(d, 8 * (size_t)n, B, 8 * ldB, 8 * (size_t)n, nr, cudaMemcpyHostToDevice, s));
            Bd = d;
            ldb = n;
        }
        double* Xt = ws.get_n<double>((size_t)n * nr);
        gather_user_to_tree(h, RAD_F64, Bd, ldb, nr, Xt, nr, true, s);
        hlu_apply_tree(lu, Xt, nr, s);
        double* Xd = xdev ? X : ws.get_n<double>((size_t)n * nr);
        scatter_tree_to_user(h, Xt, nr, nr, true, RAD_F64, Xd, xdev ? ldX : n, s);
        if (!xdev) {
            RAD_CUDA(cudaMemcpy2DAsync(X, 8 * ldX, Xd, 8 * (size_t)n, 8 * (size_t)n, nr, cudaMemcpyDeviceToHost, s));
        }
        RAD_CUDA(cudaStreamSynchronize(s));
        check_bounds_after_call();
        return RAD_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.code;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return RAD_ECUDA;
    }
}

int rad_hlu_get_stats(const rad_hlu* lu, rad_hlu_stats* st) {
    if (!lu || !st) {
        set_last_error("null argument");
        return RAD_EINVAL;
    }
    std::memset(st, 0, sizeof(*st));
    st->n = lu->n;
    st->dense_entries = lu->dense_entries;
    st->lowrank_entries = lu->lowrank_entries;
    st->max_rank = lu->max_rank;
    st->n_lowrank = lu->n_lowrank;
    st->n_dense_fallback = lu->n_fallback;
    st->precision = lu->f64 ? RAD_F64 : RAD_F32;
    st->tol = lu->tol;
    st->factor_ms = lu->factor_ms;
    st->solve_launches = (int32_t)(lu->fwd.size() + lu->bwd.size());
    return RAD_OK;
}

int rad_hlu_export(const rad_hlu* lu, double* LU) {
    NvtxRange nv_(__func__);
    try {
        RAD_REQUIRE(lu != nullptr && LU != nullptr, RAD_EINVAL, "null argument");
        const int n = lu->n;
        const int sz = lu->f64 ? 8 : 4;
        std::vector<unsigned char> dp(lu->dpool.bytes), up(lu->upool.bytes);
        RAD_CUDA(cudaMemcpy(dp.data(), lu->dpool.p, dp.size(), cudaMemcpyDeviceToHost));
        RAD_CUDA(cudaMemcpy(up.data(), lu->upool.p, up.size(), cudaMemcpyDeviceToHost));
        auto get = [&](const std::vector<unsigned char>& v, long long i) -> double {
            if (sz == 8) {
                double d;
                std::memcpy(&d, v.data() + 8 * i, 8);
                return d;
            }
            float f;
            std::memcpy(&f, v.data() + 4 * i, 4);
            return f;
        };
        std::memset(LU, 0, sizeof(double) * (size_t)n * n);
        for (const rad_hlu::Leaf& L : lu->leaves) {
            const int m = L.r1 - L.r0, nn = L.c1 - L.c0;
            for (int i = 0; i < m; ++i)
                for (int j = 0; j < nn; ++j) {
                    double v = 0.0;
                    if (L.rank < 0) {
                        v = get(dp, L.doff + i + (long long)j * m);
                    } else {
                        for (int l = 0; l < L.rank; ++l)
                            v += get(up, L.uoff + i + (long long)l * m) * get(up, L.voff + j + (long long)l * nn);
                    }
                    LU[(size_t)(L.r0 + i) * n + (L.c0 + j)] = v;
                }
        }
        return RAD_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.code;
    }
}

int rad_hlu_free(rad_hlu* lu) {
    delete lu;
    return RAD_OK;
}

}  // extern "C"
