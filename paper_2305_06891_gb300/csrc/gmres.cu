// A7-A8: batched restarted GMRES on the reflection system of Eq. (11),
//   C y = b,  C = I - diag(1 - eps) F,
// for the m + 1 right-hand sides b_c = eps o eta_c (c < m) and b_m = eps,
// followed by the facet flux of Eq. (12):
//   q_c = sigma eps o ( F y_c - eta_c o F z ),  z = y_m.
//
// All vectors are FP64, in tree order, row-major N x (m+1) so that one block
// matrix product serves every column at once.  Each Arnoldi step is one
// product with the reflection epilogue fused in, two classical Gram-Schmidt
// passes (CGS2) with FP64 inner products reduced in a fixed order, a norm, a
// normalisation (which also writes the FP32 copy the FP32 operator reads)
// and a Givens update done on the device per column.  Only the per-column
// residual estimates cross to the host each step.  A column stops when its
// estimate reaches tol; every restart recomputes the true residual
// b - C y with the stored operator.

#include <algorithm>
#include <cmath>

#include "rad_device.cuh"

namespace rad {

namespace {

constexpr int kChunkRows = 64;        // rows per inner-product chunk of wide blocks
constexpr int kChunkElems = 8192;     // elements per chunk for narrow blocks
constexpr int kNarrowCols = 128;      // flattened inner products up to this many columns

__global__ void rhs_kernel(int n, int m, const double* __restrict__ eps, const double* __restrict__ T, long long ldT,
                           const int* __restrict__ perm, double* __restrict__ eps_t, double* __restrict__ B) {
    const int nc = m + 1;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * nc) return;
    const int p = (int)(e / nc), c = (int)(e - (long long)p * nc);
    const int u = perm[p];
    const double ep = eps[u];
    if (c < m) {
        const double t = T[u + (long long)c * ldT];
        B[e] = ep * ((t * t) * (t * t));
    } else {
        B[e] = ep;
        eps_t[p] = ep;
    }
}

// partial[(l * nc + c) * nchunks + chunk] = sum over the chunk's rows of
// A_l[i][c] * Bv[i][c],  A_l = A + l * strideA.  The chunk's rows are one
// contiguous range of row-major elements; thread t (< per * nc, per =
// blockDim / nc) reads elements t, t + per*nc, ... (all of column t % nc),
// four A_l at a time, and the per threads of a column are summed in a
// fixed order through shared memory.
__global__ void __launch_bounds__(256)
mdot_kernel(const double* __restrict__ A, long long strideA, int L, const double* __restrict__ Bv,
            const int2* __restrict__ chunk, int nc, double* __restrict__ partial) {
    __shared__ double red[4][256];
    const int per = blockDim.x / nc, T = per * nc;
    const int t = threadIdx.x;
    const long long e0 = (long long)chunk[blockIdx.x].x * nc, e1 = (long long)chunk[blockIdx.x].y * nc;
    for (int l0 = 0; l0 < L; l0 += 4) {
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        if (t < T) {
            for (long long e = e0 + t; e < e1; e += T) {
                const double bv = Bv[e];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (l0 + q < L) acc[q] += A[(l0 + q) * strideA + e] * bv;
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) red[q][t] = acc[q];
        __syncthreads();
        for (int o = t; o < 4 * nc; o += blockDim.x) {
            const int q = o / nc, c = o - q * nc;
            if (l0 + q < L) {
                double sum = 0.0;
                for (int k = 0; k < per; ++k) sum += red[q][k * nc + c];
                partial[((long long)(l0 + q) * nc + c) * gridDim.x + blockIdx.x] = sum;
            }
        }
        __syncthreads();
    }
}

// Same sums for wide blocks (nc > 128): a warp takes 32 consecutive columns
// (grid y = column slab), the eight warps of a CTA take rows ty, ty + 8, ...
__global__ void __launch_bounds__(256)
mdot_wide_kernel(const double* __restrict__ A, long long strideA, int L, const double* __restrict__ Bv,
            const int2* __restrict__ chunk, int nc, double* __restrict__ partial) {
    __shared__ double red[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int c = blockIdx.y * 32 + tx;
    const int r0 = chunk[blockIdx.x].x;
    const int r1 = chunk[blockIdx.x].y;
    for (int l0 = 0; l0 < L; l0 += 4) {
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        if (c < nc) {
            for (int i = r0 + ty; i < r1; i += 8) {
                const double bv = Bv[(long long)i * nc + c];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (l0 + q < L) acc[q] += A[(l0 + q) * strideA + (long long)i * nc + c] * bv;
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            red[ty][tx] = acc[q];
            __syncthreads();
            if (ty == 0 && l0 + q < L && c < nc) {
                double s = 0.0;
                for (int w = 0; w < 8; ++w) s += red[w][tx];
                partial[((long long)(l0 + q) * nc + c) * gridDim.x + blockIdx.x] = s;
            }
            __syncthreads();
        }
    }
}

// Virtual columns: a batch handle holds several cavities (segments of the
// rows); every (segment, column) pair is its own Krylov problem, with index
// vc = segment * nc + c.  seg == nullptr means one segment.
// row and column of element e of a row-major block with nc columns (32-bit
// division while e fits, the FP64-free fast path of every vector kernel)
__device__ __forceinline__ void row_col(long long e, int nc, long long& row, int& c) {
    if (e <= 0xffffffffll) {
        const unsigned r = (unsigned)e / (unsigned)nc;
        row = r;
        c = (int)((unsigned)e - r * (unsigned)nc);
    } else {
        row = e / nc;
        c = (int)(e - row * nc);
    }
}
__device__ __forceinline__ int vcol(const int* seg, long long e, int nc) {
    long long row;
    int c;
    row_col(e, nc, row, c);
    return seg ? seg[row] * nc + c : c;
}

// rs[vc] = 1 / sqrt(ss[vc]) for active columns with ss > 0, else 0 (the
// scale of a normalisation, computed once per column)
__global__ void col_scale_kernel(int nvc, const double* __restrict__ ss, const int* __restrict__ active,
                                 double* __restrict__ rs) {
    const int vc = blockIdx.x * blockDim.x + threadIdx.x;
    if (vc >= nvc) return;
    rs[vc] = (active[vc] && ss[vc] > 0.0) ? 1.0 / sqrt(ss[vc]) : 0.0;
}

// out[l * nvc + vc] = sum over the chunks of vc's segment of
// partial[l][c][chunk]: one 128-thread CTA per output; thread t adds chunks
// k0 + t, k0 + t + 128, ... in order, then a fixed butterfly per warp and
// the four warp sums in order (the same summation order on every call).
// Chunks never straddle segments.
__global__ void __launch_bounds__(128)
reduce_chunks_kernel(const double* __restrict__ partial, const int* __restrict__ seg_chunk0, int L, int nc,
                     int nvc, int nchunks, double* out) {
    __shared__ double wsum[4];
    const int e = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int l = e / nvc, vc = e - l * nvc;
    const int sg = vc / nc, c = vc - sg * nc;
    const int k0 = seg_chunk0[sg], k1 = seg_chunk0[sg + 1];
    const double* pc = partial + ((long long)l * nc + c) * nchunks;
    double s = 0.0;
    for (int k = k0 + (int)threadIdx.x; k < k1; k += 128) s += pc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) wsum[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) out[e] = (wsum[0] + wsum[1]) + (wsum[2] + wsum[3]);
}

__global__ void add_kernel(double* __restrict__ a, const double* __restrict__ b, long long cnt) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < cnt) a[e] += b[e];
}

// W[i][c] -= sum_{l<L} V_l[i][c] h[l][c]   for active columns
__global__ void cgs_update_kernel(const double* __restrict__ V, long long strideV, int L, const double* __restrict__ h,
                                  const int* __restrict__ active, double* __restrict__ W, int n, int nc,
                                  const int* __restrict__ seg, int nvc) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * nc) return;
    const int c = vcol(seg, e, nc);
    if (!active[c]) return;
    double w = W[e];
    for (int l = 0; l < L; ++l) w -= V[l * strideV + e] * h[l * nvc + c];
    W[e] = w;
}

// Vn = W * rs (rs from col_scale_kernel: 1 / ||W|| per active column, else
// 0); optional FP32 copy with rows padded to ldp.  Also starts a cycle
// (W = residual, rs = 1 / beta).
__global__ void normalize_kernel(const double* __restrict__ W, const double* __restrict__ rs,
                                 double* __restrict__ Vn, float* __restrict__ X32, int n, int nc,
                                 const int* __restrict__ seg, int ldp) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * nc) return;
    long long row;
    int c;
    row_col(e, nc, row, c);
    const double v = W[e] * rs[seg ? seg[row] * nc + c : c];
    Vn[e] = v;
    if (X32) X32[row * ldp + c] = (float)v;
}

// FP32 copy of an n x nc row-major FP64 block, rows padded to ldp columns
// (so that the product can move them as 16-byte quads).
__global__ void to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, long long cnt, int nc, int ldp) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cnt) return;
    long long row;
    int c;
    row_col(e, nc, row, c);
    b[row * ldp + c] = (float)a[e];
}

// Per column: apply the previous Givens rotations to the new Hessenberg
// column, form the next rotation, update g and the residual estimate.
// Hm layout: Hm[(j * (R + 1) + l) * nc + c] = H(l, j).
__global__ void givens_kernel(int j, int R, int nc, double* __restrict__ Hm, const double* __restrict__ hn2,
                              double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g,
                              const double* __restrict__ bnorm, double* __restrict__ resid, int* __restrict__ active,
                              int* __restrict__ jc, double tol) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc || !active[c]) return;
    double* hcol = Hm + (long long)j * (R + 1) * nc;
    for (int i = 0; i < j; ++i) {
        const double a = hcol[i * nc + c], b = hcol[(i + 1) * nc + c];
        const double C = cs[i * nc + c], S = sn[i * nc + c];
        hcol[i * nc + c] = C * a + S * b;
        hcol[(i + 1) * nc + c] = -S * a + C * b;
    }
    const double a = hcol[j * nc + c];
    const double b = sqrt(hn2[c]);
    const double r = hypot(a, b);
    double C = 1.0, S = 0.0;
    if (r > 0.0) {
        C = a / r;
        S = b / r;
    }
    cs[j * nc + c] = C;
    sn[j * nc + c] = S;
    hcol[j * nc + c] = r;
    const double gj = g[j * nc + c];
    g[(j + 1) * nc + c] = -S * gj;
    g[j * nc + c] = C * gj;
    const double res = fabs(g[(j + 1) * nc + c]) / bnorm[c];
    resid[c] = res;
    jc[c] = j + 1;
    if (!(res > tol) || !(b > 0.0)) active[c] = 0;
}

// y = R^-1 g per column (R upper triangular, jc[c] x jc[c]).
__global__ void trisolve_kernel(int R, int nc, const double* __restrict__ Hm, const double* __restrict__ g,
                                const int* __restrict__ jc, double* __restrict__ ycoef) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const int J = jc[c];
    for (int i = J - 1; i >= 0; --i) {
        double s = g[i * nc + c];
        for (int k = i + 1; k < J; ++k) s -= Hm[((long long)k * (R + 1) + i) * nc + c] * ycoef[k * nc + c];
        const double d = Hm[((long long)i * (R + 1) + i) * nc + c];
        ycoef[i * nc + c] = d != 0.0 ? s / d : 0.0;
    }
}

// X[i][c] += sum_{l < jc[c]} V_l[i][c] y[l][c]
__global__ void update_x_kernel(const double* __restrict__ V, long long strideV, int Lmax,
                                const double* __restrict__ ycoef, const int* __restrict__ jc, double* __restrict__ X,
                                int n, int nc, const int* __restrict__ seg, int nvc) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * nc) return;
    const int c = vcol(seg, e, nc);
    const int J = min(jc[c], Lmax);
    double x = X[e];
    for (int l = 0; l < J; ++l) x += V[l * strideV + e] * ycoef[l * nvc + c];
    X[e] = x;
}

__global__ void init_g_kernel(int R, int nc, const double* __restrict__ beta2, double* __restrict__ g,
                              int* __restrict__ jc) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    for (int l = 0; l <= R; ++l) g[l * nc + c] = 0.0;
    g[c] = sqrt(beta2[c]);
    jc[c] = 0;
}

template <class FT>
__global__ void flux_kernel(int n, int m, const FT* __restrict__ FY, const int* __restrict__ perm,
                            const double* __restrict__ eps, const double* __restrict__ T, long long ldT, double sigma,
                            double* __restrict__ q, long long ldq) {
    const int nc = m + 1;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * m) return;
    const int p = (int)(e / m), c = (int)(e - (long long)p * m);
    const int u = perm[p];
    const double t = T[u + (long long)c * ldT];
    const double eta = (t * t) * (t * t);
    q[u + (long long)c * ldq] =
        sigma * eps[u] * ((double)FY[(long long)p * nc + c] - eta * (double)FY[(long long)p * nc + m]);
}

// Inputs of a solve, checked before any solver launch: every emissivity
// finite and in (0, 1] (bit 1 of *flags), every value of the n x cols
// column-major array X finite (and >= 0 when nonneg: temperatures) (bit 2).
__global__ void check_inputs_kernel(int n, const double* __restrict__ eps, const double* __restrict__ X,
                                    long long ldX, int cols, int nonneg, int* __restrict__ flags) {
    int bad = 0;
    const long long total = (long long)n * (cols + 1);
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % n);
        const long long c = e / n;
        if (c == 0) {
            const double v = eps[i];
            if (!(isfinite(v) && v > 0.0 && v <= 1.0)) bad |= 1;
        } else {
            const double v = X[(c - 1) * ldX + i];
            if (!isfinite(v) || (nonneg && v < 0.0)) bad |= 2;
        }
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (bad && (threadIdx.x & 31) == 0) atomicOr(flags, bad);
}

__global__ void axpy_kernel(double* __restrict__ X, const double* __restrict__ D, long long cnt) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < cnt) X[e] += D[e];
}

inline unsigned grid_for(long long cnt, int bs = 256) { return (unsigned)((cnt + bs - 1) / bs); }

// Inner products per virtual column (segment, column) over chunks of rows
// that never straddle a segment (for blocks of up to 128 columns about
// eight chunks per SM of 1,024 to 8,192 elements each; 64 rows for wider
// blocks).
struct ColReducer {
    int n, nc, nseg, nvc, nchunks;
    const int2* chunk;       // [r0, r1) per chunk
    const int* seg_chunk0;   // first chunk of each segment, nseg + 1 entries
    double* partial;
    cudaStream_t s;
    ColReducer(const rad_htree* h, int nc_, int Lmax, Scratch& ws, cudaStream_t st) : n((int)h->n), nc(nc_), s(st) {
        const std::vector<int64_t> one{0, h->n};
        const std::vector<int64_t>& sg = h->seg.size() >= 2 ? h->seg : one;
        nseg = (int)sg.size() - 1;
        nvc = nseg * nc;
        std::vector<int2> ch;
        std::vector<int> c0(nseg + 1);
        // narrow blocks: about eight chunks per SM, 1,024 to 8,192 elements each
        const int64_t chunk_elems = std::min<int64_t>(kChunkElems, std::max<int64_t>(1024, (int64_t)n * nc / 1216));
        for (int g = 0; g < nseg; ++g) {
            c0[g] = (int)ch.size();
            const int64_t rows = nc <= kNarrowCols ? std::max<int64_t>(1, chunk_elems / nc) : kChunkRows;
            for (int64_t r = sg[g]; r < sg[g + 1]; r += rows)
                ch.push_back(make_int2((int)r, (int)std::min<int64_t>(r + rows, sg[g + 1])));
        }
        c0[nseg] = (int)ch.size();
        nchunks = (int)ch.size();
        int2* dch = ws.get_n<int2>(ch.size());
        int* dc0 = ws.get_n<int>(c0.size());
        h2d(dch, ch, s);
        h2d(dc0, c0, s);
        chunk = dch;
        seg_chunk0 = dc0;
        partial = ws.get_n<double>((long long)nchunks * Lmax * nc);
    }
    // out[l][vc] = sum over vc's rows of A_l[i][c] Bv[i][c]
    void dots(const double* A, long long strideA, int L, const double* Bv, double* out) {
        if (nc <= kNarrowCols) {
            ProfScope ps_("gmres_dots", s);
            mdot_kernel<<<nchunks, 256, 0, s>>>(A, strideA, L, Bv, chunk, nc, partial);
        } else {
            ProfScope ps_("gmres_dots", s);
            mdot_wide_kernel<<<dim3(nchunks, (nc + 31) / 32), 256, 0, s>>>(A, strideA, L, Bv, chunk, nc, partial);
        }
        RAD_CHECK_LAUNCH();
        { ProfScope ps_("gmres_dots", s); reduce_chunks_kernel<<<(unsigned)(L * nvc), 128, 0, s>>>(partial, seg_chunk0, L, nc, nvc,
                                                                          nchunks, out); }
        RAD_CHECK_LAUNCH();
    }
};

// Runs check_inputs_kernel and fails with RAD_EINVAL naming what is wrong.
static void check_solve_inputs(int n, const double* eps, const double* X, long long ldX, int cols, bool temps,
                               Scratch& ws, cudaStream_t s) {
    int* d_flags = ws.get_n<int>(1);
    RAD_CUDA(cudaMemsetAsync(d_flags, 0, sizeof(int), s));
    const long long total = (long long)n * (cols + 1);
    const unsigned grid = (unsigned)std::min<long long>(1216, (total + 255) / 256);
    { ProfScope ps_("check_inputs", s); check_inputs_kernel<<<grid, 256, 0, s>>>(n, eps, X, ldX, cols, temps ? 1 : 0, d_flags); }
    RAD_CHECK_LAUNCH();
    int flags = 0;
    RAD_CUDA(cudaMemcpyAsync(&flags, d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    RAD_CUDA(cudaStreamSynchronize(s));
    RAD_REQUIRE(!(flags & 1), RAD_EINVAL, "every emissivity must be finite and in (0, 1]");
    RAD_REQUIRE(!(flags & 2), RAD_EINVAL,
                temps ? "every temperature must be finite and >= 0" : "every right-hand side value must be finite");
}

}  // namespace

// GMRES on C X = B in tree order (row-major N x nc).  X receives the solution.
// Each virtual column (segment of a batch, column) runs its own restarted
// GMRES: own Krylov vectors (the column's rows in that segment), Hessenberg
// matrix, rotations and stopping test; they share the operator products.
static void gmres_tree(const rad_htree* h, const double* eps_t, const double* B, int nc, const rad_solve_params* p,
                       double* X, rad_solve_info* info, Scratch& ws, cudaStream_t s) {
    const int n = (int)h->n;
    const int R = p->restart;
    const double tol = p->tol;
    const bool op64 = h->op_is_f64();
    const long long nv = (long long)n * nc;
    ColReducer red(h, nc, R + 1, ws, s);
    const int nvc = red.nvc;
    const int* seg = red.nseg > 1 ? h->d_segrow.as<int>() : nullptr;
    double* W = ws.get_n<double>(nv);
    double* V = ws.get_n<double>(nv * (R + 1));
    // row stride of the FP32 copy: the product's vector layout (1 for one
    // column, else padded to a multiple of 4 for 16-byte rows)
    const int ldp = tree_ld(nc);
    float* X32 = op64 ? nullptr : ws.get_n<float>((long long)n * ldp);
    void* Tws = ws.get(apply_workspace_bytes(h, nc));
    double* Hm = ws.get_n<double>((long long)R * (R + 1) * nvc);
    double* cs = ws.get_n<double>((long long)R * nvc);
    double* sn = ws.get_n<double>((long long)R * nvc);
    double* g = ws.get_n<double>((long long)(R + 1) * nvc);
    double* ycoef = ws.get_n<double>((long long)(R + 1) * nvc);
    double* bnorm2 = ws.get_n<double>(nvc);
    double* bnorm = ws.get_n<double>(nvc);
    double* beta2 = ws.get_n<double>(nvc);
    double* hn2 = ws.get_n<double>(nvc);
    double* rscale = ws.get_n<double>(nvc);
    double* resid = ws.get_n<double>(nvc);
    int* active = ws.get_n<int>(nvc);
    int* jc = ws.get_n<int>(nvc);

    RAD_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * nv, s));
    red.dots(B, 0, 1, B, bnorm2);
    std::vector<double> hb2(nvc), hbeta(nvc);
    RAD_CUDA(cudaMemcpyAsync(hb2.data(), bnorm2, sizeof(double) * nvc, cudaMemcpyDeviceToHost, s));
    RAD_CUDA(cudaStreamSynchronize(s));
    std::vector<double> hbn(nvc);
    for (int c = 0; c < nvc; ++c) hbn[c] = hb2[c] > 0.0 ? std::sqrt(hb2[c]) : 1.0;
    RAD_CUDA(cudaMemcpyAsync(bnorm, hbn.data(), sizeof(double) * nvc, cudaMemcpyHostToDevice, s));
    // initial residual = B (x0 = 0)
    RAD_CUDA(cudaMemcpyAsync(W, B, sizeof(double) * nv, cudaMemcpyDeviceToDevice, s));
    RAD_CUDA(cudaMemcpyAsync(beta2, bnorm2, sizeof(double) * nvc, cudaMemcpyDeviceToDevice, s));
    hbeta = hb2;

    auto apply_C = [&](const double* vin, const float* vin32, double* out, int mode) {
        Epi epi{mode, eps_t, vin, mode == kResid ? B : nullptr, nc};
        apply_tree(h, op64 ? (const void*)vin : (const void*)vin32, op64 ? nc : ldp, out, nc, nc, epi, Tws, s);
    };
    // right preconditioning with the block LU factors: the Krylov space is
    // built on C (LU)^-1 and the update is x += (LU)^-1 V y
    const rad_hlu* pre = p->precond;
    double* Zp = pre ? ws.get_n<double>(nv) : nullptr;
    auto precondition = [&](const double* vin, double* out) {
        RAD_CUDA(cudaMemcpyAsync(out, vin, sizeof(double) * nv, cudaMemcpyDeviceToDevice, s));
        hlu_apply_tree(pre, out, nc, s);
        if (X32) {
            { ProfScope ps_("gmres_convert", s); to_f32_kernel<<<grid_for(nv), 256, 0, s>>>(out, X32, nv, nc, ldp); }
            RAD_CHECK_LAUNCH();
        }
    };

    int total_iters = 0, restarts = 0, matvecs = 0, status = RAD_OK;
    double prev_max = INFINITY, max_rel = 0.0;
    std::vector<int> hact(nvc);
    for (;;) {
        // virtual columns still above tolerance take part in this cycle
        max_rel = 0.0;
        int n_act = 0;
        for (int c = 0; c < nvc; ++c) {
            const double rel = std::sqrt(std::max(hbeta[c], 0.0)) / hbn[c];
            max_rel = std::max(max_rel, rel);
            hact[c] = rel > tol ? 1 : 0;
            n_act += hact[c];
        }
        if (n_act == 0) break;
        if (total_iters >= p->max_iter || !(max_rel < 0.9 * prev_max)) {
            status = RAD_ENOTCONV;
            break;
        }
        prev_max = max_rel;
        RAD_CUDA(cudaMemcpyAsync(active, hact.data(), sizeof(int) * nvc, cudaMemcpyHostToDevice, s));
        // start a cycle: V_0 = R / beta for active columns, g = beta e_1
        { ProfScope ps_("gmres_small", s); col_scale_kernel<<<grid_for(nvc, 128), 128, 0, s>>>(nvc, beta2, active, rscale); }
        RAD_CHECK_LAUNCH();
        { ProfScope ps_("gmres_small", s); normalize_kernel<<<grid_for(nv), 256, 0, s>>>(W, rscale, V, X32, n, nc, seg, ldp); }
        RAD_CHECK_LAUNCH();
        { ProfScope ps_("gmres_small", s); init_g_kernel<<<grid_for(nvc, 128), 128, 0, s>>>(R, nvc, beta2, g, jc); }
        RAD_CHECK_LAUNCH();
        for (int j = 0; j < R && total_iters < p->max_iter; ++j) {
            double* Vj = V + (long long)j * nv;
            double* hcol = Hm + (long long)j * (R + 1) * nvc;
            // w = C v_j  (C (LU)^-1 v_j when preconditioned)
            if (pre) {
                precondition(Vj, Zp);
                apply_C(Zp, X32, W, kReflect);
            } else {
                apply_C(Vj, X32, W, kReflect);
            }
            ++matvecs;
            // CGS2: h = V^T w; w -= V h; h2 = V^T w; w -= V h2; h += h2
            for (int pass = 0; pass < 2; ++pass) {
                double* hbuf = pass == 0 ? hcol : ycoef;  // ycoef doubles as scratch here
                red.dots(V, nv, j + 1, W, hbuf);
                { ProfScope ps_("gmres_cgs_update", s); cgs_update_kernel<<<grid_for(nv), 256, 0, s>>>(V, nv, j + 1, hbuf, active, W, n, nc, seg, nvc); }
                RAD_CHECK_LAUNCH();
                if (pass == 1) {
                    { ProfScope ps_("gmres_small", s); add_kernel<<<grid_for((long long)(j + 1) * nvc), 256, 0, s>>>(hcol, ycoef, (long long)(j + 1) * nvc); }
                    RAD_CHECK_LAUNCH();
                }
            }
            red.dots(W, 0, 1, W, hn2);
            { ProfScope ps_("gmres_normalize", s); col_scale_kernel<<<grid_for(nvc, 128), 128, 0, s>>>(nvc, hn2, active, rscale); }
            RAD_CHECK_LAUNCH();
            { ProfScope ps_("gmres_normalize", s); normalize_kernel<<<grid_for(nv), 256, 0, s>>>(W, rscale, V + (long long)(j + 1) * nv, X32, n, nc, seg, ldp); }
            RAD_CHECK_LAUNCH();
            { ProfScope ps_("gmres_small", s); givens_kernel<<<grid_for(nvc, 128), 128, 0, s>>>(j, R, nvc, Hm, hn2, cs, sn, g, bnorm, resid, active, jc,
                                                            tol); }
            RAD_CHECK_LAUNCH();
            ++total_iters;
            RAD_CUDA(cudaMemcpyAsync(hact.data(), active, sizeof(int) * nvc, cudaMemcpyDeviceToHost, s));
            RAD_CUDA(cudaStreamSynchronize(s));
            int still = 0;
            for (int c = 0; c < nvc; ++c) still += hact[c];
            if (still == 0) break;
        }
        // x += V y
        { ProfScope ps_("gmres_small", s); trisolve_kernel<<<grid_for(nvc, 128), 128, 0, s>>>(R, nvc, Hm, g, jc, ycoef); }
        RAD_CHECK_LAUNCH();
        if (pre) {
            // x += (LU)^-1 (V y)
            RAD_CUDA(cudaMemsetAsync(W, 0, sizeof(double) * nv, s));
            { ProfScope ps_("gmres_update_x", s); update_x_kernel<<<grid_for(nv), 256, 0, s>>>(V, nv, R, ycoef, jc, W, n, nc, seg, nvc); }
            RAD_CHECK_LAUNCH();
            hlu_apply_tree(pre, W, nc, s);
            { ProfScope ps_("gmres_update_x", s); axpy_kernel<<<grid_for(nv), 256, 0, s>>>(X, W, nv); }
            RAD_CHECK_LAUNCH();
        } else {
            { ProfScope ps_("gmres_update_x", s); update_x_kernel<<<grid_for(nv), 256, 0, s>>>(V, nv, R, ycoef, jc, X, n, nc, seg, nvc); }
            RAD_CHECK_LAUNCH();
        }
        // true residual r = b - C x
        if (X32) {
            { ProfScope ps_("gmres_convert", s); to_f32_kernel<<<grid_for(nv), 256, 0, s>>>(X, X32, nv, nc, ldp); }
            RAD_CHECK_LAUNCH();
        }
        apply_C(X, X32, W, kResid);
        ++matvecs;
        red.dots(W, 0, 1, W, beta2);
        RAD_CUDA(cudaMemcpyAsync(hbeta.data(), beta2, sizeof(double) * nvc, cudaMemcpyDeviceToHost, s));
        RAD_CUDA(cudaStreamSynchronize(s));
        ++restarts;
    }
    if (info) {
        info->status = status;
        info->iters = total_iters;
        info->restarts = restarts;
        info->matvecs = matvecs;
        info->max_rel_residual = max_rel;
    }
}

// Mixed-precision iterative refinement: r = b - C y with the accurate
// operator (FP32 storage, FP64 accumulation), correction C d = r by GMRES on
// the fast operator to inner_tol, y += d; stops when every column's
// accurate relative residual is <= tol.
static void refine_tree(const rad_htree* h, const double* eps_t, const double* B, int nc, const rad_solve_params* p,
                        double* X, rad_solve_info* info, Scratch& ws, cudaStream_t s) {
    const int n = (int)h->n;
    const long long nv = (long long)n * nc;
    double* R = ws.get_n<double>(nv);
    double* D = ws.get_n<double>(nv);
    double* Tacc = static_cast<double*>(ws.get(apply_workspace_bytes_acc(h, nc)));
    ColReducer red(h, nc, 1, ws, s);
    const int nvc = red.nvc;
    double* bn2 = ws.get_n<double>(nvc);
    double* r2 = ws.get_n<double>(nvc);
    red.dots(B, 0, 1, B, bn2);
    std::vector<double> hb(nvc), hr(nvc);
    RAD_CUDA(cudaMemcpyAsync(hb.data(), bn2, sizeof(double) * nvc, cudaMemcpyDeviceToHost, s));
    RAD_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * nv, s));
    RAD_CUDA(cudaStreamSynchronize(s));
    rad_solve_params inner = *p;
    inner.tol = p->inner_tol;
    inner.refine = 0;
    int iters = 0, matvecs = 0, restarts = 0, step = 0, status = RAD_ENOTCONV;
    double max_rel = 0.0;
    for (;; ++step) {
        Epi epi{kResid, eps_t, X, B, nc};
        apply_tree_acc(h, X, nc, R, nc, nc, epi, Tacc, s);
        ++matvecs;
        red.dots(R, 0, 1, R, r2);
        RAD_CUDA(cudaMemcpyAsync(hr.data(), r2, sizeof(double) * nvc, cudaMemcpyDeviceToHost, s));
        RAD_CUDA(cudaStreamSynchronize(s));
        max_rel = 0.0;
        for (int c = 0; c < nvc; ++c)
            max_rel = std::max(max_rel, std::sqrt(std::max(hr[c], 0.0)) / (hb[c] > 0.0 ? std::sqrt(hb[c]) : 1.0));
        if (max_rel <= p->tol) {
            status = RAD_OK;
            break;
        }
        if (step >= p->max_refine || iters >= p->max_iter) break;
        rad_solve_info ii{};
        {
            Scratch inner_ws(s);
            gmres_tree(h, eps_t, R, nc, &inner, D, &ii, inner_ws, s);
        }
        iters += ii.iters;
        matvecs += ii.matvecs;
        restarts += ii.restarts;
        { ProfScope ps_("gmres_update_x", s); axpy_kernel<<<grid_for(nv), 256, 0, s>>>(X, D, nv); }
        RAD_CHECK_LAUNCH();
    }
    if (info) {
        info->status = status;
        info->iters = iters;
        info->restarts = restarts;
        info->matvecs = matvecs;
        info->max_rel_residual = max_rel;
        info->refinements = step;
    }
}

static void solve_tree(const rad_htree* h, const double* eps_t, const double* B, int nc, const rad_solve_params* p,
                       double* X, rad_solve_info* info, Scratch& ws, cudaStream_t s) {
    if (p->refine) refine_tree(h, eps_t, B, nc, p, X, info, ws, s);
    else gmres_tree(h, eps_t, B, nc, p, X, info, ws, s);
}

void solve_flux(const rad_htree* h, const double* eps_dev, const double* T_dev, int64_t ldT, int m, double sigma,
                const rad_solve_params* p, double* q_dev, int64_t ldq, rad_solve_info* info, cudaStream_t s) {
    const int n = (int)h->n;
    const int nc = m + 1;
    const bool op64 = h->op_is_f64();
    const long long nv = (long long)n * nc;
    Scratch ws(s);
    check_solve_inputs(n, eps_dev, T_dev, ldT, m, true, ws, s);
    double* eps_t = ws.get_n<double>(n);
    double* B = ws.get_n<double>(nv);
    double* X = ws.get_n<double>(nv);
    { ProfScope ps_("gmres_rhs", s); rhs_kernel<<<grid_for(nv), 256, 0, s>>>(n, m, eps_dev, T_dev, ldT, h->perm.as<int>(), eps_t, B); }
    RAD_CHECK_LAUNCH();
    rad_solve_info local{};
    solve_tree(h, eps_t, B, nc, p, X, &local, ws, s);
    // flux, Eq. (12): FY = F [Y z] (with the accurate operator when refining)
    void* Tws = ws.get(std::max(apply_workspace_bytes(h, nc), apply_workspace_bytes_acc(h, nc)));
    if (p->refine && !op64) {
        double* FY = ws.get_n<double>(nv);
        apply_tree_acc(h, X, nc, FY, nc, nc, Epi{kStore, nullptr, nullptr, nullptr, 0}, static_cast<double*>(Tws), s);
        { ProfScope ps_("flux", s); flux_kernel<double><<<grid_for((long long)n * m), 256, 0, s>>>(n, m, FY, h->perm.as<int>(), eps_dev, T_dev,
                                                                      ldT, sigma, q_dev, ldq); }
    } else if (op64) {
        double* FY = ws.get_n<double>(nv);
        apply_tree(h, X, nc, FY, nc, nc, Epi{kStore, nullptr, nullptr, nullptr, 0}, Tws, s);
        { ProfScope ps_("flux", s); flux_kernel<double><<<grid_for((long long)n * m), 256, 0, s>>>(n, m, FY, h->perm.as<int>(), eps_dev, T_dev,
                                                                      ldT, sigma, q_dev, ldq); }
    } else {
        const int ldp = tree_ld(nc);
        float* X32 = ws.get_n<float>((long long)n * ldp);
        float* FY = ws.get_n<float>(nv);
        { ProfScope ps_("gmres_convert", s); to_f32_kernel<<<grid_for(nv), 256, 0, s>>>(X, X32, nv, nc, ldp); }
        RAD_CHECK_LAUNCH();
        apply_tree(h, X32, ldp, FY, nc, nc, Epi{kStore, nullptr, nullptr, nullptr, 0}, Tws, s);
        { ProfScope ps_("flux", s); flux_kernel<float><<<grid_for((long long)n * m), 256, 0, s>>>(n, m, FY, h->perm.as<int>(), eps_dev, T_dev,
                                                                     ldT, sigma, q_dev, ldq); }
    }
    RAD_CHECK_LAUNCH();
    ++local.matvecs;
    RAD_CUDA(cudaStreamSynchronize(s));
    if (info) *info = local;
}

void solve_reflection(const rad_htree* h, const double* eps_dev, const double* B_dev, int64_t ldB, int nrhs,
                      const rad_solve_params* p, double* Y_dev, int64_t ldY, rad_solve_info* info, cudaStream_t s) {
    const int n = (int)h->n;
    const long long nv = (long long)n * nrhs;
    Scratch ws(s);
    check_solve_inputs(n, eps_dev, B_dev, ldB, nrhs, false, ws, s);
    double* eps_t = ws.get_n<double>(n);
    double* B = ws.get_n<double>(nv);
    double* X = ws.get_n<double>(nv);
    gather_user_to_tree(h, RAD_F64, eps_dev, n, 1, eps_t, 1, true, s);
    gather_user_to_tree(h, RAD_F64, B_dev, ldB, nrhs, B, nrhs, true, s);
    rad_solve_info local{};
    solve_tree(h, eps_t, B, nrhs, p, X, &local, ws, s);
    scatter_tree_to_user(h, X, nrhs, nrhs, true, RAD_F64, Y_dev, ldY, s);
    RAD_CUDA(cudaStreamSynchronize(s));
    if (info) *info = local;
}

}  // namespace rad
