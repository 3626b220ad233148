// A1-A3: facet geometry (§3.1), cluster tree (§4.1, Algorithm 1) and block
// tree (§4.2, Algorithm 2 with the admissibility condition Eq. 28).
//
// The cluster tree is built level by level, one CTA per cluster:
//   1. bounding box of the cluster's centroids (exact min/max reduction);
//   2. split axis = longest box extent (ties: lowest axis);
//   3. radix select (8 passes of 8 bits over an order-preserving 64-bit key
//      of the coordinate) of the floor(n/2)-th smallest (coordinate, index);
//   4. stable partition into left/right halves, so that every cluster keeps
//      its facets in ascending facet index.
// The cluster shapes (ranges) depend only on n and leaf_size and are laid
// out breadth first on the host; only boxes and the permutation are computed
// on the device.  The result is deterministic and equal bit for bit to the
// recursive definition evaluated in FP64.
//
// The block tree runs in one CTA that walks the candidate blocks level by
// level, classifying each as admissible (low-rank leaf), dense leaf (a
// cluster has no children) or split into 4 children, with block scans for
// deterministic compaction.

#include <algorithm>
#include <climits>
#include <cfloat>

#include "rad_device.cuh"

namespace rad {

namespace {

// --------------------------------------------------------------- geometry
// centroid c = ((v0 + v1) + v2) / 3, n = (v1 - v0) x (v2 - v0), A = |n| / 2.
// The centroid feeds the bit-exact tree, so its arithmetic is pinned with
// explicit round-to-nearest intrinsics (no contraction).
__global__ void geometry_tris_kernel(int n, const double* __restrict__ verts, double* __restrict__ geo,
                                     int* __restrict__ bad) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    const double* v = verts + 9ll * f;
    double c[3], e1[3], e2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        c[k] = __ddiv_rn(__dadd_rn(__dadd_rn(v[k], v[3 + k]), v[6 + k]), 3.0);
        e1[k] = __dsub_rn(v[3 + k], v[k]);
        e2[k] = __dsub_rn(v[6 + k], v[k]);
    }
    const double nx = __dsub_rn(__dmul_rn(e1[1], e2[2]), __dmul_rn(e1[2], e2[1]));
    const double ny = __dsub_rn(__dmul_rn(e1[2], e2[0]), __dmul_rn(e1[0], e2[2]));
    const double nz = __dsub_rn(__dmul_rn(e1[0], e2[1]), __dmul_rn(e1[1], e2[0]));
    const double nn = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(nx, nx), __dmul_rn(ny, ny)), __dmul_rn(nz, nz)));
    const bool ok = isfinite(c[0]) && isfinite(c[1]) && isfinite(c[2]) && isfinite(nn) && nn > 0.0;
    if (!ok) atomicOr(bad, 1);
    const int64_t N = n;
    geo[f] = c[0];
    geo[N + f] = c[1];
    geo[2 * N + f] = c[2];
    geo[3 * N + f] = ok ? nx / nn : 0.0;
    geo[4 * N + f] = ok ? ny / nn : 0.0;
    geo[5 * N + f] = ok ? nz / nn : 0.0;
    geo[6 * N + f] = 0.5 * nn;
}

__global__ void geometry_facets_kernel(int n, const double* __restrict__ c, const double* __restrict__ nrm,
                                       const double* __restrict__ a, double* __restrict__ geo,
                                       int* __restrict__ bad) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    const int64_t N = n;
    bool ok = isfinite(a[f]) && a[f] > 0.0;
    for (int k = 0; k < 3; ++k) {
        ok = ok && isfinite(c[3ll * f + k]) && isfinite(nrm[3ll * f + k]);
        geo[k * N + f] = c[3ll * f + k];
        geo[(3 + k) * N + f] = nrm[3ll * f + k];
    }
    geo[6 * N + f] = a[f];
    if (!ok) atomicOr(bad, 1);
}

// --------------------------------------------------------------- cluster tree
__device__ __forceinline__ unsigned long long order_key(double x) {
    x = x + 0.0;  // -0.0 -> +0.0: equal coordinates get equal keys
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

constexpr int kTreeNT = 1024;

__device__ __forceinline__ void warp_minmax(double& lo, double& hi) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
}

__global__ void __launch_bounds__(kTreeNT)
tree_level_kernel(const NodeShape* __restrict__ shapes, NodeBox* __restrict__ boxes, int first,
                  const double* __restrict__ cx, const double* __restrict__ cy, const double* __restrict__ cz,
                  const int* __restrict__ idx_in, int* __restrict__ idx_out,
                  unsigned long long* __restrict__ keys, int* __restrict__ err) {
    constexpr int NT = kTreeNT;
    __shared__ double s_lo[3][NT / 32], s_hi[3][NT / 32];
    __shared__ unsigned int hist[256];
    __shared__ int scan_sm[NT / 32 + 1];
    __shared__ int sel_digit, sel_want;
    __shared__ double s_box[6];

    const int node = first + blockIdx.x;
    const NodeShape nd = shapes[node];
    const int b = nd.begin, e = nd.end, n = e - b;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // 1. bounding box of the centroids (exact, order independent)
    double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (int p = b + threadIdx.x; p < e; p += NT) {
        const int f = idx_in[p];
        const double x[3] = {cx[f], cy[f], cz[f]};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], x[k]);
            hi[k] = fmax(hi[k], x[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        warp_minmax(lo[k], hi[k]);
        if (lane == 0) {
            s_lo[k][warp] = lo[k];
            s_hi[k][warp] = hi[k];
        }
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double l = lane < NT / 32 ? s_lo[k][lane] : DBL_MAX;
            double h = lane < NT / 32 ? s_hi[k][lane] : -DBL_MAX;
            warp_minmax(l, h);
            if (lane == 0) {
                s_box[k] = l;
                s_box[3 + k] = h;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        NodeBox bx;
        for (int k = 0; k < 3; ++k) {
            bx.lo[k] = s_box[k];
            bx.hi[k] = s_box[3 + k];
        }
        boxes[node] = bx;
    }
    if (nd.leaf) {
        for (int p = b + threadIdx.x; p < e; p += NT) idx_out[p] = idx_in[p];
        return;
    }

    // 2. split axis: largest extent, ties to the lowest axis
    const double ext0 = __dsub_rn(s_box[3], s_box[0]);
    const double ext1 = __dsub_rn(s_box[4], s_box[1]);
    const double ext2 = __dsub_rn(s_box[5], s_box[2]);
    int axis = 0;
    double best = ext0;
    if (ext1 > best) { axis = 1; best = ext1; }
    if (ext2 > best) { axis = 2; }
    const double* ca = axis == 0 ? cx : axis == 1 ? cy : cz;
    for (int p = b + threadIdx.x; p < e; p += NT) keys[p] = order_key(ca[idx_in[p]]);
    __syncthreads();

    // 3. radix select of the pivot key: the (h-1)-th smallest, h = floor(n/2)
    const int h = n / 2;
    unsigned long long prefix = 0ull, mask = 0ull;
    int want = h - 1;
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        for (int t = threadIdx.x; t < 256; t += NT) hist[t] = 0u;
        __syncthreads();
        for (int p = b + threadIdx.x; p < e; p += NT) {
            const unsigned long long k = keys[p];
            if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 0xffull], 1u);
        }
        __syncthreads();
        if (warp == 0) {
            // digit d holding rank `want`: lane q scans bins 8q .. 8q + 7
            unsigned loc[8], sum = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                loc[j] = hist[8 * lane + j];
                sum += loc[j];
            }
            unsigned incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int excl = (int)(incl - sum);
            if (want >= excl && want < (int)incl) {
                int cum = excl, d = 8 * lane;
#pragma unroll
                for (int j = 0; j < 7; ++j) {
                    if (want < cum + (int)loc[j]) break;
                    cum += (int)loc[j];
                    ++d;
                }
                sel_digit = d;
                sel_want = want - cum;
            }
        }
        __syncthreads();
        prefix |= (unsigned long long)sel_digit << shift;
        mask |= 0xffull << shift;
        want = sel_want;
        __syncthreads();
    }
    const unsigned long long pkey = prefix;
    const int n_eq_left = want + 1;  // equal keys that go left, in index order

    // 4. stable partition (left: key < pivot, or key == pivot among the
    //    first n_eq_left equal keys in list order): each thread takes a
    //    contiguous segment of the node, counts, two block scans give the
    //    offsets, and the thread writes its segment in order
    const int per = (n + NT - 1) / NT;
    const int s0 = min(e, b + (int)threadIdx.x * per), s1 = min(e, s0 + per);
    int cl = 0, ce = 0;
    for (int p = s0; p < s1; ++p) {
        const unsigned long long k = keys[p];
        cl += k < pkey ? 1 : 0;
        ce += k == pkey ? 1 : 0;
    }
    int eqtot;
    const int eq_before = block_excl_scan<NT, int>(ce, scan_sm, eqtot);
    const int gl = cl + min(ce, max(0, n_eq_left - eq_before));
    int ltot;
    const int l_before = block_excl_scan<NT, int>(gl, scan_sm, ltot);
    int li = 0, ri = 0, eqi = 0;
    const int r_before = (s0 - b) - l_before;
    for (int p = s0; p < s1; ++p) {
        const unsigned long long k = keys[p];
        bool left = k < pkey;
        if (k == pkey) left = eq_before + eqi++ < n_eq_left;
        const int dst = left ? b + l_before + li++ : b + h + r_before + ri++;
        const bool ok = left ? dst < b + h : (dst >= b + h && dst < e);
        if (ok) idx_out[dst] = idx_in[p];
        else atomicOr(err, 4);
    }
    if (threadIdx.x == 0 && ltot != h) atomicOr(err, 2);
}

__global__ void gather_geo_kernel(int n, const double* __restrict__ geo_user, const int* __restrict__ perm,
                                  double* __restrict__ geo_tree, int* __restrict__ iperm) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int f = perm[p];
    const int64_t N = n;
#pragma unroll
    for (int k = 0; k < 7; ++k) geo_tree[k * N + p] = geo_user[k * N + f];
    iperm[f] = p;
}

// FP32 view of the tree-ordered geometry: centroids split into hi/lo floats.
__global__ void geo32_kernel(int n, const double* __restrict__ geo, float* __restrict__ g32) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t N = n;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double c = geo[k * N + p];
        const float hi = __double2float_rn(c);
        g32[(2 * k) * N + p] = hi;
        g32[(2 * k + 1) * N + p] = __double2float_rn(c - (double)hi);
    }
#pragma unroll
    for (int k = 3; k < 7; ++k) g32[(k + 3) * N + p] = __double2float_rn(geo[k * N + p]);
}

// --------------------------------------------------------------- block tree
// Eq. (28) in squared form on the centroid boxes, FP64 with every product
// and sum rounded separately (no contraction):
//   admissible <=> dist^2 > 0 and min(diam_s^2, diam_t^2) <= (eta*eta) dist^2
__device__ __forceinline__ double sq3(double a, double b, double c) {
    return __dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(c, c));
}
__device__ __forceinline__ bool admissible(const NodeBox& s, const NodeBox& t, double eta) {
    double g[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double a = __dsub_rn(t.lo[k], s.hi[k]);
        const double c = __dsub_rn(s.lo[k], t.hi[k]);
        g[k] = fmax(0.0, fmax(a, c));
    }
    const double dist2 = sq3(g[0], g[1], g[2]);
    if (!(dist2 > 0.0)) return false;
    const double ds = sq3(__dsub_rn(s.hi[0], s.lo[0]), __dsub_rn(s.hi[1], s.lo[1]), __dsub_rn(s.hi[2], s.lo[2]));
    const double dt = sq3(__dsub_rn(t.hi[0], t.lo[0]), __dsub_rn(t.hi[1], t.lo[1]), __dsub_rn(t.hi[2], t.lo[2]));
    return fmin(ds, dt) <= __dmul_rn(__dmul_rn(eta, eta), dist2);
}

// One level of Algorithm 2 for every tree of the forest at once: each
// candidate pair (sigma, tau) becomes a far block (Eq. 28 holds), a near
// block (a leaf on either side) or its four child pairs for the next level.
// Outputs are appended with warp-aggregated atomics, so their order is not
// fixed; the host orders the blocks by (row start, column start) afterwards.
// lv[0] = candidates of this level (read), lv[1] = next level's count,
// tot[0 / 1] = far / near blocks so far.  Writes past a capacity are
// dropped; the counts keep growing so the host can retry with room.
constexpr int kLevelNT = 256;
__global__ void __launch_bounds__(kLevelNT)
block_level_kernel(const NodeShape* __restrict__ shapes, const NodeBox* __restrict__ boxes, double eta,
                   const int2* __restrict__ cur, int2* __restrict__ nxt, int cap_cand, int2* __restrict__ far_out,
                   int2* __restrict__ near_out, int cap_out, int* lv, int* tot) {
    const int ncur = min(lv[0], cap_cand);
    const int lane = threadIdx.x & 31;
    for (int base = blockIdx.x * kLevelNT; base < ncur; base += gridDim.x * kLevelNT) {
        const int t = base + (int)threadIdx.x;
        int cls = -1;
        int2 pr = make_int2(0, 0);
        NodeShape ns{}, nt{};
        if (t < ncur) {
            pr = cur[t];
            ns = shapes[pr.x];
            nt = shapes[pr.y];
            if (admissible(boxes[pr.x], boxes[pr.y], eta)) cls = 1;
            else if (ns.leaf || nt.leaf) cls = 2;
            else cls = 0;
        }
        const unsigned mf = __ballot_sync(0xffffffffu, cls == 1);
        const unsigned mn = __ballot_sync(0xffffffffu, cls == 2);
        const unsigned mc = __ballot_sync(0xffffffffu, cls == 0);
        const unsigned below = (1u << lane) - 1u;
        int bf = 0, bn = 0, bc = 0;
        if (lane == 0) {
            if (mf) bf = atomicAdd(&tot[0], __popc(mf));
            if (mn) bn = atomicAdd(&tot[1], __popc(mn));
            if (mc) bc = atomicAdd(&lv[1], 4 * __popc(mc));
        }
        bf = __shfl_sync(0xffffffffu, bf, 0);
        bn = __shfl_sync(0xffffffffu, bn, 0);
        bc = __shfl_sync(0xffffffffu, bc, 0);
        if (cls == 1) {
            const int pos = bf + __popc(mf & below);
            if (pos < cap_out) far_out[pos] = pr;
        } else if (cls == 2) {
            const int pos = bn + __popc(mn & below);
            if (pos < cap_out) near_out[pos] = pr;
        } else if (cls == 0) {
            const int pos = bc + 4 * __popc(mc & below);
            const int cs[2] = {ns.child0, ns.child1};
            const int ct[2] = {nt.child0, nt.child1};
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (pos + q < cap_cand) nxt[pos + q] = make_int2(cs[q >> 1], ct[q & 1]);
        }
    }
}

}  // namespace

void build_geometry_from_tris(rad_htree* h, const double* verts_dev, double* geo_user, cudaStream_t s) {
    Scratch ws(s);
    int* bad = ws.get_n<int>(1);
    RAD_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    const int n = (int)h->n;
    { ProfScope ps_("geometry", s); geometry_tris_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, verts_dev, geo_user, bad); }
    RAD_CHECK_LAUNCH();
    int hb = 0;
    RAD_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    RAD_CUDA(cudaStreamSynchronize(s));
    RAD_REQUIRE(hb == 0, RAD_EINVAL, "degenerate or non-finite triangle in verts");
}

void build_geometry_from_facets(rad_htree* h, const double* c, const double* nrm, const double* a,
                                double* geo_user, cudaStream_t s) {
    Scratch ws(s);
    int* bad = ws.get_n<int>(1);
    RAD_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    const int n = (int)h->n;
    { ProfScope ps_("geometry", s); geometry_facets_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, c, nrm, a, geo_user, bad); }
    RAD_CHECK_LAUNCH();
    int hb = 0;
    RAD_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    RAD_CUDA(cudaStreamSynchronize(s));
    RAD_REQUIRE(hb == 0, RAD_EINVAL, "non-finite facet data or non-positive area");
}

void build_trees(rad_htree* h, const double* geo_user, cudaStream_t s) {
    const int n = (int)h->n;
    const int leaf = h->leaf_size;
    // cluster shapes, breadth first: Algorithm 1's recursion on sizes only
    std::vector<NodeShape>& nodes = h->nodes;
    HostScope hs_shapes("host_tree_shapes");
    StageScope stage;
    nodes.clear();
    // one root per segment (cavity): a batch is a forest whose trees never
    // meet, so no block couples two cavities
    if (h->seg.empty()) h->seg = {0, (int64_t)n};
    const int nseg = (int)h->seg.size() - 1;
    std::vector<int> roots(nseg);
    for (int c = 0; c < nseg; ++c) {
        const int b0 = (int)h->seg[c], b1 = (int)h->seg[c + 1];
        roots[c] = (int)nodes.size();
        nodes.push_back(NodeShape{b0, b1, 0, -1, -1, b1 - b0 <= leaf ? 1 : 0});
    }
    for (size_t q = 0; q < nodes.size(); ++q) {
        NodeShape nd = nodes[q];
        if (nd.leaf) continue;
        const int half = (nd.end - nd.begin) / 2;
        const int c0 = (int)nodes.size();
        nodes[q].child0 = c0;
        nodes[q].child1 = c0 + 1;
        const int sz0 = half, sz1 = nd.end - nd.begin - half;
        nodes.push_back(NodeShape{nd.begin, nd.begin + half, nd.level + 1, -1, -1, sz0 <= leaf ? 1 : 0});
        nodes.push_back(NodeShape{nd.begin + half, nd.end, nd.level + 1, -1, -1, sz1 <= leaf ? 1 : 0});
    }
    const int n_nodes = (int)nodes.size();
    int depth = 0;
    for (auto& nd : nodes) depth = std::max(depth, nd.level + 1);
    h->depth = depth;
    std::vector<int> level_first(depth + 1, n_nodes);
    for (int q = n_nodes - 1; q >= 0; --q) level_first[nodes[q].level] = q;
    level_first[depth] = n_nodes;

    Scratch ws(s);
    NodeShape* d_shapes = ws.get_n<NodeShape>(n_nodes);
    NodeBox* d_boxes = ws.get_n<NodeBox>(n_nodes);
    int* idx[2] = {ws.get_n<int>(n), ws.get_n<int>(n)};
    unsigned long long* keys = ws.get_n<unsigned long long>(n);
    int* err = ws.get_n<int>(1);
    RAD_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    h2d(d_shapes, nodes, s);
    std::vector<int> ident(n);
    for (int i = 0; i < n; ++i) ident[i] = i;
    h2d(idx[0], ident, s);
    h2d(idx[1], ident, s);

    const double* cx = geo_user;
    const double* cy = geo_user + n;
    const double* cz = geo_user + 2ll * n;
    for (int lv = 0; lv < depth; ++lv) {
        const int cnt = level_first[lv + 1] - level_first[lv];
        { ProfScope ps_("cluster_tree", s); tree_level_kernel<<<cnt, kTreeNT, 0, s>>>(d_shapes, d_boxes, level_first[lv], cx, cy, cz,
                                                  idx[lv & 1], idx[(lv + 1) & 1], keys, err); }
        RAD_CHECK_LAUNCH();
    }
    int* perm_final = idx[depth & 1];

    h->perm.alloc(sizeof(int) * n, s);
    h->iperm.alloc(sizeof(int) * n, s);
    h->geo.alloc(sizeof(double) * 7 * (size_t)n, s);
    RAD_CUDA(cudaMemcpyAsync(h->perm.p, perm_final, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    { ProfScope ps_("geometry", s); gather_geo_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, geo_user, perm_final, h->geo.as<double>(),
                                                      h->iperm.as<int>()); }
    RAD_CHECK_LAUNCH();
    h->geo32.alloc(sizeof(float) * 10 * (size_t)n, s);
    { ProfScope ps_("geometry", s); geo32_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, h->geo.as<double>(), h->geo32.as<float>()); }
    RAD_CHECK_LAUNCH();

    // block tree: one launch per level over the candidates of every tree,
    // retry with larger buffers on overflow
    HostScope hs_blocks("host_block_tree_wait");
    int64_t cap64 = 0;
    for (int c = 0; c < nseg; ++c) {
        const int64_t nc_ = h->seg[c + 1] - h->seg[c];
        cap64 += 160ll * (nc_ / std::max(1, leaf) + 1) + 4096;
    }
    int cap = (int)std::min<int64_t>(1 << 28, cap64);
    std::vector<int2> far_pairs, near_pairs;
    std::vector<int2> root_pairs(nseg);
    for (int c = 0; c < nseg; ++c) root_pairs[c] = make_int2(roots[c], roots[c]);
    const int levels = depth + 1;
    bool done = false;
    for (int attempt = 0; attempt < 6 && !done; ++attempt) {
        Scratch bw(s);
        int2* candA = bw.get_n<int2>(cap);
        int2* candB = bw.get_n<int2>(cap);
        int2* far_out = bw.get_n<int2>(cap);
        int2* near_out = bw.get_n<int2>(cap);
        int* lv = bw.get_n<int>(levels + 2);      // candidates per level
        int* tot = bw.get_n<int>(2);
        RAD_CUDA(cudaMemsetAsync(lv, 0, sizeof(int) * (levels + 2), s));
        RAD_CUDA(cudaMemsetAsync(tot, 0, sizeof(int) * 2, s));
        h2d(candA, root_pairs, s);
        const int one[1] = {nseg};
        RAD_CUDA(cudaMemcpyAsync(lv, one, sizeof(int), cudaMemcpyHostToDevice, s));
        {
            ProfScope ps_("block_tree", s);
            for (int l = 0; l < levels; ++l) {
                block_level_kernel<<<152 * 8, kLevelNT, 0, s>>>(d_shapes, d_boxes, h->eta, (l & 1) ? candB : candA,
                                                                (l & 1) ? candA : candB, cap, far_out, near_out, cap,
                                                                lv + l, tot);
                RAD_CHECK_LAUNCH();
            }
        }
        std::vector<int> hl(levels + 2), ht(2);
        RAD_CUDA(cudaMemcpyAsync(hl.data(), lv, sizeof(int) * hl.size(), cudaMemcpyDeviceToHost, s));
        RAD_CUDA(cudaMemcpyAsync(ht.data(), tot, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
        RAD_CUDA(cudaStreamSynchronize(s));
        int64_t need = std::max<int64_t>(ht[0], ht[1]);
        for (int l = 0; l <= levels; ++l) need = std::max<int64_t>(need, hl[l]);
        RAD_REQUIRE(hl[levels] == 0, RAD_ECUDA, "internal error: block tree deeper than the cluster tree");
        if (need > cap) {
            RAD_REQUIRE(cap < (1 << 28), RAD_ELIMIT, "block tree too large");
            cap = (int)std::min<int64_t>(1 << 28, std::max<int64_t>(4ll * cap, need + 1024));
            continue;
        }
        far_pairs.resize(ht[0]);
        near_pairs.resize(ht[1]);
        if (ht[0]) RAD_CUDA(cudaMemcpyAsync(far_pairs.data(), far_out, sizeof(int2) * ht[0], cudaMemcpyDeviceToHost, s));
        if (ht[1]) RAD_CUDA(cudaMemcpyAsync(near_pairs.data(), near_out, sizeof(int2) * ht[1], cudaMemcpyDeviceToHost, s));
        RAD_CUDA(cudaStreamSynchronize(s));
        done = true;
    }
    RAD_REQUIRE(done, RAD_ELIMIT, "block tree did not fit");
    RAD_REQUIRE(!(far_pairs.empty() && near_pairs.empty()), RAD_ELIMIT, "block tree did not fit");

    h->boxes.resize(n_nodes);
    h->perm_h.resize(n);
    RAD_CUDA(cudaMemcpyAsync(h->boxes.data(), d_boxes, sizeof(NodeBox) * n_nodes, cudaMemcpyDeviceToHost, s));
    RAD_CUDA(cudaMemcpyAsync(h->perm_h.data(), perm_final, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
    int herr = 0;
    RAD_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    RAD_CUDA(cudaStreamSynchronize(s));
    RAD_REQUIRE(herr == 0, RAD_ECUDA, "internal error in the cluster-tree partition");

    HostScope hs_sort("host_block_list");
    // Blocks ordered by (row start, column start), which identifies a block
    // uniquely.  Lists of 8,000 blocks or more: the pairs are bucketed by
    // row range (counts per input chunk and range, then a scatter) and each
    // range is ordered by row start (counting) and, within a row start, by
    // column start, on kListParts host threads; the order does not depend on
    // the part count.
    std::vector<BlockH>& blocks = h->blocks;
    const int64_t nfp = (int64_t)far_pairs.size(), nb = nfp + (int64_t)near_pairs.size();
    RAD_REQUIRE(nb < INT32_MAX, RAD_ELIMIT, "too many blocks");
    auto pair_at = [&](int64_t i) { return i < nfp ? far_pairs[i] : near_pairs[i - nfp]; };
    constexpr int kListParts = 16;
    if (nb < 8000) {
        // small lists: build in input order, then two stable counting
        // passes (column start, then row start) over the block array
        blocks.clear();
        blocks.reserve(nb);
        for (int64_t i = 0; i < nb; ++i) {
            const int2 pr = pair_at(i);
            const NodeShape& a = nodes[pr.x];
            const NodeShape& bn = nodes[pr.y];
            const int adm = i < nfp ? 1 : 0;
            blocks.push_back(BlockH{pr.x, pr.y, a.begin, a.end, bn.begin, bn.end, adm, adm ? 0 : -1, -1, 0});
        }
        std::vector<int> cn(n + 2);
        std::vector<BlockH> tmp(blocks.size());
        for (int pass = 0; pass < 2; ++pass) {
            std::fill(cn.begin(), cn.end(), 0);
            for (auto& b : blocks) ++cn[(pass ? b.r0 : b.c0) + 1];
            for (int i = 0; i <= n; ++i) cn[i + 1] += cn[i];
            for (auto& b : blocks) tmp[cn[pass ? b.r0 : b.c0]++] = b;
            blocks.swap(tmp);
        }
        h->n_admissible = (int64_t)far_pairs.size();
        return;
    }
    const int P = kListParts;
    std::vector<int> rcut(P + 1);
    for (int q = 0; q <= P; ++q) rcut[q] = (int)((int64_t)n * q / P);
    auto range_of = [&](int r0) { return (int)(std::upper_bound(rcut.begin() + 1, rcut.end() - 1, r0) - rcut.begin()) - 1; };
    std::vector<int64_t> cnt((size_t)P * P, 0);
    parallel_parts(P, [&](int t) {
        int64_t* c = &cnt[(size_t)t * P];
        for (int64_t i = nb * t / P, e = nb * (t + 1) / P; i < e; ++i) ++c[range_of(nodes[pair_at(i).x].begin)];
    });
    std::vector<int64_t> off((size_t)P * P), rstart(P + 1, 0);
    {
        int64_t acc = 0;
        for (int q = 0; q < P; ++q) {
            rstart[q] = acc;
            for (int t = 0; t < P; ++t) {
                off[(size_t)t * P + q] = acc;
                acc += cnt[(size_t)t * P + q];
            }
        }
        rstart[P] = acc;
    }
    std::vector<int> bucket(nb);
    parallel_parts(P, [&](int t) {
        int64_t* o = &off[(size_t)t * P];
        for (int64_t i = nb * t / P, e = nb * (t + 1) / P; i < e; ++i)
            bucket[o[range_of(nodes[pair_at(i).x].begin)]++] = (int)i;
    });
    blocks.resize(nb);
    parallel_parts(P, [&](int q) {
        const int lo = rcut[q], hi = rcut[q + 1];
        const int64_t b0 = rstart[q], b1 = rstart[q + 1];
        std::vector<int> c(hi - lo + 1, 0), ord(b1 - b0);
        for (int64_t k = b0; k < b1; ++k) ++c[nodes[pair_at(bucket[k]).x].begin - lo + 1];
        for (int r = 0; r < hi - lo; ++r) c[r + 1] += c[r];
        for (int64_t k = b0; k < b1; ++k) ord[c[nodes[pair_at(bucket[k]).x].begin - lo]++] = bucket[k];
        auto c0_of = [&](int i) { return nodes[pair_at(i).y].begin; };
        for (int64_t g0 = 0; g0 < b1 - b0;) {
            const int r0 = nodes[pair_at(ord[g0]).x].begin;
            int64_t g1 = g0 + 1;
            while (g1 < b1 - b0 && nodes[pair_at(ord[g1]).x].begin == r0) ++g1;
            std::sort(ord.begin() + g0, ord.begin() + g1, [&](int x, int y) { return c0_of(x) < c0_of(y); });
            g0 = g1;
        }
        for (int64_t k = 0; k < b1 - b0; ++k) {
            const int i = ord[k];
            const int2 pr = pair_at(i);
            const NodeShape& a = nodes[pr.x];
            const NodeShape& bn = nodes[pr.y];
            const int adm = i < nfp ? 1 : 0;
            blocks[b0 + k] = BlockH{pr.x, pr.y, a.begin, a.end, bn.begin, bn.end, adm, adm ? 0 : -1, -1, 0};
        }
    });
    h->n_admissible = (int64_t)far_pairs.size();
}

}  // namespace rad
