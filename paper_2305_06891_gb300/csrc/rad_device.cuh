// Device helpers: reductions, scans and the view-factor entry of Eq. (10).
#pragma once

#include "rad_common.cuh"

namespace rad {

constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over a block of NT threads; every thread receives the total.
// `sm` needs NT/32 + 1 slots.  Reduction order is fixed (deterministic).
template <int NT, class T>
__device__ __forceinline__ T block_sum(T v, T* sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (warp == 0) {
        T t = lane < NT / 32 ? sm[lane] : T(0);
        t = warp_sum(t);
        if (lane == 0) sm[NT / 32] = t;
    }
    __syncthreads();
    T r = sm[NT / 32];
    __syncthreads();
    return r;
}

// Largest magnitude; ties go to the lowest index.  v < 0 marks "no candidate".
template <class T>
struct ArgMaxT {
    T v;
    int i;
};
using ArgMax = ArgMaxT<double>;
template <class T>
__device__ __forceinline__ ArgMaxT<T> am_better(ArgMaxT<T> a, ArgMaxT<T> b) {
    return (b.v > a.v || (b.v == a.v && b.i < a.i)) ? b : a;
}
template <class T>
__device__ __forceinline__ ArgMaxT<T> warp_argmax(ArgMaxT<T> a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ArgMaxT<T> b;
        b.v = __shfl_xor_sync(0xffffffffu, a.v, o);
        b.i = __shfl_xor_sync(0xffffffffu, a.i, o);
        a = am_better(a, b);
    }
    return a;
}
template <int NT, class T>
__device__ __forceinline__ ArgMaxT<T> block_argmax(ArgMaxT<T> a, ArgMaxT<T>* sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    a = warp_argmax(a);
    if (lane == 0) sm[warp] = a;
    __syncthreads();
    if (warp == 0) {
        ArgMaxT<T> t = lane < NT / 32 ? sm[lane] : ArgMaxT<T>{T(-1), 0x7fffffff};
        t = warp_argmax(t);
        if (lane == 0) sm[NT / 32] = t;
    }
    __syncthreads();
    ArgMaxT<T> r = sm[NT / 32];
    __syncthreads();
    return r;
}

// Exclusive scan over a block of NT threads (NT <= 1024).  `sm` needs
// NT/32 + 1 slots.  Returns the exclusive prefix; `total` gets the sum.
template <int NT, class T>
__device__ __forceinline__ T block_excl_scan(T v, T* sm, T& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) sm[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < NT / 32 ? sm[lane] : T(0);
        T wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < NT / 32) sm[lane] = wi - w;   // exclusive warp offsets
        if (lane == 31) sm[NT / 32] = wi;        // block total
    }
    __syncthreads();
    T r = sm[warp] + inc - v;
    total = sm[NT / 32];
    __syncthreads();
    return r;
}

// View factor F_ij, Eq. (10) with the 1-point centroid rule on both facets,
// in the textbook normalisation (divided by A_i):
//   d = c_j - c_i, a = n_i.d, b = -n_j.d,
//   F_ij = max(a,0) max(b,0) A_j / (pi |d|^4),  F_ii = 0.
// FP64 throughout.
__device__ __forceinline__ double vf_entry64(const Geo& g, int i, int j) {
    if (i == j) return 0.0;
    const double dx = g.cx[j] - g.cx[i];
    const double dy = g.cy[j] - g.cy[i];
    const double dz = g.cz[j] - g.cz[i];
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double a = g.nx[i] * dx + g.ny[i] * dy + g.nz[i] * dz;
    const double b = -(g.nx[j] * dx + g.ny[j] * dy + g.nz[j] * dz);
    if (!(a > 0.0) || !(b > 0.0) || !(r2 > 0.0)) return 0.0;
    const double inv = 1.0 / r2;
    return (a * inv) * (b * inv) * (g.area[j] * (1.0 / kPi));
}

// Same entry in FP32 arithmetic only.  The centroid difference is taken on
// hi/lo split coordinates, (hi_j - hi_i) + (lo_j - lo_i): the hi difference
// is exact for nearby facets (Sterbenz) and the lo terms restore the bits
// lost when the coordinates were rounded, so there is no cancellation.
__device__ __forceinline__ float vf_entry32(const Geo& g, int i, int j) {
    if (i == j) return 0.0f;
    const float dx = (g.xh[j] - g.xh[i]) + (g.xl[j] - g.xl[i]);
    const float dy = (g.yh[j] - g.yh[i]) + (g.yl[j] - g.yl[i]);
    const float dz = (g.zh[j] - g.zh[i]) + (g.zl[j] - g.zl[i]);
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float a = g.fnx[i] * dx + g.fny[i] * dy + g.fnz[i] * dz;
    const float b = -(g.fnx[j] * dx + g.fny[j] * dy + g.fnz[j] * dz);
    if (!(a > 0.0f) || !(b > 0.0f) || !(r2 > 0.0f)) return 0.0f;
    const float inv = 1.0f / r2;
    return (a * inv) * (b * inv) * (g.farea[j] * (float)(1.0 / kPi));
}

template <class CT> struct Entry;
template <> struct Entry<double> {
    static __device__ __forceinline__ double eval(const Geo& g, int i, int j) { return vf_entry64(g, i, j); }
};
template <> struct Entry<float> {
    static __device__ __forceinline__ float eval(const Geo& g, int i, int j) { return vf_entry32(g, i, j); }
};

// Storage conversions.
template <class S> struct Store;
template <> struct Store<double> {
    static __device__ __forceinline__ double put(double v) { return v; }
    static __device__ __forceinline__ double put(float v) { return (double)v; }
    static __device__ __forceinline__ double get(double v) { return v; }
};
template <> struct Store<float> {
    static __device__ __forceinline__ float put(double v) { return (float)v; }
    static __device__ __forceinline__ float put(float v) { return v; }
    static __device__ __forceinline__ float get(float v) { return v; }
};
template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ __nv_bfloat16 put(double v) { return __float2bfloat16_rn((float)v); }
    static __device__ __forceinline__ __nv_bfloat16 put(float v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ float get(__nv_bfloat16 v) { return __bfloat162float(v); }
};

}  // namespace rad
