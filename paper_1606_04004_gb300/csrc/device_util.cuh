// Device helpers shared by the kernels of the library: complex types, the
// rank/select bitmap over the direct-product lattice, block scans and
// compensated (double-float) accumulation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pq_internal.h"

namespace pq {

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

template <typename R>
__device__ __forceinline__ typename Cx<R>::T cmake(R x, R y) {
    typename Cx<R>::T v;
    v.x = x;
    v.y = y;
    return v;
}

// Bits [r*nlast, (r+1)*nlast) of the lattice bitmap: the active pattern of
// row r (bit s set <=> point (row r, last digit s) is active).
__device__ __forceinline__ uint64_t row_bits(const uint64_t* __restrict__ bits, uint32_t r,
                                             int nlast) {
    const uint64_t b0 = (uint64_t)r * (uint64_t)nlast;
    const uint32_t w = (uint32_t)(b0 >> 6);
    const int o = (int)(b0 & 63);
    uint64_t v = __ldg(bits + w) >> o;
    if (o + nlast > 64) v |= __ldg(bits + w + 1) << (64 - o);
    return nlast == 64 ? v : (v & ((1ull << nlast) - 1ull));
}

// Number of active points with linear index < b (position of b in A if b is
// active): exclusive popcount prefix of the word plus the bits below b.
__device__ __forceinline__ uint32_t rank_of(const uint64_t* __restrict__ bits,
                                            const uint32_t* __restrict__ off, uint64_t b) {
    const uint32_t w = (uint32_t)(b >> 6);
    const int o = (int)(b & 63);
    uint32_t r = __ldg(off + w);
    if (o) r += __popcll(__ldg(bits + w) & ((1ull << o) - 1ull));
    return r;
}

__device__ __forceinline__ bool bit_test(const uint64_t* __restrict__ bits, uint32_t b) {
    return (__ldg(bits + (b >> 6)) >> (b & 63)) & 1ull;
}

__device__ __forceinline__ void bit_set(uint64_t* bits, uint32_t b) {
    atomicOr(reinterpret_cast<unsigned long long*>(bits + (b >> 6)), 1ull << (b & 63));
}

// bit_set for a bitmap that only gains bits while it is being marked: a plain
// read first skips the atomic when the bit is already set (a stale read only
// costs the atomic it would have done anyway).
__device__ __forceinline__ void bit_mark(uint64_t* bits, uint32_t b) {
    const uint64_t m = 1ull << (b & 63);
    uint64_t* w = bits + (b >> 6);
    if (!(*reinterpret_cast<volatile uint64_t*>(w) & m))
        atomicOr(reinterpret_cast<unsigned long long*>(w), m);
}

// Bounds checks of the self-checking build (-DPQ_BOUNDS_CHECK): the first
// out-of-range index is recorded in cnt[CNT_FAULT..+2] and the access is
// skipped.  In the normal build the check compiles to `true`.
__device__ __forceinline__ bool pq_in_bounds(uint64_t idx, uint64_t bound, int site,
                                             int64_t* cnt) {
#ifdef PQ_BOUNDS_CHECK
    if (idx < bound) return true;
    if (cnt && atomicCAS(reinterpret_cast<unsigned long long*>(cnt + CNT_FAULT), 0ull,
                         (unsigned long long)site) == 0ull) {
        cnt[CNT_FAULT + 1] = (int64_t)idx;
        cnt[CNT_FAULT + 2] = (int64_t)bound;
    }
    return false;
#else
    (void)idx; (void)bound; (void)site; (void)cnt;
    return true;
#endif
}

// |a|^2 >= theta^2 evaluated as fl(fl(re*re) + fl(im*im)) >= fl(theta*theta)
// in FP64 without contraction (the adaption test of Sec. 2.5).
__device__ __forceinline__ bool significant64(double re, double im, double theta2) {
    return __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im)) >= theta2;
}

// FP32 values: decide in FP32 when clearly away from the threshold (relative
// error of the FP32 estimate is below 1e-6), else in exact-widened FP64.  The
// result equals the FP64 decision on the widened values.
__device__ __forceinline__ bool significant32(float re, float im, double theta2, float lo,
                                              float hi) {
    const float e = __fadd_rn(__fmul_rn(re, re), __fmul_rn(im, im));
    if (e > hi) return true;
    if (e < lo) return false;
    return significant64((double)re, (double)im, theta2);
}

// ----- double-float accumulation (error-free TwoSum, Knuth) for FP32 inputs
struct DF {
    float hi, lo;
};
__device__ __forceinline__ void df_add(DF& a, float b) {
    const float s = __fadd_rn(a.hi, b);
    const float bb = __fsub_rn(s, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, err);
}
__device__ __forceinline__ double df_value(const DF& a) { return (double)a.hi + (double)a.lo; }

// ----- warp / block sums
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Exclusive scan over a block of up to 1024 threads (blockDim multiple of 32).
// Returns the exclusive prefix of `v`; *total receives the block sum.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* sh /*32*/,
                                                         uint32_t* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;   // inclusive prefix of warp sums
    }
    __syncthreads();
    const uint32_t warp_off = wid ? sh[wid - 1] : 0;
    *total = sh[nw - 1];
    __syncthreads();
    return warp_off + x - v;
}

}  // namespace pq
