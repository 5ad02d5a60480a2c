// Deterministic grid reductions: warp shuffles, one shared-memory stage per block,
// per-block partials in global scratch, and the last block to finish (found with an
// atomic counter after a memory fence) sums the partials in block order and runs a
// finalisation functor on thread 0. The summation order depends only on the launch
// shape, so repeated runs give bit-identical results.
#pragma once
#include "internal.h"

namespace ovl {

template <int NV>
__device__ __forceinline__ void warp_sum(double v[NV]) {
#pragma unroll
    for (int k = 0; k < NV; k++)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
}

// Block-wide sum of v[NV]; the result is valid in thread 0. blockDim.x <= 1024.
template <int NV>
__device__ __forceinline__ void block_sum(double v[NV]) {
    __shared__ double sm[NV][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    warp_sum<NV>(v);
    __syncthreads();   // protect sm from a previous use in the same kernel
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; k++) sm[k][warp] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) v[k] = lane < nw ? sm[k][lane] : 0.0;
        warp_sum<NV>(v);
    }
}

// Block-wide sum of per-thread FP32 values: the warp stage in FP32 (shuffles), the sum
// over warps in FP64 by the first warp; the FP64 result is valid in thread 0. GB300 runs
// FP64 at 1/64 of its FP32 rate, so FP64 work stays at one warp per block.
template <int NV>
__device__ __forceinline__ void block_sum(const float vf[NV], double v[NV]) {
    __shared__ double sm[NV][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    float t[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) {
        t[k] = vf[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t[k] += __shfl_down_sync(0xffffffffu, t[k], off);
    }
    __syncthreads();   // protect sm from a previous use in the same kernel
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; k++) sm[k][warp] = (double)t[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) v[k] = lane < nw ? sm[k][lane] : 0.0;
        warp_sum<NV>(v);
    }
}
// Block-wide sum of per-thread float-float values: the warp stage in float-float (both
// words shuffled), the sum over warps in FP64 by the first warp.
template <int NV>
__device__ __forceinline__ void block_sum(const ff vf[NV], double v[NV]) {
    __shared__ double sm[NV][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    ff t[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) {
        t[k] = vf[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            t[k] += ff(__shfl_down_sync(0xffffffffu, t[k].hi, off), __shfl_down_sync(0xffffffffu, t[k].lo, off));
    }
    __syncthreads();   // protect sm from a previous use in the same kernel
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; k++) sm[k][warp] = t[k].to_double();
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) v[k] = lane < nw ? sm[k][lane] : 0.0;
        warp_sum<NV>(v);
    }
}
template <int NV>
__device__ __forceinline__ void block_sum(const double vd[NV], double v[NV]) {
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = vd[k];
    block_sum<NV>(v);
}

// Reduce v[NV] (per-thread FP64 or FP32 partial sums) over the grid; the last block calls
// fin(total) on thread 0 and resets the counter. Must be reached by every thread of every
// block.
template <int NV, typename T, typename Fin>
__device__ __forceinline__ void grid_reduce(const T vt[NV], RedScratch rs, Fin fin) {
    __shared__ int is_last;
    double v[NV];
    block_sum<NV>(vt, v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) rs.partials[k * kMaxRedBlocks + blockIdx.x] = v[k];
        __threadfence();
        unsigned t = atomicAdd(rs.counter, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        double s[NV];
#pragma unroll
        for (int k = 0; k < NV; k++) {
            s[k] = 0.0;
            for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
                s[k] += __ldcg(rs.partials + k * kMaxRedBlocks + b);
        }
        block_sum<NV>(s);
        if (threadIdx.x == 0) {
            fin(s);
            *rs.counter = 0u;
        }
    }
}

// As grid_reduce, but the last block runs fin(total, lane) on all 32 lanes of its first
// warp (for finalisations that are parallel over a small index, e.g. one lane per shift).
template <int NV, typename T, typename Fin>
__device__ __forceinline__ void grid_reduce_warp(const T vt[NV], RedScratch rs, Fin fin) {
    __shared__ int is_last;
    __shared__ double tot[NV];
    double v[NV];
    block_sum<NV>(vt, v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) rs.partials[k * kMaxRedBlocks + blockIdx.x] = v[k];
        __threadfence();
        unsigned t = atomicAdd(rs.counter, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        double s[NV];
#pragma unroll
        for (int k = 0; k < NV; k++) {
            s[k] = 0.0;
            for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
                s[k] += __ldcg(rs.partials + k * kMaxRedBlocks + b);
        }
        block_sum<NV>(s);
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < NV; k++) tot[k] = s[k];
        __syncthreads();
        if (threadIdx.x < 32) {
            double t2[NV];
#pragma unroll
            for (int k = 0; k < NV; k++) t2[k] = tot[k];
            fin(t2, (int)threadIdx.x);
            if (threadIdx.x == 0) *rs.counter = 0u;
        }
    }
}

// Last-block detection without values: returns true in every thread of the block that
// finishes last (after a fence that makes all blocks' global writes visible to it) and
// resets the counter. Must be reached by every thread of every block.
__device__ __forceinline__ bool grid_last_block(unsigned *counter) {
    __shared__ int is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned t = atomicAdd(counter, 1u);
        is_last = (t == gridDim.x - 1);
        if (is_last) *counter = 0u;
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

}  // namespace ovl
