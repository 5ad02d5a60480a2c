// Measured fused multiply-add throughput of the current GPU, FP64 and FP32.
//
// The FP64 stencils are bound by the FP64 pipes (GB300 issues about 2 FP64 FMAs per clock
// per SM, 1/64 of its FP32 rate), so their roofline denominator is an FP64 FMA rate, and
// the float-float stencil's is the FP32 rate. This kernel measures both on the running
// device rather than quoting nominal figures: every thread runs NC independent chains
// a_k <- a_k * s + t (enough independent chains to cover the pipe latency), grids of a
// few blocks per SM, timed with CUDA events after a warm-up launch.
#include <math.h>

#include <algorithm>
#include <string>

#include "../../include/ovl.h"
#include "internal.h"

namespace ovl {
namespace {

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) { return __fma_rn(a, b, c); }
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }

template <typename T, int NC>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, T s, T t, T *sink) {
    T a[NC];
#pragma unroll
    for (int k = 0; k < NC; k++) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 8; u++)
#pragma unroll
            for (int k = 0; k < NC; k++) a[k] = fma_t<T>(a[k], s, t);
    }
    T sum = 0;
#pragma unroll
    for (int k = 0; k < NC; k++) sum += a[k];
    if (sum == (T)-12345.0) *sink = sum;   // never true; keeps the chains alive
}

template <typename T, int NC>
cudaError_t time_peak(int blocks, int iters, T *sink, cudaStream_t st, float *ms) {
    cudaEvent_t e0, e1;
    cudaError_t e;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    k_fma_peak<T, NC><<<blocks, 256, 0, st>>>(iters, (T)0.999999, (T)1e-6, sink);   // warm-up
    cudaEventRecord(e0, st);
    k_fma_peak<T, NC><<<blocks, 256, 0, st>>>(iters, (T)0.999999, (T)1e-6, sink);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    count_launches(2);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

}  // namespace
}  // namespace ovl

using namespace ovl;

extern "C" ovl_status ovl_fma_peak(int precision, double *gflops) {
    if (!gflops || (precision != 0 && precision != 1)) return OVL_EINVAL;
    *gflops = 0.0;
    const int blocks = 8 * device_sm_count();
    void *sink = nullptr;
    cudaStream_t st = nullptr;
    ovl_status rc = OVL_OK;
    if (cudaMalloc(&sink, 16) != cudaSuccess || cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        if (sink) cudaFree(sink);
        set_thread_error("ovl_fma_peak: CUDA allocation or stream creation failed");
        return OVL_ECUDA;
    }
    // grow the trip count until one launch takes >= 20 ms
    int iters = 64, timed_iters = 64;
    float ms = 0.f;
    for (int rep = 0; rep < 24; rep++) {
        timed_iters = iters;
        cudaError_t e = precision == 0 ? time_peak<double, 8>(blocks, iters, (double *)sink, st, &ms)
                                       : time_peak<float, 16>(blocks, iters, (float *)sink, st, &ms);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_thread_error(std::string("ovl_fma_peak: ") + cudaGetErrorString(e));
            rc = OVL_ECUDA;
            break;
        }
        if (ms >= 20.f || iters > (1 << 26)) break;
        const long grown = (long)iters * (ms > 0.5f ? std::max(2, (int)ceil(20.0 / ms)) : 8);
        iters = (int)std::min(grown, 1L << 27);
    }
    if (rc == OVL_OK) {
        const double nc = precision == 0 ? 8.0 : 16.0;
        const double fmas = (double)blocks * 256.0 * timed_iters * 8.0 * nc;
        *gflops = 2.0 * fmas / (ms * 1e-3) * 1e-9;
    }
    cudaStreamDestroy(st);
    cudaFree(sink);
    return rc;
}
