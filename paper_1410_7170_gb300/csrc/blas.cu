// BLAS-1 kernels on flat arrays: deterministic reductions (norms, complex dots,
// multi-dots for Gram-Schmidt), axpy variants and precision conversion. All are
// HBM-streaming; reductions accumulate in FP64 in a fixed order.
#include "internal.h"
#include "reduce.cuh"

namespace ovl {

namespace {

struct StoreFin1 {
    double *res;
    __device__ void operator()(const double *s) const { res[0] = s[0]; }
};
struct StoreFin2 {
    double *res;
    __device__ void operator()(const double *s) const { res[0] = s[0]; res[1] = s[1]; }
};

// Per-thread partial sums are kept in the vector's own precision T (a grid-stride
// thread sees only a few elements), and so are the warp sums; warps, blocks and the grid
// are summed in FP64.
template <typename T>
__global__ void k_norm2(const T *__restrict__ x, long n, RedScratch rs, double *res) {
    T a = 0;
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
        a += x[k] * x[k];
    T v[1] = {a};
    grid_reduce<1>(v, rs, StoreFin1{res});
}

// <x, y> = sum conj(x) y over complex numbers stored as (re, im) pairs
template <typename T>
__global__ void k_cdot(const T *__restrict__ x, const T *__restrict__ y, long nc, RedScratch rs, double *res) {
    T a = 0, b = 0;
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < nc; k += (long)gridDim.x * blockDim.x) {
        const T xr = x[2 * k], xi = x[2 * k + 1];
        const T yr = y[2 * k], yi = y[2 * k + 1];
        a += xr * yr + xi * yi;
        b += xr * yi - xi * yr;
    }
    T v[2] = {a, b};
    grid_reduce<2>(v, rs, StoreFin2{res});
}

__global__ void k_axpby(double a, const double *__restrict__ x, double b, double *__restrict__ y, long n) {
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
        y[k] = a * x[k] + b * y[k];
}
__global__ void k_axpby_f(float a, const float *__restrict__ x, float b, float *__restrict__ y, long n) {
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
        y[k] = a * x[k] + b * y[k];
}
__global__ void k_caxpy(double ar, double ai, const double *__restrict__ x, double *__restrict__ y, long nc) {
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < nc; k += (long)gridDim.x * blockDim.x) {
        const double xr = x[2 * k], xi = x[2 * k + 1];
        y[2 * k] += ar * xr - ai * xi;
        y[2 * k + 1] += ar * xi + ai * xr;
    }
}

// Multi-dot: blockIdx.y = vector index; partials[k][blockIdx.x] (complex). Rows y >= m use
// w itself, so an extra row gives (||w||^2, 0) in the same pass.
template <typename T>
__global__ void k_multidot_part(const T *__restrict__ base, long stride, int m, const T *__restrict__ w, long nc,
                                double *partials) {
    const T *v = (int)blockIdx.y < m ? base + (long)blockIdx.y * stride : w;
    T a = 0, b = 0;
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < nc; k += (long)gridDim.x * blockDim.x) {
        const T vr = v[2 * k], vi = v[2 * k + 1];
        const T wr = w[2 * k], wi = w[2 * k + 1];
        a += vr * wr + vi * wi;
        b += vr * wi - vi * wr;
    }
    const T t[2] = {a, b};
    double s[2];
    block_sum<2>(t, s);
    if (threadIdx.x == 0) {
        partials[((long)blockIdx.y * gridDim.x + blockIdx.x) * 2] = s[0];
        partials[((long)blockIdx.y * gridDim.x + blockIdx.x) * 2 + 1] = s[1];
    }
}
__global__ void k_multidot_sum(const double *partials, int nb, double *out) {
    double s[2] = {0.0, 0.0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        s[0] += partials[((long)blockIdx.x * nb + b) * 2];
        s[1] += partials[((long)blockIdx.x * nb + b) * 2 + 1];
    }
    block_sum<2>(s);
    if (threadIdx.x == 0) {
        out[2 * blockIdx.x] = s[0];
        out[2 * blockIdx.x + 1] = s[1];
    }
}

// out = scale (w - sum_j h_j v_j) with h the complex dot products of a multi-dot (device
// memory, FP64): the Gram-Schmidt update and normalisation of an Arnoldi step in one pass.
template <typename T>
__global__ void k_orth_scale(const T *__restrict__ base, long stride, int m, const double *__restrict__ h,
                             double scale, const T *__restrict__ w, T *__restrict__ out, long nc) {
    __shared__ T cs[2 * 128];
    for (int k = threadIdx.x; k < 2 * m; k += blockDim.x) cs[k] = (T)(-h[k]);
    __syncthreads();
    const T sc = (T)scale;
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < nc; k += (long)gridDim.x * blockDim.x) {
        T ar = w[2 * k], ai = w[2 * k + 1];
        for (int j = 0; j < m; j++) {
            const T *v = base + (long)j * stride;
            const T vr = v[2 * k], vi = v[2 * k + 1];
            ar += cs[2 * j] * vr - cs[2 * j + 1] * vi;
            ai += cs[2 * j] * vi + cs[2 * j + 1] * vr;
        }
        out[2 * k] = sc * ar;
        out[2 * k + 1] = sc * ai;
    }
}

template <typename T>
__global__ void k_multiaxpy(const T *__restrict__ base, long stride, int m, const double *__restrict__ c,
                            T *__restrict__ w, long nc) {
    __shared__ T cs[2 * 128];   // coefficients in the vectors' precision
    for (int k = threadIdx.x; k < 2 * m; k += blockDim.x) cs[k] = (T)c[k];
    __syncthreads();
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < nc; k += (long)gridDim.x * blockDim.x) {
        T ar = w[2 * k], ai = w[2 * k + 1];
        for (int j = 0; j < m; j++) {
            const T *v = base + (long)j * stride;
            const T vr = v[2 * k], vi = v[2 * k + 1];
            ar += cs[2 * j] * vr - cs[2 * j + 1] * vi;
            ai += cs[2 * j] * vi + cs[2 * j + 1] * vr;
        }
        w[2 * k] = ar;
        w[2 * k + 1] = ai;
    }
}

__global__ void k_d2f(const double *__restrict__ x, float *__restrict__ y, long n) {
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
        y[k] = (float)x[k];
}
__global__ void k_f2d(const float *__restrict__ x, double *__restrict__ y, long n) {
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
        y[k] = (double)x[k];
}
__global__ void k_nonfinite(const double *__restrict__ x, long n, int *flag) {
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
        if (!isfinite(x[k])) atomicExch(flag, 1);
}

inline int stream_grid(long n) {
    long b = (n + kBlock - 1) / kBlock;
    const long cap = 152L * 16;   // enough resident blocks to fill 152 SMs several times
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t dev_norm2(const double *x, long n, double *res, RedScratch rs, cudaStream_t st) {
    k_norm2<double><<<red_grid(n), kBlock, 0, st>>>(x, n, rs, res);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t dev_norm2_f(const float *x, long n, double *res, RedScratch rs, cudaStream_t st) {
    k_norm2<float><<<red_grid(n), kBlock, 0, st>>>(x, n, rs, res);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t dev_cdot(const double *x, const double *y, long n, double *res, RedScratch rs, cudaStream_t st) {
    k_cdot<double><<<red_grid(n / 2), kBlock, 0, st>>>(x, y, n / 2, rs, res);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t dev_cdot_f(const float *x, const float *y, long n, double *res, RedScratch rs, cudaStream_t st) {
    k_cdot<float><<<red_grid(n / 2), kBlock, 0, st>>>(x, y, n / 2, rs, res);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t dev_axpby(double a, const double *x, double b, double *y, long n, cudaStream_t st) {
    k_axpby<<<stream_grid(n), kBlock, 0, st>>>(a, x, b, y, n);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t dev_axpby_f(float a, const float *x, float b, float *y, long n, cudaStream_t st) {
    k_axpby_f<<<stream_grid(n), kBlock, 0, st>>>(a, x, b, y, n);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t dev_caxpy(double ar, double ai, const double *x, double *y, long n, cudaStream_t st) {
    k_caxpy<<<stream_grid(n / 2), kBlock, 0, st>>>(ar, ai, x, y, n / 2);
    count_launches(1);
    return cudaGetLastError();
}

constexpr int kMdBlocks = 256;   // partial blocks per vector of a multi-dot

cudaError_t dev_multidot(const double *base, long stride, int m, const double *w, long n, double *out,
                         double *partials, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    int gx = (int)((n / 2 + kBlock - 1) / kBlock);
    if (gx > kMdBlocks) gx = kMdBlocks;
    if (gx < 1) gx = 1;
    k_multidot_part<double><<<dim3(gx, m), kBlock, 0, st>>>(base, stride, m, w, n / 2, partials);
    k_multidot_sum<<<m, kBlock, 0, st>>>(partials, gx, out);
    count_launches(2);
    return cudaGetLastError();
}
cudaError_t dev_multidot_f(const float *base, long stride, int m, const float *w, long n, double *out,
                           double *partials, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    int gx = (int)((n / 2 + kBlock - 1) / kBlock);
    if (gx > kMdBlocks) gx = kMdBlocks;
    if (gx < 1) gx = 1;
    k_multidot_part<float><<<dim3(gx, m), kBlock, 0, st>>>(base, stride, m, w, n / 2, partials);
    k_multidot_sum<<<m, kBlock, 0, st>>>(partials, gx, out);
    count_launches(2);
    return cudaGetLastError();
}
cudaError_t dev_multidot_norm_f(const float *base, long stride, int m, const float *w, long n, double *out,
                                double *partials, cudaStream_t st) {
    int gx = (int)((n / 2 + kBlock - 1) / kBlock);
    if (gx > kMdBlocks) gx = kMdBlocks;
    if (gx < 1) gx = 1;
    k_multidot_part<float><<<dim3(gx, m + 1), kBlock, 0, st>>>(base, stride, m, w, n / 2, partials);
    k_multidot_sum<<<m + 1, kBlock, 0, st>>>(partials, gx, out);
    count_launches(2);
    return cudaGetLastError();
}
cudaError_t dev_orth_scale_f(const float *base, long stride, int m, const double *h, double scale, const float *w,
                             float *out, long n, cudaStream_t st) {
    k_orth_scale<float><<<stream_grid(n / 2), kBlock, 0, st>>>(base, stride, m, h, scale, w, out, n / 2);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t dev_multiaxpy(const double *base, long stride, int m, const double *c, double *w, long n,
                          cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    k_multiaxpy<double><<<stream_grid(n / 2), kBlock, 0, st>>>(base, stride, m, c, w, n / 2);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t dev_multiaxpy_f(const float *base, long stride, int m, const double *c, float *w, long n,
                            cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    k_multiaxpy<float><<<stream_grid(n / 2), kBlock, 0, st>>>(base, stride, m, c, w, n / 2);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t dev_d2f(const double *x, float *y, long n, cudaStream_t st) {
    k_d2f<<<stream_grid(n), kBlock, 0, st>>>(x, y, n);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t dev_f2d(const float *x, double *y, long n, cudaStream_t st) {
    k_f2d<<<stream_grid(n), kBlock, 0, st>>>(x, y, n);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t dev_nonfinite(const double *x, long n, int *flag, cudaStream_t st) {
    k_nonfinite<<<stream_grid(n), kBlock, 0, st>>>(x, n, flag);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace ovl
