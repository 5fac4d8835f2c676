// Line-searched, rejectable coarse-grid correction (Table solver-config, "coarse
// correction"; the step and the acceptance test are this library's readings): with r
// the level's residual before the correction, c the prolongated coarse correction and
// q = K c,
//   alpha = (c.r) / (c.q)   (the energy-optimal step along c, computed from r; 1 for an
//                            exact Galerkin correction),  kept iff alpha >= theta,
// then x += alpha c (alpha = 0 when rejected). Minimising ||r - alpha q|| instead, or
// rejecting on the residual norm before post-smoothing, cripples this V-cycle (measured).
// Dot products in FP64 with a fixed order: per-block sums, then one thread sums them in
// block order.
#pragma once
#include <cuda_runtime.h>

namespace gf {

constexpr int LS_THREADS = 256;

// per-block (c.r, c.q) into partial[2 b + {0, 1}]
template <typename T>
__global__ void __launch_bounds__(LS_THREADS) ls_dots_kernel(const T* __restrict__ c, const T* __restrict__ r,
                                                             const T* __restrict__ q, long long n,
                                                             double* __restrict__ partial, const int* __restrict__ halt)
{
    if (halt != nullptr && *halt != 0) return;
    __shared__ double red[2][LS_THREADS / 32];
    double cr = 0.0, cq = 0.0;
    for (long long i = (long long)blockIdx.x * LS_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * LS_THREADS) {
        const double ci = (double)c[i];
        cr = fma(ci, (double)r[i], cr);
        cq = fma(ci, (double)q[i], cq);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cr += __shfl_down_sync(0xffffffffu, cr, o);
        cq += __shfl_down_sync(0xffffffffu, cq, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][warp] = cr;
        red[1][warp] = cq;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double s = 0.0;
        for (int w = 0; w < LS_THREADS / 32; ++w) s += red[threadIdx.x][w];
        partial[2 * blockIdx.x + threadIdx.x] = s;
    }
}

__global__ void ls_finish_kernel(const double* __restrict__ partial, int nb, double theta, double* __restrict__ alpha,
                                 const int* __restrict__ halt)
{
    if (threadIdx.x != 0) return;
    if (halt != nullptr && *halt != 0) return;
    double cr = 0.0, cq = 0.0;
    for (int b = 0; b < nb; ++b) {
        cr += partial[2 * b + 0];
        cq += partial[2 * b + 1];
    }
    const double a = (cq > 0.0) ? cr / cq : 0.0;
    *alpha = (cq > 0.0 && a >= theta) ? a : 0.0;
}

template <typename T>
__global__ void ls_axpy_kernel(T* __restrict__ x, const T* __restrict__ c, long long n, const double* __restrict__ alpha,
                               const int* __restrict__ halt)
{
    if (halt != nullptr && *halt != 0) return;
    const T a = (T)(*alpha);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] += a * c[i];
}

}  // namespace gf
