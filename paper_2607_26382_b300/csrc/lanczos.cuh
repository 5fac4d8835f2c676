// Extreme eigenvalues for the floor-conditioning diagnostic (Sec. 4.1.3): Lanczos on
// the free-DOF operator K (matrix-free FP64) for lambda_max, and on its dense FP64
// inverse for 1 / lambda_min. Every vector is short (one reduced grid, <= 8192 DOFs),
// so a step's vector work runs in one block with a fixed reduction order.
#pragma once
#include <cuda_runtime.h>

namespace gf {

constexpr int LZ_THREADS = 1024, LZ_MAX = 512;   // threads of the step kernel, Lanczos steps

struct LzState {
    double alpha[LZ_MAX], beta[LZ_MAX + 1];   // T = tridiag(beta, alpha, beta); beta[0] = 0
    double lo, hi;                            // extreme eigenvalues of T (lanczos_tridiag_kernel)
};

// fixed-order block sum of per-thread values
__device__ __forceinline__ double lz_block_sum(double v, double* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < LZ_THREADS / 32; ++w) s += red[w];
    return s;
}

// v0 = ones on the free DOFs (DOF q fixed when (q/3) % NX == 0), normalised; vprev = 0
__global__ void __launch_bounds__(LZ_THREADS) lanczos_start_kernel(double* __restrict__ v, double* __restrict__ vprev,
                                                                   long long n, int NX, LzState* __restrict__ st)
{
    __shared__ double red[LZ_THREADS / 32];
    double s = 0.0;
    for (long long q = threadIdx.x; q < n; q += LZ_THREADS) {
        const double x = ((q / 3) % NX == 0) ? 0.0 : 1.0;
        v[q] = x;
        vprev[q] = 0.0;
        s += x * x;
    }
    const double inv = 1.0 / sqrt(lz_block_sum(s, red));
    for (long long q = threadIdx.x; q < n; q += LZ_THREADS) v[q] *= inv;
    if (threadIdx.x == 0) st->beta[0] = 0.0;
}

// Step j with w = Op v_j:  alpha_j = w.v_j,  w -= alpha_j v_j + beta_j v_{j-1}, then the
// same projection once more against v_j and v_{j-1} (local re-orthogonalisation),
// beta_{j+1} = ||w||, and the new vector w / beta_{j+1} written over v_{j-1} (the caller
// swaps the two buffers).
__global__ void __launch_bounds__(LZ_THREADS) lanczos_step_kernel(double* __restrict__ w, const double* __restrict__ v,
                                                                  double* __restrict__ vprev, long long n, int j,
                                                                  LzState* __restrict__ st)
{
    __shared__ double red[LZ_THREADS / 32];
    const double bj = st->beta[j];
    double s = 0.0;
    for (long long q = threadIdx.x; q < n; q += LZ_THREADS) s = fma(w[q], v[q], s);
    const double a = lz_block_sum(s, red);
    double s1 = 0.0, s2 = 0.0;
    for (long long q = threadIdx.x; q < n; q += LZ_THREADS) {
        const double x = w[q] - a * v[q] - bj * vprev[q];
        w[q] = x;
        s1 = fma(x, v[q], s1);
        s2 = fma(x, vprev[q], s2);
    }
    const double c1 = lz_block_sum(s1, red);
    const double c2 = lz_block_sum(s2, red);
    double s3 = 0.0;
    for (long long q = threadIdx.x; q < n; q += LZ_THREADS) {
        const double x = w[q] - c1 * v[q] - c2 * vprev[q];
        w[q] = x;
        s3 = fma(x, x, s3);
    }
    const double b = sqrt(lz_block_sum(s3, red));
    const double inv = b > 0.0 ? 1.0 / b : 0.0;
    for (long long q = threadIdx.x; q < n; q += LZ_THREADS) vprev[q] = w[q] * inv;
    if (threadIdx.x == 0) {
        st->alpha[j] = a + c1;
        st->beta[j + 1] = b;
    }
}

// number of eigenvalues of T_k below x (Sturm sequence of the LDL^T pivots)
__device__ int lz_sturm_count(const LzState* st, int k, double x)
{
    int c = 0;
    double d = 1.0;
    for (int i = 0; i < k; ++i) {
        const double b2 = (i > 0) ? st->beta[i] * st->beta[i] : 0.0;
        d = (st->alpha[i] - x) - (i > 0 ? b2 / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++c;
    }
    return c;
}

// lowest and highest eigenvalue of T_k by bisection inside its Gershgorin interval
__global__ void lanczos_tridiag_kernel(LzState* __restrict__ st, int k)
{
    if (threadIdx.x != 0) return;
    double glo = 1e300, ghi = -1e300;
    for (int i = 0; i < k; ++i) {
        const double r = (i > 0 ? fabs(st->beta[i]) : 0.0) + (i + 1 < k ? fabs(st->beta[i + 1]) : 0.0);
        glo = fmin(glo, st->alpha[i] - r);
        ghi = fmax(ghi, st->alpha[i] + r);
    }
    for (int which = 0; which < 2; ++which) {
        double a = glo, b = ghi;   // which = 0: smallest (count(x) >= 1), 1: largest (count(x) >= k)
        for (int it = 0; it < 200 && b - a > 1e-15 * fmax(fabs(a), fabs(b)); ++it) {
            const double m = 0.5 * (a + b);
            const bool right = which == 0 ? (lz_sturm_count(st, k, m) >= 1) : (lz_sturm_count(st, k, m) >= k);
            if (right) b = m;
            else a = m;
        }
        if (which == 0) st->lo = 0.5 * (a + b);
        else st->hi = 0.5 * (a + b);
    }
}

}  // namespace gf
