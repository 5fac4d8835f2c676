// Chebyshev smoothing for the V-cycle, the alternative to node-block Jacobi that
// Table "solver-config" names (degree and interval are readings):
//   degree nu1 (pre) / nu2 (post) Chebyshev semi-iteration on M = D_b^{-1} K over
//   [lambda_max / 30, 1.1 lambda_max], D_b the 3x3 node blocks;
//   step 0: d = (1/theta) D_b^{-1} r, x += d; step k: d = rho_k rho_{k-1} d +
//   (2 rho_k / delta) D_b^{-1} r, x += d (theta, delta: centre and half width of the
//   interval, rho_0 = delta / theta, rho_k = 1 / (2 theta / delta - rho_{k-1})).
// lambda_max of every smoothing level comes from 15 power iterations on M started
// from the all-ones vector on the free DOFs; the estimate and the step coefficients
// stay in device memory, so the captured solve graphs remain valid across floors.
#pragma once
#include <cuda_runtime.h>

namespace gf {

constexpr int CHEB_MAXDEG = 16, CHEB_POWER_ITERS = 15;

// K x at node n (x == nullptr reads as zero) and the node's 3x3 diagonal block
// (db: d00 d11 d22 d01 d02 d12). Fixed nodes (i == 0) of x read as zero.
template <typename T, typename ET>
__device__ __forceinline__ void cheb_gather(int i, int j, int k, const T* __restrict__ x,
                                            const ET* __restrict__ E, GridDims d, const K0Param<T>& K0,
                                            T (&a)[3], T (&db)[6])
{
    const int NX = d.nx + 1, NY = d.ny + 1;
#pragma unroll
    for (int q = 0; q < 3; ++q) a[q] = T(0);
#pragma unroll
    for (int q = 0; q < 6; ++q) db[q] = T(0);
#pragma unroll
    for (int oz = 0; oz < 2; ++oz)
#pragma unroll
        for (int oy = 0; oy < 2; ++oy)
#pragma unroll
            for (int ox = 0; ox < 2; ++ox) {
                const int ex = i - 1 + ox, ey = j - 1 + oy, ez = k - 1 + oz;
                if (ex < 0 || ex >= d.nx || ey < 0 || ey >= d.ny || ez < 0 || ez >= d.nz) continue;
                const T Ee = (T)E[ex + (long long)d.nx * (ey + (long long)d.ny * ez)];
                const int an = local_index(1 - ox, 1 - oy, 1 - oz);
                if (x != nullptr) {
                    T t0 = 0, t1 = 0, t2 = 0;
#pragma unroll
                    for (int bz = 0; bz < 2; ++bz)
#pragma unroll
                        for (int by = 0; by < 2; ++by)
#pragma unroll
                            for (int bx = 0; bx < 2; ++bx) {
                                const int bl = local_index(bx, by, bz);
                                const int ni = ex + bx;
                                if (ni == 0) continue;
                                const long long m = ni + (long long)NX * ((ey + by) + (long long)NY * (ez + bz));
                                const T u0 = x[3 * m + 0], u1 = x[3 * m + 1], u2 = x[3 * m + 2];
                                const T* r0 = &K0.k[(3 * an + 0) * 24 + 3 * bl];
                                const T* r1 = &K0.k[(3 * an + 1) * 24 + 3 * bl];
                                const T* r2 = &K0.k[(3 * an + 2) * 24 + 3 * bl];
                                t0 = fma(r0[0], u0, fma(r0[1], u1, fma(r0[2], u2, t0)));
                                t1 = fma(r1[0], u0, fma(r1[1], u1, fma(r1[2], u2, t1)));
                                t2 = fma(r2[0], u0, fma(r2[1], u1, fma(r2[2], u2, t2)));
                            }
                    a[0] = fma(Ee, t0, a[0]);
                    a[1] = fma(Ee, t1, a[1]);
                    a[2] = fma(Ee, t2, a[2]);
                }
                db[0] = fma(Ee, K0.k[(3 * an + 0) * 24 + 3 * an + 0], db[0]);
                db[1] = fma(Ee, K0.k[(3 * an + 1) * 24 + 3 * an + 1], db[1]);
                db[2] = fma(Ee, K0.k[(3 * an + 2) * 24 + 3 * an + 2], db[2]);
                db[3] = fma(Ee, K0.k[(3 * an + 0) * 24 + 3 * an + 1], db[3]);
                db[4] = fma(Ee, K0.k[(3 * an + 0) * 24 + 3 * an + 2], db[4]);
                db[5] = fma(Ee, K0.k[(3 * an + 1) * 24 + 3 * an + 2], db[5]);
            }
}

// z = D^{-1} r for the symmetric 3x3 block db, by its adjugate
template <typename T>
__device__ __forceinline__ void cheb_block_solve(const T (&db)[6], T r0, T r1, T r2, T (&z)[3])
{
    const T d00 = db[0], d11 = db[1], d22 = db[2], d01 = db[3], d02 = db[4], d12 = db[5];
    const T c00 = d11 * d22 - d12 * d12;
    const T c01 = d02 * d12 - d01 * d22;
    const T c02 = d01 * d12 - d02 * d11;
    const T c11 = d00 * d22 - d02 * d02;
    const T c12 = d01 * d02 - d00 * d12;
    const T c22 = d00 * d11 - d01 * d01;
    const T inv = T(1) / (d00 * c00 + d01 * c01 + d02 * c02);
    z[0] = inv * (c00 * r0 + c01 * r1 + c02 * r2);
    z[1] = inv * (c01 * r0 + c11 * r1 + c12 * r2);
    z[2] = inv * (c02 * r0 + c12 * r1 + c22 * r2);
}

// One Chebyshev step: r = b - K x (x == nullptr: x = 0), d = c1 d + c2 D^{-1} r
// (d not read when c1 == 0), xo = x + d. coef = {c1, c2} of this level and step.
template <typename T, typename ET>
__global__ void __launch_bounds__(256)
cheb_step_kernel(const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ xo, T* __restrict__ dv,
                 const ET* __restrict__ E, GridDims d, const __grid_constant__ K0Param<T> K0,
                 const double* __restrict__ coef, const int* __restrict__ halt)
{
    if (halt != nullptr && *halt != 0) return;
    const int NX = d.nx + 1, NY = d.ny + 1;
    const long long nn = (long long)NX * NY * (d.nz + 1);
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    int i, j, k;
    node_coords(n, NX, NY, i, j, k);
    if (i == 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xo[3 * n + c] = T(0);
            dv[3 * n + c] = T(0);
        }
        return;
    }
    T a[3], db[6], z[3];
    cheb_gather<T, ET>(i, j, k, x, E, d, K0, a, db);
    cheb_block_solve<T>(db, b[3 * n + 0] - a[0], b[3 * n + 1] - a[1], b[3 * n + 2] - a[2], z);
    const T c1 = (T)coef[0], c2 = (T)coef[1];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T dn = (coef[0] != 0.0) ? c1 * dv[3 * n + c] + c2 * z[c] : c2 * z[c];
        dv[3 * n + c] = dn;
        xo[3 * n + c] = (x != nullptr ? x[3 * n + c] : T(0)) + dn;
    }
}

// ---- lambda_max by the power method -------------------------------------------
// w = D^{-1} K v (fixed entries 0)
template <typename T, typename ET>
__global__ void __launch_bounds__(256)
dinvk_kernel(const T* __restrict__ v, T* __restrict__ w, const ET* __restrict__ E, GridDims d,
             const __grid_constant__ K0Param<T> K0)
{
    const int NX = d.nx + 1, NY = d.ny + 1;
    const long long nn = (long long)NX * NY * (d.nz + 1);
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    int i, j, k;
    node_coords(n, NX, NY, i, j, k);
    T a[3], db[6], z[3];
    if (i == 0) {
        w[3 * n + 0] = w[3 * n + 1] = w[3 * n + 2] = T(0);
        return;
    }
    cheb_gather<T, ET>(i, j, k, v, E, d, K0, a, db);
    cheb_block_solve<T>(db, a[0], a[1], a[2], z);
    w[3 * n + 0] = z[0];
    w[3 * n + 1] = z[1];
    w[3 * n + 2] = z[2];
}

// v = 1 on free DOFs, 0 on fixed (DOF q is fixed when (q/3) % NX == 0)
template <typename T>
__global__ void cheb_ones_kernel(T* __restrict__ v, long long n, int NX)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) v[q] = ((q / 3) % NX == 0) ? T(0) : T(1);
}

// out[0] = sum_q w_q^2 in FP64, one block, fixed order (deterministic)
template <typename T>
__global__ void __launch_bounds__(1024) cheb_sumsq_kernel(const T* __restrict__ w, long long n, double* __restrict__ out)
{
    __shared__ double red[32];
    double s = 0.0;
    for (long long q = threadIdx.x; q < n; q += 1024) {
        const double x = (double)w[q];
        s = fma(x, x, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < 32; ++q) t += red[q];
        out[0] = t;
    }
}

// v = w / sqrt(ss)
template <typename T>
__global__ void cheb_normalize_kernel(const T* __restrict__ w, T* __restrict__ v, long long n,
                                      const double* __restrict__ ss)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) v[q] = (T)((double)w[q] / sqrt(ss[0]));
}

// lambda = sqrt(ss) (the last iterate's ||M v||, ||v|| = 1) and the step coefficients
// {c1, c2} for k = 0 .. CHEB_MAXDEG-1 on [lambda/30, 1.1 lambda]
__global__ void cheb_coef_kernel(const double* __restrict__ ss, double* __restrict__ lam, double* __restrict__ coef)
{
    if (threadIdx.x != 0) return;
    const double l = sqrt(ss[0]);
    *lam = l;
    const double a = l / 30.0, b = 1.1 * l;
    const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
    coef[0] = 0.0;
    coef[1] = 1.0 / theta;
    double rho = 1.0 / sigma;
    for (int k = 1; k < CHEB_MAXDEG; ++k) {
        const double rn = 1.0 / (2.0 * sigma - rho);
        coef[2 * k + 0] = rn * rho;
        coef[2 * k + 1] = 2.0 * rn / delta;
        rho = rn;
    }
}

}  // namespace gf
