// The optimisation loop around the state solve (Sec. 3.1): linear-hat density
// filter and its adjoint, the optimality-criteria (OC) update with a move limit and
// a bisection on the volume multiplier, and the compliance f^T u. All element-wise
// or stencil work on the element grid, HBM-bound.
#pragma once
#include <cuda_runtime.h>

namespace gf {

// Filter radius in cells: weights w(d) = r - |d| for |d| < r over integer offsets d.
__device__ __forceinline__ double hat_weight(int dx, int dy, int dz, double r)
{
    const double w = r - sqrt((double)(dx * dx + dy * dy + dz * dz));
    return w > 0.0 ? w : 0.0;
}

__device__ __forceinline__ double hat_row_sum(int ex, int ey, int ez, GridDims d, double r, int R)
{
    double W = 0.0;
    for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                const int jx = ex + dx, jy = ey + dy, jz = ez + dz;
                if (jx < 0 || jx >= d.nx || jy < 0 || jy >= d.ny || jz < 0 || jz >= d.nz) continue;
                W += hat_weight(dx, dy, dz, r);
            }
    return W;
}

// out_e = sum_e' w(e,e') x_e' / sum_e' w(e,e')       (filter)
// out_e' = sum_e w(e,e') g_e / W_e                   (adjoint: chain rule through the filter)
template <bool ADJOINT>
__global__ void __launch_bounds__(256)
hat_filter_kernel(const double* __restrict__ x, double* __restrict__ out, GridDims d, double r, int R)
{
    const long long ne = (long long)d.nx * d.ny * d.nz;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const int ex = (int)(e % d.nx);
    const long long t = e / d.nx;
    const int ey = (int)(t % d.ny), ez = (int)(t / d.ny);
    double s = 0.0, W = 0.0;
    for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                const int jx = ex + dx, jy = ey + dy, jz = ez + dz;
                if (jx < 0 || jx >= d.nx || jy < 0 || jy >= d.ny || jz < 0 || jz >= d.nz) continue;
                const double w = hat_weight(dx, dy, dz, r);
                if (w == 0.0) continue;
                const long long j = jx + (long long)d.nx * (jy + (long long)d.ny * jz);
                if (ADJOINT) {
                    s += w * x[j] / hat_row_sum(jx, jy, jz, d, r, R);
                } else {
                    s += w * x[j];
                    W += w;
                }
            }
    out[e] = ADJOINT ? s : s / W;
}

// ---- OC update with bisection on lambda (state in device memory) ----------------
struct OCState {
    double l1, l2, lmid;
    int done, iters;
};

__device__ __forceinline__ double oc_candidate(double x, double dc, double dv, double lam, double move)
{
    const double be = sqrt(fmax(-dc, 0.0) / (lam * dv));
    const double lo = fmax(0.0, x - move), hi = fmin(1.0, x + move);
    return fmin(fmax(x * be, lo), hi);
}

__global__ void oc_init_kernel(OCState* st)
{
    st->l1 = 0.0;
    st->l2 = 1e9;
    st->done = 0;
    st->iters = 0;
}

// One bisection iteration, part 1: stop test, lmid, and per-block partial sums of
// x_new(lmid) (deterministic partition).
__global__ void __launch_bounds__(256)
oc_partial_kernel(const double* __restrict__ x, const double* __restrict__ dc, const double* __restrict__ dv,
                  long long n, double move, double tol, OCState* __restrict__ st, double* __restrict__ partial)
{
    __shared__ double red[8];
    if (st->done) return;
    const double l1 = st->l1, l2 = st->l2;
    const double lmid = 0.5 * (l1 + l2);
    const long long chunk = (n + gridDim.x - 1) / gridDim.x;
    const long long r0 = (long long)blockIdx.x * chunk;
    const long long r1 = r0 + chunk < n ? r0 + chunk : n;
    double s = 0.0;
    for (long long e = r0 + threadIdx.x; e < r1; e += blockDim.x) s += oc_candidate(x[e], dc[e], dv[e], lmid, move);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += red[w];
        partial[blockIdx.x] = b;
    }
    (void)tol;
}

// part 2 (one thread): mean(x_new) vs volfrac moves the bracket; the stop test is
// the relative bracket width, checked before each iteration as in the oracle.
__global__ void oc_bisect_kernel(const double* __restrict__ partial, int nblocks, long long n, double volfrac,
                                 double tol, int max_iters, OCState* __restrict__ st)
{
    if (threadIdx.x != 0 || st->done) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partial[b];
    const double lmid = 0.5 * (st->l1 + st->l2);
    st->lmid = lmid;
    if (s / (double)n > volfrac) st->l1 = lmid;
    else st->l2 = lmid;
    st->iters += 1;
    if ((st->l2 - st->l1) / (st->l1 + st->l2) <= tol || st->iters >= max_iters) st->done = 1;
}

// x_new at the last evaluated lmid
__global__ void oc_apply_kernel(const double* __restrict__ x, const double* __restrict__ dc,
                                const double* __restrict__ dv, double* __restrict__ xnew, long long n, double move,
                                const OCState* __restrict__ st)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    xnew[e] = oc_candidate(x[e], dc[e], dv[e], st->lmid, move);
}

// partial dot products: partial[b] = sum over block b's chunk of a*b
__global__ void __launch_bounds__(256)
dot_partial_kernel(const double* __restrict__ a, const double* __restrict__ b, long long n,
                   double* __restrict__ partial)
{
    __shared__ double red[8];
    const long long chunk = (n + gridDim.x - 1) / gridDim.x;
    const long long r0 = (long long)blockIdx.x * chunk;
    const long long r1 = r0 + chunk < n ? r0 + chunk : n;
    double s = 0.0;
    for (long long e = r0 + threadIdx.x; e < r1; e += blockDim.x) s = fma(a[e], b[e], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        partial[blockIdx.x] = t;
    }
}

}  // namespace gf
