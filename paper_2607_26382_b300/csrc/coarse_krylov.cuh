// The coarse-level inner Krylov solve (Table solver-config: inner Krylov steps on the
// coarse level) in one CTA: k steps of FGMRES(k) from x = 0 on the coarsest level's
// matrix-free operator, preconditioned by its 3x3 node-block Jacobi operator. The
// coarsest level holds at most a few thousand DOFs, so the multi-launch inner solve of
// finecorr.cuh spends its time in ~10 launches per step; here the steps, the
// Gram-Schmidt passes and the Givens update run in one launch, separated by barriers.
//
// The basis V and the preconditioned vectors Z, (2k + 1) n values, live in the CTA's
// shared memory (the caller uses this kernel only when they fit; a single SM waiting on
// L2 round trips was latency-bound). Dots: warp q takes basis vector q (lanes over rows,
// then a fixed shuffle tree), accumulated in the vectors' precision per lane (as in
// finecorr.cuh) and stored in FP64. Stop rules are the inner solve's: a zero rotated
// pivot drops the step, h_{j+1,j} <= 1e-14 ||K z_j|| or a zero projected residual ends
// the solve.
#pragma once
#include <cuda_runtime.h>

namespace gf {

constexpr int CK_THREADS = 1024, CK_WARPS = CK_THREADS / 32;
constexpr int CK_SMEM_MAX = 200 * 1024;   // bytes of V and Z the one-CTA solve takes

template <typename T>
using CkAcc = typename std::conditional<sizeof(T) == sizeof(float), float, double>::type;

// y_n = (K u)_n, or (diag) the node block D_n, of node n of the level (fixed nodes: 0 / I)
template <typename T>
__device__ __forceinline__ void ck_node(long long n, const T* u, const T* __restrict__ E, GridDims d,
                                        const K0Param<T>& K0, T (&y)[3], T (&D)[6], bool diag)
{
    const int NX = d.nx + 1, NY = d.ny + 1;
    int i, j, k;
    node_coords(n, NX, NY, i, j, k);
    y[0] = y[1] = y[2] = T(0);
    for (int q = 0; q < 6; ++q) D[q] = T(0);
    if (i == 0) return;
    for (int oz = 0; oz < 2; ++oz)
        for (int oy = 0; oy < 2; ++oy)
            for (int ox = 0; ox < 2; ++ox) {
                const int ex = i - 1 + ox, ey = j - 1 + oy, ez = k - 1 + oz;
                if (ex < 0 || ex >= d.nx || ey < 0 || ey >= d.ny || ez < 0 || ez >= d.nz) continue;
                const T Ee = E[ex + (long long)d.nx * (ey + (long long)d.ny * ez)];
                const int a = local_index(1 - ox, 1 - oy, 1 - oz);
                if (diag) {
                    D[0] = fma(Ee, K0.k[(3 * a + 0) * 24 + 3 * a + 0], D[0]);
                    D[1] = fma(Ee, K0.k[(3 * a + 1) * 24 + 3 * a + 1], D[1]);
                    D[2] = fma(Ee, K0.k[(3 * a + 2) * 24 + 3 * a + 2], D[2]);
                    D[3] = fma(Ee, K0.k[(3 * a + 0) * 24 + 3 * a + 1], D[3]);
                    D[4] = fma(Ee, K0.k[(3 * a + 0) * 24 + 3 * a + 2], D[4]);
                    D[5] = fma(Ee, K0.k[(3 * a + 1) * 24 + 3 * a + 2], D[5]);
                    continue;
                }
                T t0 = 0, t1 = 0, t2 = 0;
                for (int bz = 0; bz < 2; ++bz)
                    for (int by = 0; by < 2; ++by)
                        for (int bx = 0; bx < 2; ++bx) {
                            if (ex + bx == 0) continue;   // fixed node: reads as 0
                            const int bl = local_index(bx, by, bz);
                            const long long m = (ex + bx) + (long long)NX * ((ey + by) + (long long)NY * (ez + bz));
                            const T u0 = u[3 * m], u1 = u[3 * m + 1], u2 = u[3 * m + 2];
                            const T* r0 = &K0.k[(3 * a + 0) * 24 + 3 * bl];
                            const T* r1 = &K0.k[(3 * a + 1) * 24 + 3 * bl];
                            const T* r2 = &K0.k[(3 * a + 2) * 24 + 3 * bl];
                            t0 = fma(r0[0], u0, fma(r0[1], u1, fma(r0[2], u2, t0)));
                            t1 = fma(r1[0], u0, fma(r1[1], u1, fma(r1[2], u2, t1)));
                            t2 = fma(r2[0], u0, fma(r2[1], u1, fma(r2[2], u2, t2)));
                        }
                y[0] = fma(Ee, t0, y[0]);
                y[1] = fma(Ee, t1, y[1]);
                y[2] = fma(Ee, t2, y[2]);
            }
}

// out[q] = dot(Vs + q ld, w) for q < cnt (warp q, lanes over rows), FP64 results
template <typename T>
__device__ __forceinline__ void ck_dots(const T* Vs, long long ld, const T* w, long long n, int cnt, double* out)
{
    using A = CkAcc<T>;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = warp; q < cnt; q += CK_WARPS) {
        const T* v = Vs + q * ld;
        A s = A(0);
        for (long long r = lane; r < n; r += 32) s = fma((A)v[r], (A)w[r], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) out[q] = (double)s;
    }
}

template <typename T>
__global__ void __launch_bounds__(CK_THREADS)
coarse_fgmres_kernel(const T* b, T* x, const T* __restrict__ E, GridDims d, const __grid_constant__ K0Param<T> K0,
                     int steps, const int* __restrict__ halt)
{
    using A = CkAcc<T>;
    extern __shared__ __align__(16) unsigned char ck_smem[];
    __shared__ double H[(FC_MAX + 1) * FC_MAX], g[FC_MAX + 1], cs[FC_MAX], sn[FC_MAX], y[FC_MAX];
    __shared__ double h1[FC_MAX + 2], h2[FC_MAX + 1];
    __shared__ double s_beta, s_hn;
    __shared__ int s_stop, s_J;
    if (halt != nullptr && *halt != 0) return;
    const long long nodes = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1), n = 3 * nodes, ld = n;
    const int tid = threadIdx.x;
    T* V = reinterpret_cast<T*>(ck_smem);     // (steps + 1) x n
    T* Z = V + (long long)(steps + 1) * n;    // steps x n
    // beta = ||b||, V_0 = b / beta
    ck_dots<T>(b, 0, b, n, 1, h1);
    __syncthreads();
    if (tid == 0) {
        s_beta = sqrt(h1[0]);
        g[0] = s_beta;
        s_J = 0;
        s_stop = !(s_beta > 0.0);
    }
    __syncthreads();
    if (s_stop) return;                 // b = 0: x stays 0
    {
        const A inv = (A)(1.0 / s_beta);
        for (long long r = tid; r < n; r += CK_THREADS) V[r] = (T)((A)b[r] * inv);
    }
    __syncthreads();
    for (int j = 0; j < steps; ++j) {
        T* vj = V + j * ld;
        T* zj = Z + j * ld;
        T* w = V + (j + 1) * ld;
        for (long long nd = tid; nd < nodes; nd += CK_THREADS) {   // z_j = D^{-1} v_j
            T yv[3], D[6];
            ck_node<T>(nd, vj, E, d, K0, yv, D, true);
            const T r0 = vj[3 * nd], r1 = vj[3 * nd + 1], r2 = vj[3 * nd + 2];
            if ((nd % (d.nx + 1)) == 0) {
                zj[3 * nd] = zj[3 * nd + 1] = zj[3 * nd + 2] = T(0);
            } else {
                const T zero[3] = {T(0), T(0), T(0)};
                node_block_update<T, T>(D[0], D[1], D[2], D[3], D[4], D[5], r0, r1, r2, zero, zj + 3 * nd, T(1));
            }
        }
        __syncthreads();
        for (long long nd = tid; nd < nodes; nd += CK_THREADS) {   // w = K z_j
            T yv[3], D[6];
            ck_node<T>(nd, zj, E, d, K0, yv, D, false);
            w[3 * nd] = yv[0];
            w[3 * nd + 1] = yv[1];
            w[3 * nd + 2] = yv[2];
        }
        __syncthreads();
        ck_dots<T>(V, ld, w, n, j + 1, h1);          // h1 = V^T w
        ck_dots<T>(w, 0, w, n, 1, h1 + FC_MAX + 1);   // ||w||^2 before orthogonalisation
        __syncthreads();
        for (int pass = 0; pass < 2; ++pass) {       // w -= V h, twice (CGS2)
            const double* h = pass == 0 ? h1 : h2;
            for (long long r = tid; r < n; r += CK_THREADS) {
                A s = A(0);
                for (int i = 0; i <= j; ++i) s = fma((A)h[i], (A)V[i * ld + r], s);
                w[r] = (T)((A)w[r] - s);
            }
            __syncthreads();
            if (pass == 0) {
                ck_dots<T>(V, ld, w, n, j + 1, h2);
                __syncthreads();
            }
        }
        ck_dots<T>(w, 0, w, n, 1, &s_hn);
        __syncthreads();
        if (tid == 0) {
            const double hn = sqrt(s_hn);
            const int ldh = FC_MAX + 1;
            double* col = H + j * ldh;
            for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
            col[j + 1] = hn;
            for (int i = 0; i < j; ++i) {
                const double a = col[i], bb = col[i + 1];
                col[i] = cs[i] * a + sn[i] * bb;
                col[i + 1] = -sn[i] * a + cs[i] * bb;
            }
            const double a = col[j], bb = col[j + 1];
            const double rho = hypot(a, bb);
            if (rho == 0.0) {
                s_stop = 1;   // breakdown: the step is dropped
            } else {
                cs[j] = a / rho;
                sn[j] = bb / rho;
                col[j] = rho;
                col[j + 1] = 0.0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                s_J = j + 1;
                s_hn = hn;
                if (g[j + 1] == 0.0 || j + 1 >= steps || hn <= 1e-14 * sqrt(h1[FC_MAX + 1])) s_stop = 1;
            }
        }
        __syncthreads();
        if (s_stop) break;
        {
            const A inv = (A)(1.0 / s_hn);
            for (long long r = tid; r < n; r += CK_THREADS) w[r] = (T)((A)w[r] * inv);
        }
        __syncthreads();
    }
    if (tid == 0) {   // y = R^{-1} g over the kept columns
        const int ldh = FC_MAX + 1, J = s_J;
        for (int i = J - 1; i >= 0; --i) {
            double s = g[i];
            for (int c = i + 1; c < J; ++c) s -= H[c * ldh + i] * y[c];
            y[i] = s / H[i * ldh + i];
        }
    }
    __syncthreads();
    const int J = s_J;
    for (long long r = tid; r < n; r += CK_THREADS) {   // x = Z y
        A s = A(0);
        for (int i = 0; i < J; ++i) s = fma((A)y[i], (A)Z[i * ld + r], s);
        x[r] = (T)s;
    }
}

}  // namespace gf
