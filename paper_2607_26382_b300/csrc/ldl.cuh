// The coarsest level's dense FP64 inverse from a banded LDL^T factorisation.
//
// The coarsest operator restricted to the free DOFs, A (m x m, symmetric positive
// definite), has no non-zero with |p - q| > b (the band of the compact order, coarse_axes).
// Its inverse Z = A^-1 is applied as a dense GEMV in every V-cycle (the exact coarsest
// solve of the V-cycle, Sec. 3.5 / Table solver-config), so Z is formed explicitly, in
// FP64, in two passes over blocks of LDL_C pivots:
//
//  1. A = L D L^T, right-looking by blocks J = [j0, j1): the diagonal block is factored
//     in place (ldl_diag_kernel), the rows below it in the band get L_rJ from a forward
//     substitution with L_JJ (ldl_panel_kernel), and the band below the block loses
//     L_rJ D_J L_qJ^T (ldl_update_kernel). The factor stays inside the band: about
//     m b^2 / 2 FMAs.
//  2. From L^T Z = D^-1 L^-1 (an upper-triangular left side against a lower-triangular
//     right side), block by block from the last: with K the pivots after J and
//     X_KJ = Z_KK L_KJ,
//        Z_KJ = -X_KJ L_JJ^-1                               (ldl_inv_rows_kernel)
//        Z_JJ = L_JJ^-T (D_J^-1 + L_KJ^T X_KJ) L_JJ^-1       (ldl_inv_diag_kernel: the
//                                                            right factor by rows;
//                                                            ldl_inv_diag2_kernel: the
//                                                            left one by columns)
//     L_KJ is non-zero only in the b rows after J, so the products run over b terms:
//     about m^2 b / 2 FMAs for the whole dense inverse, against the m^3 / 2 of a sweep.
//
// Every triangular solve with L_JJ is column oriented inside one warp: lane t owns
// unknown t, and once unknown s is final it is broadcast with a shuffle and every lane
// still open takes one FMA, so a solve costs LDL_C FP64 instructions per warp. The order
// of every sum is fixed, so Z does not depend on the launch shape. Z is written in full
// (both triangles) into an m x m row-major buffer; sym_expand maps it to the n x n
// operator of all DOFs.
#pragma once
#include <cuda_runtime.h>

namespace gf {

constexpr int LDL_C = 32;   // pivots per block (one warp lane per pivot)
constexpr int LDL_WARPS = 4;

// Asynchronous 8-byte global -> shared copies (cp.async): a thread issues all of its
// staging copies before any completes, then waits for them (cp.async.wait_all) ahead of
// the CTA barrier, so the staging costs one memory round trip instead of one per element.
__device__ __forceinline__ void ldl_cp8(double* smem, const double* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void ldl_cp_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// A dot product over n terms of (a[k], b[k * bs]) in four interleaved partial sums, added
// as (s0 + s1) + (s2 + s3): four independent FMA chains instead of one.
__device__ __forceinline__ double ldl_dot4(const double* __restrict__ a, const double* __restrict__ b, int bs, int n)
{
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int k = 0;
    for (; k + 4 <= n; k += 4) {
        s0 = fma(a[k], b[(long long)k * bs], s0);
        s1 = fma(a[k + 1], b[(long long)(k + 1) * bs], s1);
        s2 = fma(a[k + 2], b[(long long)(k + 2) * bs], s2);
        s3 = fma(a[k + 3], b[(long long)(k + 3) * bs], s3);
    }
    if (k < n) s0 = fma(a[k], b[(long long)k * bs], s0);
    if (k + 1 < n) s1 = fma(a[k + 1], b[(long long)(k + 1) * bs], s1);
    if (k + 2 < n) s2 = fma(a[k + 2], b[(long long)(k + 2) * bs], s2);
    return (s0 + s1) + (s2 + s3);
}

// 1 / d in FP64 by Newton-Raphson on x -> x (2 - d x) from the FP32 reciprocal of d: two
// steps take its ~2^-23 relative error to FP64 rounding (each step squares it). Outside
// the FP32 range of 1 / d the FP64 division is used.
__device__ __forceinline__ double ldl_recip(double d)
{
    const double a = fabs(d);
    if (!(a > 1e-30 && a < 1e30)) return 1.0 / d;
    double x = (double)__frcp_rn((float)d);
    double e = fma(-d, x, 1.0);
    x = fma(x, e, x);
    e = fma(-d, x, 1.0);
    return fma(x, e, x);
}

// Rows of the band below block J: [j1, ldl_band_end) (row r can couple to a pivot of J
// only if r < j1 + b).
__host__ __device__ inline int ldl_band_end(int m, int j1, int b)
{
    return min(m, j1 + b);
}

// Step s of the factor: block J = [j0, j0 + c), band rows [j0 + c, r1); false past the
// last block.
__host__ __device__ inline bool ldl_factor_step(int m, int b, int s, int& j0, int& c, int& r1)
{
    j0 = LDL_C * s;
    if (j0 >= m) return false;
    c = min(LDL_C, m - j0);
    r1 = ldl_band_end(m, j0 + c, b);
    return true;
}

// Step s of the inverse: the blocks from the last one back; band rows [j0 + c, kend).
__host__ __device__ inline bool ldl_inverse_step(int m, int b, int s, int& j0, int& c, int& kend)
{
    const int blk = (m + LDL_C - 1) / LDL_C - 1 - s;
    if (blk < 0) return false;
    j0 = LDL_C * blk;
    c = min(LDL_C, m - j0);
    kend = ldl_band_end(m, j0 + c, b);
    return true;
}

// One coarsest matrix and its buffers: M (m x m: A, then its factor), Z (m x m: the
// inverse), dinv (m), Xs (m x LDL_C), Qs (LDL_C x LDL_C); b the band.
struct LdlState {
    double* M;
    double* Z;
    double* dinv;
    double* Xs;
    double* Qs;
    int m, b;
};

// 1a. Factor the diagonal block J = [j0, j0 + c) of M (its lower triangle already holds
// A_JJ minus the earlier blocks' updates): afterwards M[j0+r][j0+t] = L_rt (r > t) and
// M[j0+t][j0+t] = d_t; dinv[j0+t] = 1 / d_t. One CTA of 512 threads, one barrier per
// pivot: the trailing entries are updated from pivot t's unscaled column (S keeps it; L is
// scaled once at the end), and the thread that finishes the next pivot forms its
// reciprocal.
__device__ __forceinline__ void ldl_diag_body(double* __restrict__ M, int m, int j0, int c, double* __restrict__ dinv)
{
    __shared__ double S[LDL_C][LDL_C + 1];
    __shared__ double ip[LDL_C];
    const int tid = threadIdx.x;
    for (int e = tid; e < c * c; e += blockDim.x) {
        const int r = e / c, q = e % c;
        S[r][q] = q <= r ? M[(long long)(j0 + r) * m + j0 + q] : 0.0;
    }
    __syncthreads();
    if (tid == 0) ip[0] = ldl_recip(S[0][0]);
    __syncthreads();
    for (int t = 0; t < c - 1; ++t) {
        const double it = ip[t];
        const int w = c - t - 1;   // trailing size
        for (int e = tid; e < w * (w + 1) / 2; e += blockDim.x) {
            // e -> (r, q), 0 <= q <= r < w, row-major over the trailing lower triangle
            int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
            while ((r + 1) * (r + 2) / 2 <= e) ++r;
            while (r * (r + 1) / 2 > e) --r;
            const int q = e - r * (r + 1) / 2;
            const int R = t + 1 + r, Q = t + 1 + q;
            const double l = S[R][t] * it;
            S[R][Q] = fma(-l, S[Q][t], S[R][Q]);
            if (r == 0) ip[t + 1] = ldl_recip(S[R][Q]);   // (t+1, t+1): the next pivot, now final
        }
        __syncthreads();
    }
    for (int e = tid; e < c * c; e += blockDim.x) {
        const int r = e / c, q = e % c;
        if (q < r) {
            M[(long long)(j0 + r) * m + j0 + q] = S[r][q] * ip[q];
        } else if (q == r) {
            M[(long long)(j0 + r) * m + j0 + r] = S[r][r];
            dinv[j0 + r] = ip[r];
        }
    }
}

// Lane t of a warp: the column-oriented forward substitution y (L_JJ)^T = x for one row
// (y_t = x_t - sum_{s<t} y_s L_ts), given x_t in acc; L_JJ in Lj (shared). Returns y_t.
__device__ __forceinline__ double ldl_fwd_row(double acc, const double (*__restrict__ Lj)[LDL_C + 1], int c, int lane)
{
    for (int s = 0; s < c; ++s) {
        const double ys = __shfl_sync(0xffffffffu, acc, s);
        if (lane > s && lane < c) acc = fma(-ys, Lj[lane][s], acc);
    }
    return acc;
}

// Lane t: the column-oriented backward substitution z L_JJ = x for one row
// (z_t = x_t - sum_{s>t} z_s L_st), given x_t in acc. Returns z_t.
__device__ __forceinline__ double ldl_bwd_row(double acc, const double (*__restrict__ Lj)[LDL_C + 1], int c, int lane)
{
    for (int s = c - 1; s >= 0; --s) {
        const double zs = __shfl_sync(0xffffffffu, acc, s);
        if (lane < s) acc = fma(-zs, Lj[s][lane], acc);
    }
    return acc;
}

// L_JJ (strict lower part, unit diagonal implied) from M into shared memory (the copies
// are waited for by the caller's ldl_cp_wait and barrier).
__device__ __forceinline__ void ldl_load_ljj(const double* __restrict__ M, int m, int j0, int c,
                                             double (*__restrict__ Lj)[LDL_C + 1])
{
    for (int e = threadIdx.x; e < LDL_C * LDL_C; e += blockDim.x) {
        const int r = e / LDL_C, q = e % LDL_C;
        if (r < c && q < r) ldl_cp8(&Lj[r][q], M + (long long)(j0 + r) * m + j0 + q);
        else Lj[r][q] = 0.0;
    }
}

// 1b. The band rows below block J: L_rJ from (L_rJ D_J) L_JJ^T = M_rJ by the forward
// substitution, then the scaling by 1 / d. One warp per row r in [j1, band end).
__device__ __forceinline__ void ldl_panel_body(double* __restrict__ M, int m, int j0, int c, int r1,
                                               const double* __restrict__ dinv, int bid)
{
    __shared__ double Lj[LDL_C][LDL_C + 1];
    ldl_load_ljj(M, m, j0, c, Lj);
    ldl_cp_wait();
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int r = j0 + c + bid * LDL_WARPS + (threadIdx.x >> 5);
    if (r >= r1) return;   // whole warps leave together
    double* row = M + (long long)r * m + j0;
    double acc = lane < c ? row[lane] : 0.0;
    acc = ldl_fwd_row(acc, Lj, c, lane);
    if (lane < c) row[lane] = acc * dinv[j0 + lane];
}

// 1c. The band below block J loses L_rJ D_J L_qJ^T: entries (r, q), j1 <= q <= r < r1, as
// 16 x 16 tiles of the lower triangle (tile b in row-major order over the tiles with
// tq <= tp). The c products of an entry run in pivot order; d_t is read from the diagonal.
__device__ __forceinline__ void ldl_update_body(double* __restrict__ M, int m, int j0, int c, int r1, int bid)
{
    __shared__ double Lr[16][LDL_C + 1], Wq[16][LDL_C + 1];
    int b = bid, tp = 0;
    while (b > tp) {   // lower tiles row by row: row tp holds tp + 1 tiles
        b -= tp + 1;
        ++tp;
    }
    const int tq = b;
    const int j1 = j0 + c;
    const int p0 = j1 + 16 * tp, q0 = j1 + 16 * tq;
    for (int e = threadIdx.x; e < 16 * LDL_C; e += blockDim.x) {
        const int i = e / LDL_C, t = e % LDL_C;
        const int pr = p0 + i, qr = q0 + i;
        Lr[i][t] = (pr < r1 && t < c) ? M[(long long)pr * m + j0 + t] : 0.0;
        Wq[i][t] = (qr < r1 && t < c) ? M[(long long)qr * m + j0 + t] * M[(long long)(j0 + t) * m + j0 + t] : 0.0;
    }
    __syncthreads();
    const int r = p0 + (threadIdx.x >> 4), q = q0 + (threadIdx.x & 15);
    if (r >= r1 || q > r) return;
    double acc = M[(long long)r * m + q];
    const int i = threadIdx.x >> 4, k = threadIdx.x & 15;
    for (int t = 0; t < c; ++t) acc = fma(-Lr[i][t], Wq[k][t], acc);
    M[(long long)r * m + q] = acc;
}

// 2a. Rows i of Z below block J (i in [j1, m)): X_iJ = sum_{k in [j1, kend)} Z[i][k] L[k][J],
// then Z_iJ = -X_iJ L_JJ^-1 by the backward substitution; written to Z[i][J] and, as its
// transpose, to Z[J][i]. One warp per row; lane t owns column j0 + t. The band rows
// [j1, kend) also keep X in Xs (row-major, LDL_C wide) for ldl_inv_diag_kernel. The
// CTA stages the band's L rows and each warp its row of Z in shared memory.
__device__ __forceinline__ void ldl_inv_rows_body(const double* __restrict__ M, double* __restrict__ Z, int m, int j0,
                                                  int c, int kend, double* __restrict__ Xs, int bid)
{
    extern __shared__ __align__(16) double ldl_smem[];
    const int j1 = j0 + c, nk = kend - j1;
    double(*Lj)[LDL_C + 1] = reinterpret_cast<double(*)[LDL_C + 1]>(ldl_smem);
    double* Lb = ldl_smem + LDL_C * (LDL_C + 1);          // [nk][LDL_C]: L[j1 + k][j0 + t]
    double* Zr = Lb + (long long)nk * LDL_C;               // [LDL_WARPS][nk]: the warps' rows of Z
    ldl_load_ljj(M, m, j0, c, Lj);
    for (int e = threadIdx.x; e < nk * LDL_C; e += blockDim.x) {
        const int k = e / LDL_C, t = e % LDL_C;
        if (t < c) ldl_cp8(Lb + e, M + (long long)(j1 + k) * m + j0 + t);
        else Lb[e] = 0.0;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int i = j1 + bid * LDL_WARPS + wid;
    double* zr = Zr + (long long)wid * nk;
    if (i < m)
        for (int k = lane; k < nk; k += 32) ldl_cp8(zr + k, Z + (long long)i * m + j1 + k);
    ldl_cp_wait();
    __syncthreads();
    if (i >= m) return;   // whole warps leave together
    const double x = ldl_dot4(zr, Lb + lane, LDL_C, nk);
    if (lane < c && i < kend) Xs[(long long)(i - j1) * LDL_C + lane] = x;
    double z = ldl_bwd_row(-x, Lj, c, lane);
    if (lane < c) {
        Z[(long long)i * m + j0 + lane] = z;
        Z[(long long)(j0 + lane) * m + i] = z;
    }
}

// 2b. Row s of Q = (D_J^-1 + Y) L_JJ^-1 with Y = L_KJ^T X_KJ (Y_st = sum_k L[k][j0+s] X[k][t]
// over the band rows): the sum, split over the CTA's warps in k (each warp one stretch,
// added in warp order), then the backward substitution by warp 0. One CTA per row s; Q to
// Qs (LDL_C x LDL_C).
__device__ __forceinline__ void ldl_inv_diag_body(const double* __restrict__ M, int m, int j0, int c, int kend,
                                                  const double* __restrict__ Xs, const double* __restrict__ dinv,
                                                  double* __restrict__ Qs, int s)
{
    extern __shared__ __align__(16) double ldl_smem[];
    __shared__ double Lj[LDL_C][LDL_C + 1];
    __shared__ double part[LDL_WARPS][LDL_C];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, j1 = j0 + c;
    const int nk = kend - j1, per = (nk + LDL_WARPS - 1) / LDL_WARPS;
    double* Lc = ldl_smem;          // [nk]: L[j1 + k][j0 + s]
    double* Xk = ldl_smem + nk;     // [nk][LDL_C]: the band rows of X
    ldl_load_ljj(M, m, j0, c, Lj);
    for (int k = threadIdx.x; k < nk; k += blockDim.x) ldl_cp8(Lc + k, M + (long long)(j1 + k) * m + j0 + s);
    for (int e = threadIdx.x; e < nk * LDL_C; e += blockDim.x) ldl_cp8(Xk + e, Xs + e);
    ldl_cp_wait();
    __syncthreads();
    const int k0 = min(nk, wid * per), k1 = min(nk, k0 + per);
    const double y = lane < c ? ldl_dot4(Lc + k0, Xk + (long long)k0 * LDL_C + lane, LDL_C, k1 - k0) : 0.0;
    part[wid][lane] = y;
    __syncthreads();
    if (wid != 0) return;
    double ys = part[0][lane];
    for (int w = 1; w < LDL_WARPS; ++w) ys += part[w][lane];
    if (lane == s) ys += dinv[j0 + s];
    const double q = ldl_bwd_row(ys, Lj, c, lane);
    if (lane < c) Qs[s * LDL_C + lane] = q;
}

// 2c. Z_JJ = L_JJ^-T Q, column w by column: L_JJ^T z = Q[.][w] is the backward
// substitution z_s = Q_sw - sum_{u>s} L_us z_u (lane s owns z_s). One warp per column w,
// LDL_WARPS columns per CTA; the upper entries (s <= w) are kept and mirrored, so Z_JJ is
// exactly symmetric.
__device__ __forceinline__ void ldl_inv_diag2_body(const double* __restrict__ M, double* __restrict__ Z, int m, int j0,
                                                   int c, const double* __restrict__ Qs, int bid)
{
    __shared__ double Lj[LDL_C][LDL_C + 1];
    ldl_load_ljj(M, m, j0, c, Lj);
    ldl_cp_wait();
    __syncthreads();
    const int lane = threadIdx.x & 31, w = bid * LDL_WARPS + (threadIdx.x >> 5);
    if (w >= c) return;   // whole warps leave together
    double acc = lane < c ? Qs[lane * LDL_C + w] : 0.0;
    acc = ldl_bwd_row(acc, Lj, c, lane);
    if (lane <= w) {
        Z[(long long)(j0 + lane) * m + j0 + w] = acc;
        Z[(long long)(j0 + w) * m + j0 + lane] = acc;
    }
}

// ---- launches: one matrix (the step's block passed in), or a batch of them in lockstep
// (state blockIdx.z, its block of step s derived from its own size and band; CTAs past a
// state's work leave). Same bodies, so a batched state is bit-identical to one grid.
__global__ void __launch_bounds__(512) ldl_diag_kernel(LdlState S, int j0, int c)
{
    ldl_diag_body(S.M, S.m, j0, c, S.dinv);
}
__global__ void __launch_bounds__(LDL_WARPS * 32) ldl_panel_kernel(LdlState S, int j0, int c, int r1)
{
    ldl_panel_body(S.M, S.m, j0, c, r1, S.dinv, blockIdx.x);
}
__global__ void __launch_bounds__(256) ldl_update_kernel(LdlState S, int j0, int c, int r1)
{
    ldl_update_body(S.M, S.m, j0, c, r1, blockIdx.x);
}
__global__ void __launch_bounds__(LDL_WARPS * 32) ldl_inv_rows_kernel(LdlState S, int j0, int c, int kend)
{
    ldl_inv_rows_body(S.M, S.Z, S.m, j0, c, kend, S.Xs, blockIdx.x);
}
__global__ void __launch_bounds__(LDL_WARPS * 32) ldl_inv_diag_kernel(LdlState S, int j0, int c, int kend)
{
    ldl_inv_diag_body(S.M, S.m, j0, c, kend, S.Xs, S.dinv, S.Qs, blockIdx.x);
}
__global__ void __launch_bounds__(LDL_WARPS * 32) ldl_inv_diag2_kernel(LdlState S, int j0, int c)
{
    ldl_inv_diag2_body(S.M, S.Z, S.m, j0, c, S.Qs, blockIdx.x);
}

// CTAs each launch needs for a block (the batched launches take the largest over states).
__host__ __device__ inline int ldl_panel_ctas(int j1, int r1) { return (r1 - j1 + LDL_WARPS - 1) / LDL_WARPS; }
__host__ __device__ inline int ldl_update_ctas(int j1, int r1)
{
    const int T = (r1 - j1 + 15) / 16;
    return T * (T + 1) / 2;
}
__host__ __device__ inline int ldl_rows_ctas(int m, int j1) { return (m - j1 + LDL_WARPS - 1) / LDL_WARPS; }
__host__ __device__ inline int ldl_diag2_ctas(int c) { return (c + LDL_WARPS - 1) / LDL_WARPS; }
__host__ __device__ inline size_t ldl_rows_smem(int nk)
{
    return sizeof(double) * ((size_t)LDL_C * (LDL_C + 1) + (size_t)nk * (LDL_C + LDL_WARPS));
}
__host__ __device__ inline size_t ldl_diag_smem(int nk) { return sizeof(double) * (size_t)nk * (LDL_C + 1); }

__global__ void __launch_bounds__(512) ldl_diag_batch_kernel(const LdlState* __restrict__ st,
                                                             const int* __restrict__ active, int s)
{
    int j0, c, r1;
    if (!active[blockIdx.z]) return;
    const LdlState S = st[blockIdx.z];
    if (!ldl_factor_step(S.m, S.b, s, j0, c, r1)) return;
    ldl_diag_body(S.M, S.m, j0, c, S.dinv);
}
__global__ void __launch_bounds__(LDL_WARPS * 32) ldl_panel_batch_kernel(const LdlState* __restrict__ st,
                                                                          const int* __restrict__ active, int s)
{
    int j0, c, r1;
    if (!active[blockIdx.z]) return;
    const LdlState S = st[blockIdx.z];
    if (!ldl_factor_step(S.m, S.b, s, j0, c, r1) || j0 + c >= S.m) return;
    if ((int)blockIdx.x >= ldl_panel_ctas(j0 + c, r1)) return;
    ldl_panel_body(S.M, S.m, j0, c, r1, S.dinv, blockIdx.x);
}
__global__ void __launch_bounds__(256) ldl_update_batch_kernel(const LdlState* __restrict__ st,
                                                               const int* __restrict__ active, int s)
{
    int j0, c, r1;
    if (!active[blockIdx.z]) return;
    const LdlState S = st[blockIdx.z];
    if (!ldl_factor_step(S.m, S.b, s, j0, c, r1) || j0 + c >= S.m) return;
    if ((int)blockIdx.x >= ldl_update_ctas(j0 + c, r1)) return;
    ldl_update_body(S.M, S.m, j0, c, r1, blockIdx.x);
}
__global__ void __launch_bounds__(LDL_WARPS * 32) ldl_inv_rows_batch_kernel(const LdlState* __restrict__ st,
                                                                             const int* __restrict__ active, int s)
{
    int j0, c, kend;
    if (!active[blockIdx.z]) return;
    const LdlState S = st[blockIdx.z];
    if (!ldl_inverse_step(S.m, S.b, s, j0, c, kend) || j0 + c >= S.m) return;
    if ((int)blockIdx.x >= ldl_rows_ctas(S.m, j0 + c)) return;
    ldl_inv_rows_body(S.M, S.Z, S.m, j0, c, kend, S.Xs, blockIdx.x);
}
__global__ void __launch_bounds__(LDL_WARPS * 32) ldl_inv_diag_batch_kernel(const LdlState* __restrict__ st,
                                                                             const int* __restrict__ active, int s)
{
    int j0, c, kend;
    if (!active[blockIdx.z]) return;
    const LdlState S = st[blockIdx.z];
    if (!ldl_inverse_step(S.m, S.b, s, j0, c, kend) || (int)blockIdx.x >= c) return;
    ldl_inv_diag_body(S.M, S.m, j0, c, kend, S.Xs, S.dinv, S.Qs, blockIdx.x);
}
__global__ void __launch_bounds__(LDL_WARPS * 32) ldl_inv_diag2_batch_kernel(const LdlState* __restrict__ st,
                                                                              const int* __restrict__ active, int s)
{
    int j0, c, kend;
    if (!active[blockIdx.z]) return;
    const LdlState S = st[blockIdx.z];
    if (!ldl_inverse_step(S.m, S.b, s, j0, c, kend) || (int)blockIdx.x >= ldl_diag2_ctas(c)) return;
    ldl_inv_diag2_body(S.M, S.Z, S.m, j0, c, S.Qs, blockIdx.x);
}

}  // namespace gf
