// CGS2 Gram-Schmidt passes of FGMRES in double-float arithmetic (FP32 pipe).
//
// On B300 the FP64 pipe runs at 1/64 of the FP32 rate, and the native CGS2 step costs
// four FP64 multiply-adds per basis entry (V^T w, w -= V h with V^T w fused, w -= V h'
// with ||w||^2), so it is FP64-bound rather than bandwidth-bound. Here every Krylov
// vector also lives as an unevaluated pair of floats (hi + lo, ~48 significant
// bits; Dekker 1971), and the passes run entirely on FP32 instructions:
//   product   a*b:  p = ah*bh, e = fma(ah, bh, -p) + ah*bl + al*bh   (exact p + e up to
//                   the low-part terms, Dekker's product via FMA)
//   sum       s+p:  Knuth's TwoSum on the high parts, the low parts added plainly
// w = K z_j arrives as a pair from the split-integer operator; only the FP64 copy of
// v_{j+1} (the V-cycle's right-hand side) and per-block partial sums use the FP64
// pipe. The results match native FP64 Gram-Schmidt to ~2^-47 relative;
// h, the rotations and the least-squares update stay in FP64, and acceptance is
// still decided by the native FP64 recomputed residual.
#pragma once
#include <cuda_runtime.h>

namespace gf {

__device__ __forceinline__ float2 dd_from_double(double x)
{
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ double dd_to_double(float h, float l) { return (double)h + (double)l; }

// (sh, sl) += (ah, al) * (bh, bl)
__device__ __forceinline__ void dd_mac(float ah, float al, float bh, float bl, float& sh, float& sl)
{
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float s = sh + p;
    const float bb = s - sh;
    const float err = (sh - (s - bb)) + (p - bb);
    sh = s;
    sl += err + e;
}

// (ah, al) += (bh, bl)
__device__ __forceinline__ void dd_add(float& ah, float& al, float bh, float bl)
{
    const float s = ah + bh;
    const float bb = s - ah;
    const float err = (ah - (s - bb)) + (bh - bb);
    ah = s;
    al += bl + err;
}

// normalised (h, l) of (ah, al) - (sh, sl): |l| <= ulp(h)/2, as stored
__device__ __forceinline__ float2 dd_sub_norm(float ah, float al, float sh, float sl)
{
    const float s = ah - sh;
    const float bb = s - ah;
    const float err = (ah - (s - bb)) + (-sh - bb);
    const float t = err + (al - sl);
    const float h = s + t;
    return make_float2(h, t - (h - s));
}

// ---- pass layout ---------------------------------------------------------------
// A block takes a contiguous chunk of rows in tiles of DD_TILE rows; within a tile,
// warp k owns the basis vectors q = k, k + 8, k + 16, ... and every lane DD_U rows
// (lane + 32 u). Each basis entry is loaded by exactly one thread, a thread holds
// only NV/8 accumulators (low register count, full occupancy, many loads in
// flight), and the per-row sums over q that the update passes need are combined
// across the 8 warps through shared memory in a fixed order (deterministic).
constexpr int DD_WARPS = 8, DD_THREADS = 32 * DD_WARPS, DD_U = 4, DD_TILE = 32 * DD_U;

__device__ __forceinline__ void dd_block_rows(long long n, long long& r0, long long& r1)
{
    const long long tiles = (n + DD_TILE - 1) / DD_TILE;
    const long long per = (tiles + gridDim.x - 1) / gridDim.x;
    r0 = (long long)blockIdx.x * per * DD_TILE;
    r1 = r0 + per * DD_TILE < n ? r0 + per * DD_TILE : n;
}

__device__ __forceinline__ void dd_warp_sum(float& h, float& l)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_down_sync(0xffffffffu, h, o), ol = __shfl_down_sync(0xffffffffu, l, o);
        dd_add(h, l, oh, ol);
    }
}

// Cross-block finish: every block stores its partial pairs, the last block to arrive
// (atomic ticket after a fence) sums them in block order, lanes striding over the
// blocks and then a fixed shuffle tree, writes dst[0..cnt) in FP64 and re-arms the
// ticket. No block waits on another, and the order of the sum does not depend on
// the order of arrival (deterministic).
// With xdst != nullptr, column xcol is summed the same way into *xdst as well.
__device__ __forceinline__ void dd_finish(const float2* pdd, int stride, int cnt, double* dst,
                                          unsigned int* ticket, int xcol = 0, double* xdst = nullptr)
{
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = gridDim.x;
    const int total = cnt + (xdst != nullptr ? 1 : 0);
    for (int q = warp; q < total; q += DD_WARPS) {
        const int col = q < cnt ? q : xcol;
        float h = 0.f, l = 0.f;
#pragma unroll 4
        for (int b = lane; b < nb; b += 32) {
            const float2 v = __ldcg(pdd + (long long)b * stride + col);
            dd_add(h, l, v.x, v.y);
        }
        dd_warp_sum(h, l);
        if (lane == 0) *(q < cnt ? dst + q : xdst) = dd_to_double(h, l);
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

// pass 1: partial[b][q] = sum_r Vd_q[r] wd[r] (q < NV, zero for q >= nv),
//         partial[b][NV] = ||wd||^2; the sums land in st->h1
template <int NV>
__device__ __forceinline__ void dd_dots_row(const float2* __restrict__ Vd, long long ld, int nv,
                                            const float2* __restrict__ wd, long long n, float2* __restrict__ partial)
{
    constexpr int QW = NV / DD_WARPS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float ah[QW + 1], al[QW + 1];
#pragma unroll
    for (int k = 0; k <= QW; ++k) ah[k] = al[k] = 0.f;
    long long r0, r1;
    dd_block_rows(n, r0, r1);
    for (long long t0 = r0; t0 < r1; t0 += DD_TILE) {
        float2 x[DD_U];
#pragma unroll
        for (int u = 0; u < DD_U; ++u) {
            const long long r = t0 + lane + 32 * u;
            x[u] = r < r1 ? wd[r] : make_float2(0.f, 0.f);
        }
        float2 v[QW][DD_U];   // all loads of the tile first, then the arithmetic
#pragma unroll
        for (int k = 0; k < QW; ++k) {
            const int q = warp + DD_WARPS * k;
#pragma unroll
            for (int u = 0; u < DD_U; ++u) {
                const long long r = t0 + lane + 32 * u;
                v[k][u] = (q < nv && r < r1) ? Vd[q * ld + r] : make_float2(0.f, 0.f);
            }
        }
#pragma unroll
        for (int k = 0; k < QW; ++k)
#pragma unroll
            for (int u = 0; u < DD_U; ++u) dd_mac(v[k][u].x, v[k][u].y, x[u].x, x[u].y, ah[k], al[k]);
        if (warp == 0) {
#pragma unroll
            for (int u = 0; u < DD_U; ++u) dd_mac(x[u].x, x[u].y, x[u].x, x[u].y, ah[QW], al[QW]);
        }
    }
    float2* row = partial + (long long)blockIdx.x * (NV + 1);
#pragma unroll
    for (int k = 0; k < QW; ++k) {
        dd_warp_sum(ah[k], al[k]);
        if (lane == 0) row[warp + DD_WARPS * k] = make_float2(ah[k], al[k]);
    }
    if (warp == 0) {
        dd_warp_sum(ah[QW], al[QW]);
        if (lane == 0) row[NV] = make_float2(ah[QW], al[QW]);
    }
}

template <int NV>
__global__ void __launch_bounds__(DD_THREADS)
ddgs_dots_kernel(const float2* __restrict__ Vd, long long ld, int nv, const float2* __restrict__ wd,
                 long long n, float2* __restrict__ partial, KState* __restrict__ st, unsigned int* ticket)
{
    if (st->status != KS_RUN) return;
    dd_dots_row<NV>(Vd, ld, nv, wd, n, partial);
    dd_finish(partial, NV + 1, NV + 1, st->h1, ticket);   // h1[0..NV), ||w||^2 in h1[NV]
}

// h (FP64, from the state) as double-float pairs in shared memory
template <int NV>
__device__ __forceinline__ void dd_load_h(const double* __restrict__ h, int nv, float2* hs)
{
    if (threadIdx.x < NV) hs[threadIdx.x] = threadIdx.x < nv ? dd_from_double(h[threadIdx.x]) : make_float2(0.f, 0.f);
    __syncthreads();
}

// Shared part of the two update passes for one tile: loads v (kept in registers),
// each warp's partial sum_q h_q v_q per row into part[warp][.], then the first
// DD_TILE threads combine the warps in order, form wd_new = wd - sum, store it, and
// return it (zero outside [r0, r1)) in wn_s. Ends with every thread past a barrier.
template <int NV>
__device__ __forceinline__ void dd_update_tile(const float2* __restrict__ Vd, long long ld, int nv,
                                               float2* __restrict__ wd, long long t0, long long r1,
                                               const float2* hs, float2 (&v)[NV / DD_WARPS][DD_U],
                                               float2 (*part)[DD_TILE], float2* wn_s)
{
    constexpr int QW = NV / DD_WARPS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < QW; ++k) {
        const int q = warp + DD_WARPS * k;
#pragma unroll
        for (int u = 0; u < DD_U; ++u) {
            const long long r = t0 + lane + 32 * u;
            v[k][u] = (q < nv && r < r1) ? Vd[q * ld + r] : make_float2(0.f, 0.f);
        }
    }
#pragma unroll
    for (int u = 0; u < DD_U; ++u) {
        float sh = 0.f, sl = 0.f;
#pragma unroll
        for (int k = 0; k < QW; ++k) {
            const float2 h = hs[warp + DD_WARPS * k];
            dd_mac(h.x, h.y, v[k][u].x, v[k][u].y, sh, sl);
        }
        part[warp][lane + 32 * u] = make_float2(sh, sl);
    }
    __syncthreads();
    if (threadIdx.x < DD_TILE) {
        const long long r = t0 + threadIdx.x;
        float sh = 0.f, sl = 0.f;
#pragma unroll
        for (int w = 0; w < DD_WARPS; ++w) dd_add(sh, sl, part[w][threadIdx.x].x, part[w][threadIdx.x].y);
        float2 wn = make_float2(0.f, 0.f);
        if (r < r1) {
            const float2 x = wd[r];
            wn = dd_sub_norm(x.x, x.y, sh, sl);
            wd[r] = wn;
        }
        wn_s[threadIdx.x] = wn;
    }
    __syncthreads();
}

// pass 2: wd -= sum_q h1_q Vd_q ; partial[b][q] = sum_r Vd_q[r] wd_new[r] (q < nv); sums in st->h2
template <int NV>
__global__ void __launch_bounds__(DD_THREADS)
ddgs_update_dots_kernel(const float2* __restrict__ Vd, long long ld, int nv, float2* __restrict__ wd,
                        long long n, float2* __restrict__ partial, KState* __restrict__ st,
                        unsigned int* ticket)
{
    if (st->status != KS_RUN) return;
    constexpr int QW = NV / DD_WARPS;
    __shared__ float2 hs[NV];
    __shared__ float2 part[DD_WARPS][DD_TILE];
    __shared__ float2 wn_s[DD_TILE];
    dd_load_h<NV>(st->h1, nv, hs);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float ah[QW], al[QW];
#pragma unroll
    for (int k = 0; k < QW; ++k) ah[k] = al[k] = 0.f;
    long long r0, r1;
    dd_block_rows(n, r0, r1);
    for (long long t0 = r0; t0 < r1; t0 += DD_TILE) {
        float2 v[QW][DD_U];
        dd_update_tile<NV>(Vd, ld, nv, wd, t0, r1, hs, v, part, wn_s);
#pragma unroll
        for (int k = 0; k < QW; ++k)
#pragma unroll
            for (int u = 0; u < DD_U; ++u) {
                const float2 x = wn_s[lane + 32 * u];
                dd_mac(v[k][u].x, v[k][u].y, x.x, x.y, ah[k], al[k]);
            }
    }
    float2* row = partial + (long long)blockIdx.x * NV;
#pragma unroll
    for (int k = 0; k < QW; ++k) {
        dd_warp_sum(ah[k], al[k]);
        if (lane == 0) row[warp + DD_WARPS * k] = make_float2(ah[k], al[k]);
    }
    dd_finish(partial, NV, NV, st->h2, ticket);
}

// pass 3: wd -= sum_q h2_q Vd_q ; partial[b][0] = ||wd_new||^2 (block part); sum in st->ww
// wd -= sum_q h_q Vd_q over this block's rows; partial[b] = the block part of ||wd_new||^2
template <int NV>
__device__ __forceinline__ void dd_update_norm_row(const float2* __restrict__ Vd, long long ld, int nv,
                                                   float2* __restrict__ wd, long long n,
                                                   float2* __restrict__ partial, const double* h)
{
    constexpr int QW = NV / DD_WARPS;
    __shared__ float2 hs[NV];
    __shared__ float2 part[DD_WARPS][DD_TILE];
    __shared__ float2 wn_s[DD_TILE];
    __shared__ float2 red[DD_WARPS];
    dd_load_h<NV>(h, nv, hs);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float nh = 0.f, nl = 0.f;
    long long r0, r1;
    dd_block_rows(n, r0, r1);
    for (long long t0 = r0; t0 < r1; t0 += DD_TILE) {
        float2 v[QW][DD_U];
        dd_update_tile<NV>(Vd, ld, nv, wd, t0, r1, hs, v, part, wn_s);
        if (threadIdx.x < DD_TILE) {
            const float2 x = wn_s[threadIdx.x];
            dd_mac(x.x, x.y, x.x, x.y, nh, nl);
        }
    }
    dd_warp_sum(nh, nl);
    if (lane == 0) red[warp] = make_float2(nh, nl);
    __syncthreads();
    if (threadIdx.x == 0) {
        float h = 0.f, l = 0.f;
#pragma unroll
        for (int w = 0; w < DD_WARPS; ++w) dd_add(h, l, red[w].x, red[w].y);
        partial[blockIdx.x] = make_float2(h, l);
    }
}

template <int NV>
__global__ void __launch_bounds__(DD_THREADS)
ddgs_update_norm_kernel(const float2* __restrict__ Vd, long long ld, int nv, float2* __restrict__ wd,
                        long long n, float2* __restrict__ partial, KState* __restrict__ st,
                        unsigned int* ticket)
{
    if (st->status != KS_RUN) return;
    dd_update_norm_row<NV>(Vd, ld, nv, wd, n, partial, st->h2);
    dd_finish(partial, 1, 1, &st->ww, ticket);
}

// ---- long restarts: the basis in slices of NV vectors ------------------------------
// The double-float counterparts of the FP64 slice passes: dots of one slice against
// wd into dst[0..nv) (and ||wd||^2 into *wwdst when given), and wd -= Vd_slice h_slice
// (with ||wd_new||^2 into *wwdst when given: the last slice of the second update).
template <int NV>
__global__ void __launch_bounds__(DD_THREADS)
ddgs_slice_dots_kernel(const float2* __restrict__ Vd, long long ld, int nv, const float2* __restrict__ wd,
                       long long n, float2* __restrict__ partial, const KState* st, unsigned int* ticket,
                       double* dst, double* wwdst)
{
    if (st->status != KS_RUN) return;
    dd_dots_row<NV>(Vd, ld, nv, wd, n, partial);
    dd_finish(partial, NV + 1, nv, dst, ticket, NV, wwdst);
}

template <int NV>
__global__ void __launch_bounds__(DD_THREADS)
ddgs_slice_update_kernel(const float2* __restrict__ Vd, long long ld, int nv, float2* __restrict__ wd,
                         long long n, float2* __restrict__ partial, const KState* st, unsigned int* ticket,
                         const double* h, double* wwdst)
{
    if (st->status != KS_RUN) return;
    dd_update_norm_row<NV>(Vd, ld, nv, wd, n, partial, h);
    if (wwdst != nullptr) dd_finish(partial, 1, 1, wwdst, ticket);
}

// v_{j+1} = wd * inv: the double-float basis vector in place, and its FP64 value
// (the V-cycle's right-hand side) into v.
__global__ void ddgs_scale_kernel(float2* __restrict__ wd, double* __restrict__ v, long long n,
                                  const KState* __restrict__ st)
{
    if (st->status != KS_RUN) return;
    const float2 s = dd_from_double(st->inv);
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (long long)gridDim.x * blockDim.x) {
        const float2 x = wd[r];
        const float p = x.x * s.x;
        float e = fmaf(x.x, s.x, -p);
        e = fmaf(x.x, s.y, e);
        e = fmaf(x.y, s.x, e);
        const float h = p + e;
        const float l = e - (h - p);
        wd[r] = make_float2(h, l);
        v[r] = dd_to_double(h, l);
    }
}

// cycle start: v_0 *= inv in FP64 (as the native path) and its double-float copy
__global__ void ddgs_scale_fp64_kernel(double* __restrict__ v, float2* __restrict__ vd, long long n,
                                       const KState* __restrict__ st)
{
    if (st->status != KS_RUN) return;
    const double s = st->inv;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (long long)gridDim.x * blockDim.x) {
        const double x = v[r] * s;
        v[r] = x;
        vd[r] = dd_from_double(x);
    }
}

}  // namespace gf
