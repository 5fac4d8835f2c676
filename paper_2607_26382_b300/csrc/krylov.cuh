// FGMRES(m) device kernels: fused classical Gram-Schmidt with one re-orthogonalisation
// (CGS2), deterministic two-stage reductions, the Givens/Hessenberg update and the
// residual history on the device, so the host only polls a stop flag.
//
// Right-preconditioned flexible GMRES (Saad 1993), as used by the paper's outer
// solver (Sec. 3.5 "Why a flexible Krylov method", Table residual-semantics):
//   z_j = B v_j, w = K z_j, h = V^T w, w -= V h, h' = V^T w, w -= V h', h += h',
//   h_{j+1,j} = ||w||, rotate, g_{j+1} = -s g_j, g_j = c g_j, history = |g_{j+1}|/||f||.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace gf {

constexpr int KRY_NV = 32;      // basis vectors per fused Gram-Schmidt pass (one register accumulator each)
constexpr int KRY_MMAX = 300;   // restart cap; past KRY_NV vectors the passes run over slices of KRY_NV
constexpr int RED_THREADS = 256;

enum { KS_RUN = 0, KS_STOP = 1 };

struct KState {
    double H[(KRY_MMAX + 1) * KRY_MMAX];   // column-major, ld = KRY_MMAX+1
    double cs[KRY_MMAX], sn[KRY_MMAX], g[KRY_MMAX + 1];
    double h1[KRY_MMAX + 2];               // first-pass dots (+ ||w||^2 in slot NV)
    double h2[KRY_MMAX + 1];               // second-pass dots
    double y[KRY_MMAX];
    double ww;                             // ||w||^2 after CGS2
    double fnorm, tol, inv, beta;
    int k, kmax, m, J, status, flag, j;
    int skip;                              // 1: this state sits out (batched solves)
};

// ---------------------------------------------------------------- reductions --
__host__ __device__ constexpr int pow2_at_least(int v)
{
    return v <= 1 ? 1 : 2 * pow2_at_least((v + 1) / 2);
}

// Sums P values (a power of two <= 32) over the 32 lanes of a warp by transposition: at the
// level with lane offset o each lane keeps one half of its values (the upper half when its
// bit o is set), sends the other half to lane ^ o and adds what it receives, so the P
// values cost P - 1 shuffles and adds instead of 5 P; then the lanes that hold the same
// value (those sharing their top log2 P bits) add theirs. Lane l returns the warp's sum
// of value l / (32 / P).
template <int P>
__device__ __forceinline__ double warp_transpose_sum(double (&v)[P], int lane)
{
#pragma unroll
    for (int h = P / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const double lo = v[i], hi = v[i + h];
            v[i] = (up ? hi : lo) + __shfl_xor_sync(0xffffffffu, up ? lo : hi, o);
        }
    }
    double s = v[0];
#pragma unroll
    for (int o = 16 / P; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// partial[b][q] = sum over the block's T threads of acc[q], q < nv: each warp sums its
// values by transposition (the first 32; an NV of 33 adds its last value by a shuffle
// tree), then thread q adds the warps' sums in warp order.
template <int NV, int T = RED_THREADS>
__device__ __forceinline__ void block_reduce_store(double (&acc)[NV], int nv, double* __restrict__ out_row)
{
    constexpr int NT = NV < 32 ? NV : 32;   // values summed by transposition
    constexpr int P = pow2_at_least(NT);
    constexpr int SPREAD = 32 / P;          // lanes that end up with one value
    __shared__ double red[T / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double v[P];
#pragma unroll
    for (int q = 0; q < P; ++q) v[q] = q < NT ? acc[q] : 0.0;
    const double s = warp_transpose_sum<P>(v, lane);
    if (lane % SPREAD == 0 && lane / SPREAD < NT) red[warp][lane / SPREAD] = s;
#pragma unroll
    for (int q = NT; q < NV; ++q) {   // NV = 33: the norm slot
        double t = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) red[warp][q] = t;
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < T / 32; ++w) t += red[w][threadIdx.x];
        out_row[threadIdx.x] = t;
    }
}

// Cross-block finish of the FP64 passes: every block has stored its partial row; the last
// block to arrive (atomic ticket after a fence) sums column q < cnt over the blocks in
// reduce_partials_kernel's order (lane l takes blocks l, l + 32, ... in turn, then a
// shuffle tree), writes dst[q] and re-arms the ticket. No block waits on another, and the
// sums do not depend on the order of arrival.
__device__ __forceinline__ bool fp64_finish(const double* partial, int stride, int cnt, double* dst,
                                            unsigned int* ticket)
{
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return false;
    __threadfence();
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int nb = gridDim.x;
    for (int q = threadIdx.x >> 5; q < cnt; q += nw) {
        double s = 0.0;
#pragma unroll 8
        for (int b = lane; b < nb; b += 32) s += __ldcg(partial + (long long)b * stride + q);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) dst[q] = s;
    }
    if (threadIdx.x == 0) *ticket = 0u;
    return true;
}

// Step j's Arnoldi tail, one warp (defined with arnoldi_tail_kernel below).
__device__ __forceinline__ void arnoldi_tail_warp(KState* st, double* hist, int j, int ww0_slot,
                                                  volatile int* host_status, double breakdown_rtol, double* col,
                                                  double* cs, double* sn, int lane);

// rows of block b: [b*chunk, min(n, (b+1)*chunk))
__device__ __forceinline__ void block_rows(long long n, long long& r0, long long& r1)
{
    const long long chunk = (n + gridDim.x - 1) / gridDim.x;
    r0 = (long long)blockIdx.x * chunk;
    r1 = r0 + chunk < n ? r0 + chunk : n;
}

// The three FP64 passes of CGS2 over the rows of a block. Each thread takes rows
// r, r + RED_THREADS, ... in order; CgsRows<NV>::value of them per iteration have all
// their loads (predicated) in flight together, then the FP64 multiply-adds run for the nv
// live vectors only: the FP64 pipe, not memory, bounds these passes on B300 once nv is a
// few vectors, and a multiply-add by a zero entry would cost as much as a real one. Below
// that the rows in flight hide the HBM latency (four rows per iteration for NV = 8; the
// results do not depend on it). The grid is the blocks resident at once (gf_grid::nbc).
template <int NV>
struct CgsRows {
    static constexpr int value = NV <= 8 ? 4 : 1;
};

// pass 1: partial[b][i] = sum_r V_i[r] w[r] (i < nv), partial[b][nv] = sum_r w[r]^2
// (NV = 32: the row's vectors in two groups of 16, loaded together per group, so that
// two blocks fit on an SM; the multiply-adds run in the same order)
template <int NV>
__global__ void __launch_bounds__(RED_THREADS, NV >= 16 ? 2 : 1)
cgs_dots_kernel(const double* __restrict__ V, long long ld, int nv, const double* __restrict__ w,
                long long n, double* __restrict__ partial, const KState* st, KState* fin = nullptr,
                unsigned int* ticket = nullptr)
{
    constexpr int ROWS = CgsRows<NV>::value;
    constexpr int G = NV == 32 ? 16 : NV;   // vectors loaded together
    if (st->status != KS_RUN) return;
    double acc[NV + 1];
#pragma unroll
    for (int q = 0; q <= NV; ++q) acc[q] = 0.0;
    long long r0, r1;
    block_rows(n, r0, r1);
    for (long long r = r0 + threadIdx.x; r < r1; r += (long long)RED_THREADS * ROWS) {
        double wr[ROWS];
#pragma unroll
        for (int u = 0; u < ROWS; ++u) {
            const long long rr = r + (long long)u * RED_THREADS;
            wr[u] = (u == 0 || rr < r1) ? w[rr] : 0.0;
        }
#pragma unroll
        for (int g0 = 0; g0 < NV; g0 += G) {
            if (g0 >= nv) break;
            double v[ROWS][G];
#pragma unroll
            for (int u = 0; u < ROWS; ++u) {
                const long long rr = r + (long long)u * RED_THREADS;
                const bool ok = u == 0 || rr < r1;   // row r itself is inside the range
#pragma unroll
                for (int q = 0; q < G; ++q) v[u][q] = (ok && g0 + q < nv) ? V[(g0 + q) * ld + rr] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < ROWS; ++u) {
                if (r + (long long)u * RED_THREADS >= r1) break;
#pragma unroll
                for (int q = 0; q < G; ++q) {
                    if (g0 + q >= nv) break;
                    acc[g0 + q] = fma(v[u][q], wr[u], acc[g0 + q]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < ROWS; ++u) {
            if (r + (long long)u * RED_THREADS >= r1) break;
            acc[NV] = fma(wr[u], wr[u], acc[NV]);
        }
    }
    // row layout: dots in slots [0, nv), ||w||^2 in slot NV (row stride NV + 1)
    block_reduce_store<NV + 1>(acc, NV + 1, partial + (long long)blockIdx.x * (NV + 1));
    if (ticket != nullptr) fp64_finish(partial, NV + 1, NV + 1, fin->h1, ticket);   // h1, ||w||^2 in h1[NV]
}

// pass 2: w -= sum_i h1_i V_i ; partial[b][i] = sum_r V_i[r] w_new[r]
// (the update runs as w_new = fma(-h_nv-1, V_nv-1, ... fma(-h_0, V_0, w)): nv FMAs, no
// separate subtraction; the negated coefficients are formed once per block). T threads
// per block: 128 when the grid leaves half of each SM to other streams (its NV = 32 form
// holds up to 255 registers per thread).
template <int NV, int T = RED_THREADS>
__global__ void __launch_bounds__(T)
cgs_update_dots_kernel(const double* __restrict__ V, long long ld, int nv, double* __restrict__ w,
                       long long n, double* __restrict__ partial, const KState* st, KState* fin = nullptr,
                       unsigned int* ticket = nullptr)
{
    constexpr int ROWS = CgsRows<NV>::value;
    if (st->status != KS_RUN) return;
    __shared__ double h[NV];   // -h1
    double acc[NV];
    if (threadIdx.x < NV) h[threadIdx.x] = threadIdx.x < nv ? -st->h1[threadIdx.x] : 0.0;
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = 0.0;
    __syncthreads();
    long long r0, r1;
    block_rows(n, r0, r1);
    for (long long r = r0 + threadIdx.x; r < r1; r += (long long)T * ROWS) {
        double wr[ROWS], v[ROWS][NV];
#pragma unroll
        for (int u = 0; u < ROWS; ++u) {
            const long long rr = r + (long long)u * T;
            const bool ok = u == 0 || rr < r1;   // row r itself is inside the range
            wr[u] = ok ? w[rr] : 0.0;
#pragma unroll
            for (int q = 0; q < NV; ++q) v[u][q] = (ok && q < nv) ? V[q * ld + rr] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < ROWS; ++u) {
            const long long rr = r + (long long)u * T;
            if (rr >= r1) break;
            double s = wr[u];
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                if (q >= nv) break;
                s = fma(h[q], v[u][q], s);
            }
            const double wn = s;
            w[rr] = wn;
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                if (q >= nv) break;
                acc[q] = fma(v[u][q], wn, acc[q]);
            }
        }
    }
    block_reduce_store<NV, T>(acc, nv, partial + (long long)blockIdx.x * NV);
    if (ticket != nullptr) fp64_finish(partial, NV, nv, fin->h2, ticket);
}

// pass 3: w -= sum_i h2_i V_i ; partial[b][0] = ||w_new||^2 (block part)
// (NV = 32: two groups of 16 vectors, as in pass 1; the update as in pass 2, from -h2)
template <int NV>
__global__ void __launch_bounds__(RED_THREADS, NV >= 16 ? 2 : 1)
cgs_update_norm_kernel(const double* __restrict__ V, long long ld, int nv, double* __restrict__ w,
                       long long n, double* __restrict__ partial, const KState* st, KState* fin, unsigned int* ticket,
                       double* tail_hist, int j, int ww0_slot, volatile int* host_status, double breakdown_rtol)
{
    constexpr int ROWS = CgsRows<NV>::value;
    constexpr int G = NV == 32 ? 16 : NV;
    if (st->status != KS_RUN) return;
    __shared__ double h[NV];   // -h2
    if (threadIdx.x < NV) h[threadIdx.x] = threadIdx.x < nv ? -st->h2[threadIdx.x] : 0.0;
    __syncthreads();
    double acc[1] = {0.0};
    long long r0, r1;
    block_rows(n, r0, r1);
    for (long long r = r0 + threadIdx.x; r < r1; r += (long long)RED_THREADS * ROWS) {
        double s[ROWS], wr[ROWS];
#pragma unroll
        for (int u = 0; u < ROWS; ++u) {
            const long long rr = r + (long long)u * RED_THREADS;
            wr[u] = (u == 0 || rr < r1) ? w[rr] : 0.0;
            s[u] = wr[u];
        }
#pragma unroll
        for (int g0 = 0; g0 < NV; g0 += G) {
            if (g0 >= nv) break;
            double v[ROWS][G];
#pragma unroll
            for (int u = 0; u < ROWS; ++u) {
                const long long rr = r + (long long)u * RED_THREADS;
                const bool ok = u == 0 || rr < r1;   // row r itself is inside the range
#pragma unroll
                for (int q = 0; q < G; ++q) v[u][q] = (ok && g0 + q < nv) ? V[(g0 + q) * ld + rr] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < ROWS; ++u) {
#pragma unroll
                for (int q = 0; q < G; ++q) {
                    if (g0 + q >= nv) break;
                    s[u] = fma(h[g0 + q], v[u][q], s[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < ROWS; ++u) {
            const long long rr = r + (long long)u * RED_THREADS;
            if (rr >= r1) break;
            const double wn = s[u];
            w[rr] = wn;
            acc[0] = fma(wn, wn, acc[0]);
        }
    }
    block_reduce_store<1>(acc, 1, partial + blockIdx.x);
    if (ticket != nullptr && fp64_finish(partial, 1, 1, &fin->ww, ticket) && tail_hist != nullptr) {
        // the last block also runs step j's Arnoldi tail (arnoldi_tail_kernel's warp)
        __shared__ double col[KRY_MMAX + 1], cs[KRY_MMAX], sn[KRY_MMAX];
        __syncthreads();   // ||w||^2 stored before warp 0 reads it
        if (threadIdx.x < 32)
            arnoldi_tail_warp(fin, tail_hist, j, ww0_slot, host_status, breakdown_rtol, col, cs, sn, (int)threadIdx.x);
    }
}

template <int NV>
__global__ void __launch_bounds__(RED_THREADS)
cgs_slice_update_kernel(const double* __restrict__ V, long long ld, int nv, double* __restrict__ w,
                        long long n, const double* hsl, double* __restrict__ partial, const KState* st)
{
    if (st->status != KS_RUN) return;
    __shared__ double h[NV];
    if (threadIdx.x < NV) h[threadIdx.x] = threadIdx.x < nv ? hsl[threadIdx.x] : 0.0;
    __syncthreads();
    double acc[1] = {0.0};
    long long r0, r1;
    block_rows(n, r0, r1);
    for (long long r = r0 + threadIdx.x; r < r1; r += RED_THREADS) {
        double v[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] = q < nv ? V[q * ld + r] : 0.0;
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            if (q >= nv) break;
            s = fma(h[q], v[q], s);
        }
        const double wn = w[r] - s;
        w[r] = wn;
        acc[0] = fma(wn, wn, acc[0]);
    }
    if (partial != nullptr) block_reduce_store<1>(acc, 1, partial + blockIdx.x);
}

// dst[i] = sum_b partial[b * stride + src0 + i], i < cnt, in reduce_partials_kernel's
// order; dst is a slot range of the state (a slice of h1 or h2, ||w||^2).
__global__ void reduce_slice_kernel(const double* __restrict__ partial, int nblocks, int stride, int src0, int cnt,
                                    double* dst, const KState* st)
{
    if (st->status != KS_RUN) return;
    const int lane = threadIdx.x & 31;
    for (int q = threadIdx.x >> 5; q < cnt; q += blockDim.x >> 5) {
        double s = 0.0;
#pragma unroll 8
        for (int b = lane; b < nblocks; b += 32) s += partial[(long long)b * stride + src0 + q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) dst[q] = s;
    }
}

// Sum partial[b][i] over blocks b (fixed order: deterministic). One warp per i.
// dst selects where the sums go in the state: 0 -> h1[0..cnt), 1 -> h2[0..cnt),
// 2 -> ww (cnt == 1).
__global__ void reduce_partials_kernel(const double* __restrict__ partial, int nblocks, int stride, int cnt,
                                       KState* __restrict__ st, int dst, int check_status)
{
    if (check_status && st->status != KS_RUN) return;
    const int lane = threadIdx.x & 31;
    const int i = threadIdx.x >> 5;
    for (int q = i; q < cnt; q += blockDim.x >> 5) {
        double s = 0.0;
        // unrolled so the loads are in flight together; the additions keep their order
#pragma unroll 8
        for (int b = lane; b < nblocks; b += 32) s += partial[(long long)b * stride + q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) {
            if (dst == 0) st->h1[q] = s;
            else if (dst == 1) st->h2[q] = s;
            else st->ww = s;
        }
    }
}

// ---------------------------------------------------------------- Arnoldi tail --
// One warp: stage column j of H and the stored rotations in shared memory (one round
// of parallel loads), then one thread applies the rotations, forms the new one,
// updates g, records the history and decides whether to stop. The serial recurrence
// reads only shared memory: from global memory, each step's loads would wait behind
// the previous step's store to the same struct.
__device__ __forceinline__ void arnoldi_tail_warp(KState* st, double* hist, int j, int ww0_slot,
                                                  volatile int* host_status, double breakdown_rtol, double* col,
                                                  double* cs, double* sn, int lane)
{
    if (st->status != KS_RUN) return;   // uniform over the warp
    for (int i = lane; i <= j; i += 32) col[i] = st->h1[i] + st->h2[i];
    for (int i = lane; i < j; i += 32) {
        cs[i] = st->cs[i];
        sn[i] = st->sn[i];
    }
    const double hnext = sqrt(st->ww);
    __syncwarp();
    if (lane == 0) {
        col[j + 1] = hnext;
        for (int i = 0; i < j; ++i) {
            const double a = col[i], b = col[i + 1];
            col[i] = cs[i] * a + sn[i] * b;
            col[i + 1] = -sn[i] * a + cs[i] * b;
        }
    }
    __syncwarp();
    const int ldh = KRY_MMAX + 1;
    double* Hc = st->H + (long long)j * ldh;
    for (int i = lane; i < j; i += 32) Hc[i] = col[i];   // rows 0..j-1 are final
    if (lane != 0) return;
    const double wnorm0 = sqrt(st->h1[ww0_slot]);
    const double a = col[j], b = col[j + 1];
    const double rho = hypot(a, b);
    st->j = j;
    if (rho == 0.0) {            // degenerate column: breakdown, drop the step
        Hc[j] = a;
        Hc[j + 1] = b;
        st->status = KS_STOP;
        st->flag = 2;
        st->J = j;
        *host_status = KS_STOP;
        return;
    }
    const double c = a / rho, s = b / rho;
    st->cs[j] = c;
    st->sn[j] = s;
    Hc[j] = rho;
    Hc[j + 1] = 0.0;
    const double gj = st->g[j];
    st->g[j + 1] = -s * gj;
    st->g[j] = c * gj;
    st->k += 1;
    st->J = j + 1;
    const double est = fabs(st->g[j + 1]) / st->fnorm;
    hist[st->k] = est;
    if (est <= st->tol) {
        st->status = KS_STOP;
        st->flag = 0;
    } else if (st->k >= st->kmax) {
        st->status = KS_STOP;
        st->flag = 1;
    } else if (hnext <= breakdown_rtol * wnorm0) {
        st->status = KS_STOP;
        st->flag = 2;
    } else {
        st->inv = 1.0 / hnext;
    }
    if (st->status == KS_STOP) *host_status = KS_STOP;
}

__global__ void arnoldi_tail_kernel(KState* __restrict__ st, double* __restrict__ hist, int j,
                                    int ww0_slot, volatile int* host_status, double breakdown_rtol)
{
    __shared__ double col[KRY_MMAX + 1], cs[KRY_MMAX], sn[KRY_MMAX];
    arnoldi_tail_warp(st, hist, j, ww0_slot, host_status, breakdown_rtol, col, cs, sn, (int)threadIdx.x);
}

// Cycle start: beta = ||r||, history[k] = beta/||f|| (a true residual), g = beta e1.
__global__ void cycle_start_tail_kernel(KState* __restrict__ st, double* __restrict__ hist,
                                        volatile int* host_status, int first)
{
    if (threadIdx.x != 0 || st->skip) return;
    const double beta = sqrt(st->h1[0]);          // ||M f - K x||
    if (first) st->fnorm = sqrt(st->h1[1]);       // ||M f||
    st->beta = beta;
    st->J = 0;
    const double rel = beta / st->fnorm;
    hist[st->k] = rel;
    for (int i = 0; i <= st->m; ++i) st->g[i] = 0.0;
    st->g[0] = beta;
    if (rel <= st->tol) {
        st->status = KS_STOP;
        st->flag = 0;
    } else if (st->k >= st->kmax) {
        st->status = KS_STOP;
        st->flag = 1;
    } else {
        st->status = KS_RUN;
        st->inv = 1.0 / beta;
    }
    *host_status = st->status;
}

// Upper-triangular back substitution H[0:J,0:J] y = g[0:J].
__global__ void backsolve_kernel(KState* __restrict__ st)
{
    if (threadIdx.x != 0 || st->skip) return;
    const int ldh = KRY_MMAX + 1;
    const int J = st->J;
    for (int i = J - 1; i >= 0; --i) {
        double s = st->g[i];
        for (int c = i + 1; c < J; ++c) s -= st->H[(long long)c * ldh + i] * st->y[c];
        st->y[i] = s / st->H[(long long)i * ldh + i];
    }
}

// x += sum_{i<J} y_i Z_i
__global__ void __launch_bounds__(256)
update_x_kernel(double* __restrict__ x, const double* __restrict__ Z, long long ld, long long n,
                const KState* __restrict__ st)
{
    __shared__ double ys[KRY_MMAX];
    if (st->skip) return;
    const int J = st->J;
    for (int i = threadIdx.x; i < J; i += blockDim.x) ys[i] = st->y[i];
    __syncthreads();
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (long long)gridDim.x * blockDim.x) {
        double s = x[r];
        for (int i = 0; i < J; ++i) s = fma(ys[i], Z[i * ld + r], s);
        x[r] = s;
    }
}

// v *= st->inv (skipped once stopped)
__global__ void scale_kernel(double* __restrict__ v, long long n, const KState* __restrict__ st, int check_status)
{
    if (check_status && st->status != KS_RUN) return;
    const double s = st->inv;
    // four independent entries per thread and iteration (loads in flight together)
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; r + 3 * stride < n; r += 4 * stride) {
        const double a0 = v[r], a1 = v[r + stride], a2 = v[r + 2 * stride], a3 = v[r + 3 * stride];
        v[r] = a0 * s;
        v[r + stride] = a1 * s;
        v[r + 2 * stride] = a2 * s;
        v[r + 3 * stride] = a3 * s;
    }
    for (; r < n; r += stride) v[r] *= s;
}

// r = M f - y (y = K x) into r; partial[b][0] = ||r||^2, partial[b][1] = ||M f||^2.
// fixed DOFs: (r/3) % NX == 0.
__global__ void __launch_bounds__(RED_THREADS)
residual_norms_kernel(const double* __restrict__ f, const double* y, double* r,
                      long long n, int NX, double* __restrict__ partial, int y_is_zero,
                      const int* __restrict__ halt, const uint8_t* __restrict__ fix = nullptr)
{
    if (halt != nullptr && *halt != 0) return;
    double acc[2] = {0.0, 0.0};
    long long r0, r1;
    block_rows(n, r0, r1);
    for (long long q = r0 + threadIdx.x; q < r1; q += RED_THREADS) {
        const bool fixed = fix ? ((fix[q / 3] >> (int)(q % 3)) & 1) != 0 : ((q / 3) % NX) == 0;
        const double fv = fixed ? 0.0 : f[q];
        const double rv = y_is_zero ? fv : fv - y[q];
        if (r) r[q] = rv;
        acc[0] = fma(rv, rv, acc[0]);
        acc[1] = fma(fv, fv, acc[1]);
    }
    block_reduce_store<2>(acc, 2, partial + (long long)blockIdx.x * 2);
}

// masked copy (fixed entries -> 0), optional type conversion
// (fix: per-node fixed-component bits, or null for the clamped face x = 0)
template <typename TI, typename TO>
__global__ void masked_convert_kernel(const TI* a, TO* b, long long n, int NX,
                                      const int* __restrict__ halt, const uint8_t* __restrict__ fix)
{
    if (halt != nullptr && *halt != 0) return;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const bool fixed = fix ? ((fix[q / 3] >> (int)(q % 3)) & 1) != 0 : ((q / 3) % NX) == 0;
        b[q] = fixed ? TO(0) : convert<TO>(a[q]);
    }
}

// Dense GEMV for the coarsest solve: x = A b, A row-major FP64 (n x n); one warp per row.
template <typename TB, typename TX>
__global__ void __launch_bounds__(256)
dense_gemv_kernel(const double* __restrict__ A, const TB* __restrict__ b, TX* __restrict__ x, int n,
                  const int* __restrict__ halt)
{
    if (halt != nullptr && *halt != 0) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const double* row = A + (long long)warp * n;
    double s = 0.0;
    for (int c = lane; c < n; c += 32) s = fma(row[c], (double)b[c], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) x[warp] = (TX)s;
}

// Coarsest solve with the inverse of the free-DOF operator (m x m row-major FP64, the
// LDL^T path's Z): x[idx[r]] = sum_c Z[r][c] b[idx[c]], and x = 0 on the fixed DOFs
// (pos < 0). Each CTA stages b's free entries in shared memory (as FP64), every thread's
// index and value loads issued eight at a time; one warp per row. With m even the row is
// read as 16-byte pairs, lane p taking pairs p, p + 32, ... into eight partial sums
// (columns 2p and 2p + 1 of the four pairs in flight), added in a fixed tree; with m odd,
// single columns into four partial sums. Then the warp's lanes in a fixed tree.
template <typename TB, typename TX>
__global__ void __launch_bounds__(256)
free_gemv_kernel(const double* __restrict__ Z, int m, const int* __restrict__ idx, const TB* __restrict__ b,
                 TX* __restrict__ x, int n, const int* __restrict__ pos, const int* __restrict__ halt)
{
    if (halt != nullptr && *halt != 0) return;
    extern __shared__ double gemv_b[];
    for (int c0 = threadIdx.x; c0 < m; c0 += 8 * blockDim.x) {
        int ix[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = c0 + u * blockDim.x;
            ix[u] = c < m ? idx[c] : 0;
        }
        double bv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) bv[u] = (double)b[ix[u]];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = c0 + u * blockDim.x;
            if (c < m) gemv_b[c] = bv[u];
        }
    }
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        if (pos[q] < 0) x[q] = TX(0);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= m) return;
    const double* row = Z + (long long)r * m;
    double s;
    if ((m & 1) == 0) {   // rows start on 16-byte boundaries
        const double2* row2 = reinterpret_cast<const double2*>(row);
        const int m2 = m >> 1;
        double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        int p = lane;
        for (; p + 96 < m2; p += 128) {
            double2 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = row2[p + 32 * u];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[2 * u] = fma(v[u].x, gemv_b[2 * (p + 32 * u)], a[2 * u]);
                a[2 * u + 1] = fma(v[u].y, gemv_b[2 * (p + 32 * u) + 1], a[2 * u + 1]);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (p + 32 * u < m2) {
                const double2 v = row2[p + 32 * u];
                a[2 * u] = fma(v.x, gemv_b[2 * (p + 32 * u)], a[2 * u]);
                a[2 * u + 1] = fma(v.y, gemv_b[2 * (p + 32 * u) + 1], a[2 * u + 1]);
            }
        s = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    } else {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int c = lane;
        for (; c + 96 < m; c += 128) {
            s0 = fma(row[c], gemv_b[c], s0);
            s1 = fma(row[c + 32], gemv_b[c + 32], s1);
            s2 = fma(row[c + 64], gemv_b[c + 64], s2);
            s3 = fma(row[c + 96], gemv_b[c + 96], s3);
        }
        if (c < m) s0 = fma(row[c], gemv_b[c], s0);
        if (c + 32 < m) s1 = fma(row[c + 32], gemv_b[c + 32], s1);
        if (c + 64 < m) s2 = fma(row[c + 64], gemv_b[c + 64], s2);
        s = (s0 + s1) + (s2 + s3);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) x[idx[r]] = (TX)s;
}

// Gauss-Jordan inversion of an SPD matrix without pivoting, two pivots per launch on a
// double-buffered matrix. The step on pivot k maps A to A' with
//   row k:   A'_kq = A_kq / A_kk            (1 / A_kk at q = k)
//   others:  A'_pq = A_pq - A_pk A'_kq      (-A_pk / A_kk at q = k)
// and the step on pivot k+1 applies the same formula to A'. A block owns a 32 x 32
// tile of the output: it forms the two reciprocals, the tile's row-k and row-(k+1)
// factors and its column-k and column-(k+1) values once in shared memory, then every
// entry costs one FMA per pivot. Same arithmetic as one launch per pivot.
constexpr int GJ_T = 32, GJ_R = 8;   // tile edge; thread rows (each thread GJ_T / GJ_R rows)

__device__ __forceinline__ void gj_tile(const double* __restrict__ A, double* __restrict__ D, int n, int k,
                                        int p0, int q0)
{
    __shared__ double rq0[GJ_T], rq1[GJ_T], cp0[GJ_T], cp1[GJ_T], sc[3];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int k1 = k + 1;
    const bool two = k1 < n;
    if (tx == 0 && ty == 0) {
        const double piv0 = 1.0 / A[(long long)k * n + k];
        sc[0] = piv0;
        if (two) {
            const double r0k1 = A[(long long)k * n + k1] * piv0;                  // A'_{k,k1}
            sc[2] = r0k1;
            sc[1] = 1.0 / (A[(long long)k1 * n + k1] - A[(long long)k1 * n + k] * r0k1);   // 1 / A'_{k1,k1}
        }
    }
    __syncthreads();
    if (ty == 0) {   // row factors of the tile's columns
        const int q = q0 + tx;
        if (q < n) {
            const double r0 = ((q == k) ? 1.0 : A[(long long)k * n + q]) * sc[0];
            rq0[tx] = r0;
            if (two) {
                const double a1 = ((q == k) ? 0.0 : A[(long long)k1 * n + q]) - A[(long long)k1 * n + k] * r0;
                rq1[tx] = ((q == k1) ? 1.0 : a1) * sc[1];
            }
        }
    } else if (ty == 1) {   // column values of the tile's rows
        const int p = p0 + tx;
        if (p < n) {
            const double c0 = A[(long long)p * n + k];
            cp0[tx] = c0;
            if (two) cp1[tx] = (p == k) ? sc[2] : (A[(long long)p * n + k1] - c0 * sc[2]);   // A'_{p,k1}
        }
    }
    __syncthreads();
    const int q = q0 + tx;
    if (q >= n) return;
    for (int r = ty; r < GJ_T; r += GJ_R) {
        const int p = p0 + r;
        if (p >= n) break;
        const double a1 = (p == k) ? rq0[tx] : (((q == k) ? 0.0 : A[(long long)p * n + q]) - cp0[r] * rq0[tx]);
        double out = a1;
        if (two) out = (p == k1) ? rq1[tx] : (((q == k1) ? 0.0 : a1) - cp1[r] * rq1[tx]);
        D[(long long)p * n + q] = out;
    }
}

// Pivots k and k+1 (k alone when k+1 == n) from Ain into Aout. Grid: tiles of GJ_T.
__global__ void __launch_bounds__(GJ_T * GJ_R)
gj_step_kernel(const double* __restrict__ Ain, double* __restrict__ Aout, int n, int k)
{
    gj_tile(Ain, Aout, n, k, blockIdx.y * GJ_T, blockIdx.x * GJ_T);
}

// Symmetric blocked Gauss-Jordan (the sweep on a block of SGJ_B pivots per launch),
// keeping only the upper triangle. With the pivots K = {0..k-1} already swept the
// matrix is [[A_KK^-1, A_KK^-1 A_KU], [-A_UK A_KK^-1, S]] (S the Schur complement,
// symmetric), so its upper triangle determines it. Sweeping the next block B with
// P = (M_BB)^-1 and, for p outside B, V_p = M_{p,B} (read from the upper triangle) and
// W_p = P V_p gives, for p <= q:
//   p, q in B:        P
//   p in B, q > B:    (W_q)_p
//   p < B, q in B:    -(W_p)_q
//   otherwise:        M_pq - s V_p . W_q,  s = -1 when q < k (both already swept), else +1.
// Every entry costs SGJ_B FMAs per launch on n^2/2 entries: n^3/2 FMAs in all, half of
// the full-matrix two-pivot form. A block owns a SGJ_T x SGJ_T upper tile and forms W
// for its columns (and rows, when the tile holds the pivot columns). P of each step is
// computed once: one extra block of the launch forms the next pivot block's entries
// with the tile's operations and inverts it while the tiles run, leaving P for the next
// launch in a small buffer (sym_gj_first_kernel makes the first one).
constexpr int SGJ_B = 8, SGJ_T = 64;

// In-place inverse of the bb x bb SPD block S by the sweep (threads 0 .. SGJ_B^2 - 1 own
// one entry each; every thread of the block must call it).
__device__ __forceinline__ void sgj_invert_block(double (*S)[SGJ_B], int bb, int tid)
{
    const int bi = tid / SGJ_B, bj = tid % SGJ_B;
    const bool own = tid < SGJ_B * SGJ_B && bi < bb && bj < bb;
    for (int j = 0; j < bb; ++j) {
        double nv = 0.0;
        if (own) {   // one reciprocal per pivot, the same in every lane (no divergent divides)
            const double ip = 1.0 / S[j][j], rj = S[j][bj] * ip, ci = S[bi][j], old = S[bi][bj];
            if (bi == j) nv = (bj == j) ? ip : rj;
            else nv = (bj == j) ? -ci * ip : old - ci * rj;
        }
        __syncthreads();
        if (own) S[bi][bj] = nv;
        __syncthreads();
    }
}

// P of the first pivot block (pivots 0 .. SGJ_B-1) from the upper triangle of M. One block.
__global__ void __launch_bounds__(256) sym_gj_first_kernel(const double* __restrict__ M, int n, double* __restrict__ Pout)
{
    __shared__ double S[SGJ_B][SGJ_B];
    const int tid = threadIdx.x, bb = min(SGJ_B, n);
    const int bi = tid / SGJ_B, bj = tid % SGJ_B;
    if (tid < SGJ_B * SGJ_B && bi < bb && bj < bb) S[bi][bj] = M[(long long)min(bi, bj) * n + max(bi, bj)];
    __syncthreads();
    sgj_invert_block(S, bb, tid);
    if (tid < SGJ_B * SGJ_B) Pout[tid] = (bi < bb && bj < bb) ? S[bi][bj] : 0.0;
}

// V_p's entry i for the pivot block at k (bb pivots): 0 inside the block and past n.
__device__ __forceinline__ double sgj_v(const double* __restrict__ Min, int n, int k, int bb, int p, int i)
{
    if (p >= n || i >= bb) return 0.0;
    if (p < k) return Min[(long long)p * n + k + i];
    if (p >= k + bb) return Min[(long long)(k + i) * n + p];
    return 0.0;
}

__device__ __forceinline__ void sym_gj_tile(const double* __restrict__ Min, double* __restrict__ Mout, int n, int k,
                                            int tp, int tq, const double* __restrict__ Pin)
{
    __shared__ double Pm[SGJ_B][SGJ_B];
    __shared__ double Vp[SGJ_B][SGJ_T], Vq[SGJ_B][SGJ_T], Wq[SGJ_B][SGJ_T], Wp[SGJ_B][SGJ_T];
    const int tid = threadIdx.y * 16 + threadIdx.x;
    const int bb = min(SGJ_B, n - k);
    const int p0 = tp * SGJ_T, q0 = tq * SGJ_T;
    if (tid < SGJ_B * SGJ_B) Pm[tid / SGJ_B][tid % SGJ_B] = Pin[tid];
    for (int e = tid; e < SGJ_B * SGJ_T; e += 256) {
        const int i = e / SGJ_T, r = e % SGJ_T;
        Vp[i][r] = sgj_v(Min, n, k, bb, p0 + r, i);
        Vq[i][r] = sgj_v(Min, n, k, bb, q0 + r, i);
    }
    // this thread's old entries start its accumulators (loaded early, so that their
    // latency hides behind the dots)
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int p = p0 + threadIdx.y + 16 * a, q = q0 + threadIdx.x + 16 * b;
            acc[a][b] = (p < n && q < n && q >= p) ? Min[(long long)p * n + q] : 0.0;
        }
    __syncthreads();
    // W for the tile's columns, stored as -s W_q (the sign of the update), and for its rows
    // when the tile holds the pivot columns
    const bool need_wp = q0 < k + bb && q0 + SGJ_T > k;
    for (int e = tid; e < SGJ_B * SGJ_T; e += 256) {
        const int i = e / SGJ_T, r = e % SGJ_T;
        double a = 0.0, c = 0.0;
        for (int j = 0; j < bb; ++j) {
            a = fma(Pm[i < bb ? i : 0][j], Vq[j][r], a);
            if (need_wp) c = fma(Pm[i < bb ? i : 0][j], Vp[j][r], c);
        }
        const double w = (i < bb) ? a : 0.0;
        Wq[i][r] = (q0 + r < k) ? w : -w;
        Wp[i][r] = (i < bb) ? c : 0.0;
    }
    __syncthreads();
    // acc_pq += V_p . (-s W_q), register-blocked 4 x 4 (each operand read once per pivot;
    // the pivots run in the same order for every entry)
#pragma unroll
    for (int i = 0; i < SGJ_B; ++i) {
        double vp[4], wq[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) vp[a] = Vp[i][threadIdx.y + 16 * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) wq[b] = Wq[i][threadIdx.x + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fma(vp[a], wq[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int r = threadIdx.y + 16 * a, p = p0 + r;
        if (p >= n) break;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int c = threadIdx.x + 16 * b, q = q0 + c;
            if (q >= n || q < p) continue;
            const bool inp = p >= k && p < k + bb, inq = q >= k && q < k + bb;
            double out;
            if (inp && inq) out = Pm[p - k][q - k];
            else if (inp) out = -Wq[p - k][c];   // q > B, so stored as -W_q
            else if (inq) out = -Wp[q - k][r];
            else out = acc[a][b];
            Mout[(long long)p * n + q] = out;
        }
    }
}

// The next pivot block's P (pivots kn = k + SGJ_B onwards) after this launch's step: its
// entries formed with the tile's operations in the tile's order (so bit-identical to what
// the tile writes), then inverted. Run by one extra block, the first one dispatched,
// while the tiles run.
__device__ __forceinline__ void sym_gj_next_p(const double* __restrict__ Min, int n, int k,
                                              const double* __restrict__ Pin, double* __restrict__ Pout)
{
    __shared__ double Pm[SGJ_B][SGJ_B], Vn[SGJ_B][SGJ_B], Wn[SGJ_B][SGJ_B], Pn[SGJ_B][SGJ_B];
    const int tid = threadIdx.y * 16 + threadIdx.x;
    const int bb = min(SGJ_B, n - k), kn = k + SGJ_B, bbn = min(SGJ_B, n - kn);
    if (bbn <= 0) return;   // uniform over the block
    const int bi = tid / SGJ_B, bj = tid % SGJ_B;
    const bool own = tid < SGJ_B * SGJ_B && bi < bbn && bj < bbn;
    const int p = kn + min(bi, bj), q = kn + max(bi, bj);   // q > k: the update's sign is -
    double acc = own ? Min[(long long)p * n + q] : 0.0;
    if (tid < SGJ_B * SGJ_B) {
        Pm[bi][bj] = Pin[tid];
        Vn[bi][bj] = sgj_v(Min, n, k, bb, kn + bj, bi);   // V_{kn + bj}, entry bi
    }
    __syncthreads();
    if (tid < SGJ_B * SGJ_B) {   // -W of the next block's columns, as the tile stores it
        double w = 0.0;
        for (int j = 0; j < bb; ++j) w = fma(Pm[bi < bb ? bi : 0][j], Vn[j][bj], w);
        Wn[bi][bj] = -((bi < bb) ? w : 0.0);
    }
    __syncthreads();
    if (own) {
        for (int i = 0; i < SGJ_B; ++i) acc = fma(Vn[i][p - kn], Wn[i][q - kn], acc);
        Pn[bi][bj] = acc;
    }
    __syncthreads();
    sgj_invert_block(Pn, bbn, tid);
    if (tid < SGJ_B * SGJ_B) Pout[tid] = (bi < bbn && bj < bbn) ? Pn[bi][bj] : 0.0;
}

// Upper tile b (row-major over the T x T tiles with tq >= tp) -> (tp, tq).
__device__ __forceinline__ void sgj_upper_tile(int b, int T, int& tp, int& tq)
{
    int r = b, row = 0;
    while (row < T && r >= T - row) {
        r -= T - row;
        ++row;
    }
    tp = row;
    tq = row + r;
}

// The band: with A_pq = 0 for |p - q| > band, sweeping the pivots before k leaves
// S = A_UU - A_UK A_KK^-1 A_KU banded too, so V_p = M_{p,B} = 0 (exactly: untouched zero
// entries of A) for p >= k + SGJ_B + band, and W_q = P V_q = 0 there. Step k changes only
// the entries with p, q below sgj_active(n, k, band); the rest still hold A's entries in
// both buffers (both start as A), so only the tiles whose columns start below that bound
// are launched. For the coarsest level's 27-point coupling this leaves about half of the
// n^3/2 work (the swept part fills in; the part ahead stays banded).
__host__ __device__ inline int sgj_active(int n, int k, int band)
{
    return min(n, k + SGJ_B + band);
}

// Pivots k .. k+SGJ_B-1 from Min into Mout (upper triangles) with P = Pin. Grid: block 0
// leaves the next block's P in Pout; blocks 1 .. T (T + 1) / 2 take the upper SGJ_T tiles
// of the leading T x T tiles, T = ceil(sgj_active(n, k, band) / SGJ_T). Only working
// blocks are launched, so the block scheduler's round-robin gives every SM at most
// ceil(tiles / SMs) tiles.
__global__ void __launch_bounds__(256)
sym_gj_kernel(const double* __restrict__ Min, double* __restrict__ Mout, int n, int k, const double* __restrict__ Pin,
              double* __restrict__ Pout, int tiles)
{
    if (blockIdx.x == 0) {
        sym_gj_next_p(Min, n, k, Pin, Pout);
        return;
    }
    int tp, tq;
    sgj_upper_tile((int)blockIdx.x - 1, tiles, tp, tq);
    sym_gj_tile(Min, Mout, n, k, tp, tq, Pin);
}

// The full n x n inverse A from the inverse U over the free DOFs (upper triangle, m x m):
// A[p][q] = U[min(a, b)][max(a, b)] with a = pos[p], b = pos[q]; a fixed DOF (pos -1) gets
// an identity row and column. U and A do not overlap.
__device__ __forceinline__ void sym_expand(const double* __restrict__ U, int m, const int* __restrict__ pos,
                                           double* __restrict__ A, int n, long long e0, long long stride)
{
    const long long nn = (long long)n * n;
    for (long long e = e0; e < nn; e += stride) {
        const int p = (int)(e / n), q = (int)(e % n);
        const int a = pos[p], b = pos[q];
        A[e] = (a < 0 || b < 0) ? (p == q ? 1.0 : 0.0) : U[(long long)min(a, b) * m + max(a, b)];
    }
}

__global__ void sym_expand_kernel(const double* __restrict__ U, int m, const int* __restrict__ pos,
                                  double* __restrict__ A, int n)
{
    sym_expand(U, m, pos, A, n, (long long)blockIdx.x * blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

}  // namespace gf
