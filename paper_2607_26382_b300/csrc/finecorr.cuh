// Fine-level adaptive correction after the V-cycle (Table solver-config): with z the
// V-cycle's output and r = v - K z, run k steps of an inner FGMRES(k) from d = 0 on
// K d = r, preconditioned by the 3x3 node-block Jacobi operator (first_sweep_kernel with
// omega = 1), and apply z += d only if the recomputed residual norm ||r - K d|| is below
// ||r||. Everything runs on the device (the decisions included), so the correction sits
// inside the captured Arnoldi-step graphs.
//
// Each inner step: Z_j = D^{-1} V_j, w = K Z_j (written into V_{j+1}), two classical
// Gram-Schmidt passes, the Givens update of the k x k least-squares problem, and
// V_{j+1} = w / ||w||. A thread accumulates its few rows in the vectors' precision (FP32
// for the mixed form: FP64 FMAs run at 1/64 rate on this GPU, and a dozen rows per thread
// lose nothing an FP32 inner solve keeps), the warp sums follow in that precision, and
// the block and grid sums are FP64: a pass's per-block partial sums are summed in block
// order by the last block to arrive (atomic ticket after a fence).
// Stop rules as in the outer solver: a zero rotated pivot drops the step (breakdown),
// h_{j+1,j} <= 1e-14 ||K z_j|| keeps it and stops, a zero projected residual stops.
#pragma once
#include <cuda_runtime.h>
#include <type_traits>

namespace gf {

constexpr int FC_MAX = 32, FC_THREADS = 256, FC_SLOTS = FC_MAX + 2;

struct FcState {
    double H[(FC_MAX + 1) * FC_MAX];   // rotated Hessenberg, column-major, ld FC_MAX + 1
    double g[FC_MAX + 1], cs[FC_MAX], sn[FC_MAX], y[FC_MAX];
    double h1[FC_SLOTS];               // pass-1 dots; slot FC_MAX + 1: ||w||^2 before orthogonalisation
    double h2[FC_MAX + 1];             // pass-2 dots
    double beta, hnext;
    int J;          // columns kept
    int stop;       // 1: the remaining inner steps are skipped
    int skip;       // 1: the whole correction is skipped (zero residual, or the outer solve halted)
    int accept;     // the correction lowered the recomputed residual norm
    unsigned ticket;
};

// block-sum cnt values of every thread's acc[] and write them to partial[blockIdx.x][];
// returns true in the block that arrives last (after all blocks' partials are visible)
template <typename T>
using FcAcc = typename std::conditional<sizeof(T) == sizeof(float), float, double>::type;

template <int K, typename A>
__device__ __forceinline__ bool fc_block_partials(const A (&acc)[K], int cnt, double* __restrict__ partial,
                                                 unsigned* ticket)
{
    __shared__ double red[FC_THREADS / 32][K];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        A v = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][i] = (double)v;
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
        double s = 0.0;
        for (int w = 0; w < FC_THREADS / 32; ++w) s += red[w][threadIdx.x];
        partial[(long long)blockIdx.x * FC_SLOTS + threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// In the last block: fin[i] = sum over blocks of partial[b][i], i < cnt, by all threads --
// warp w takes slots w, w + 8, ..., lane l the blocks l, l + 32, ... (L2 loads), then a
// fixed shuffle tree: the same order on every run. Ends with a barrier.
__device__ __forceinline__ void fc_finish_sums(const double* __restrict__ partial, int nb, int cnt, double* fin)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < cnt; i += FC_THREADS / 32) {
        double s = 0.0;
        for (int b = lane; b < nb; b += 32) s += __ldcg(partial + (long long)b * FC_SLOTS + i);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) fin[i] = s;
    }
    __syncthreads();
}

// beta = ||r||; skip when it is zero or the outer solve has halted
template <typename T>
__global__ void __launch_bounds__(FC_THREADS) fc_start_kernel(const T* __restrict__ r, long long n, FcState* st,
                                                             double* __restrict__ partial, const int* __restrict__ halt)
{
    using A = FcAcc<T>;
    A acc[1] = {A(0)};
    for (long long i = (long long)blockIdx.x * FC_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * FC_THREADS)
        acc[0] = fma((A)r[i], (A)r[i], acc[0]);
    __shared__ double fin[1];
    if (!fc_block_partials<1>(acc, 1, partial, &st->ticket)) return;   // block-uniform
    fc_finish_sums(partial, gridDim.x, 1, fin);
    if (threadIdx.x == 0) {
        const double b = sqrt(fin[0]);
        const bool halted = halt != nullptr && *halt != 0;
        st->beta = b;
        st->g[0] = b;
        st->J = 0;
        st->accept = 0;
        st->skip = (halted || !(b > 0.0)) ? 1 : 0;
        st->stop = st->skip;
        st->ticket = 0u;
    }
}

// V_0 = r / beta
template <typename T>
__global__ void fc_scale_kernel(const T* __restrict__ r, T* __restrict__ v0, long long n, const FcState* st)
{
    if (st->stop) return;
    const FcAcc<T> inv = (FcAcc<T>)(1.0 / st->beta);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v0[i] = (T)((FcAcc<T>)r[i] * inv);
}

// pass 1: h1_i = V_i . w (i <= j) and ||w||^2
template <typename T>
__global__ void __launch_bounds__(FC_THREADS) fc_dots1_kernel(const T* __restrict__ V, long long ld,
                                                             const T* __restrict__ w, long long n, int j, FcState* st,
                                                             double* __restrict__ partial)
{
    if (st->stop) return;
    using A = FcAcc<T>;
    A acc[FC_SLOTS];
#pragma unroll
    for (int i = 0; i < FC_SLOTS; ++i) acc[i] = A(0);
    for (long long r = (long long)blockIdx.x * FC_THREADS + threadIdx.x; r < n; r += (long long)gridDim.x * FC_THREADS) {
        const A wr = (A)w[r];
#pragma unroll
        for (int i = 0; i <= FC_MAX; ++i)
            if (i <= j) acc[i] = fma((A)V[(long long)i * ld + r], wr, acc[i]);
        acc[FC_MAX + 1] = fma(wr, wr, acc[FC_MAX + 1]);
    }
    __shared__ double fin[FC_SLOTS];
    if (!fc_block_partials<FC_SLOTS>(acc, FC_SLOTS, partial, &st->ticket)) return;   // block-uniform
    fc_finish_sums(partial, gridDim.x, FC_SLOTS, fin);
    if (threadIdx.x <= j || threadIdx.x == FC_MAX + 1) st->h1[threadIdx.x] = fin[threadIdx.x];
    if (threadIdx.x == 0) st->ticket = 0u;
}

// pass 2: w -= sum_i h1_i V_i, then h2_i = V_i . w
template <typename T>
__global__ void __launch_bounds__(FC_THREADS) fc_dots2_kernel(const T* __restrict__ V, long long ld, T* __restrict__ w,
                                                             long long n, int j, FcState* st,
                                                             double* __restrict__ partial)
{
    if (st->stop) return;
    using A = FcAcc<T>;
    __shared__ A h[FC_MAX + 1];
    if (threadIdx.x <= j) h[threadIdx.x] = (A)st->h1[threadIdx.x];
    __syncthreads();
    A acc[FC_MAX + 1];
#pragma unroll
    for (int i = 0; i <= FC_MAX; ++i) acc[i] = A(0);
    for (long long r = (long long)blockIdx.x * FC_THREADS + threadIdx.x; r < n; r += (long long)gridDim.x * FC_THREADS) {
        A wr = (A)w[r];
#pragma unroll
        for (int i = 0; i <= FC_MAX; ++i)
            if (i <= j) wr = fma(-h[i], (A)V[(long long)i * ld + r], wr);
        w[r] = (T)wr;
        const A wt = (A)w[r];
#pragma unroll
        for (int i = 0; i <= FC_MAX; ++i)
            if (i <= j) acc[i] = fma((A)V[(long long)i * ld + r], wt, acc[i]);
    }
    __shared__ double fin[FC_MAX + 1];
    if (!fc_block_partials<FC_MAX + 1>(acc, j + 1, partial, &st->ticket)) return;   // block-uniform
    fc_finish_sums(partial, gridDim.x, j + 1, fin);
    if (threadIdx.x <= j) st->h2[threadIdx.x] = fin[threadIdx.x];
    if (threadIdx.x == 0) st->ticket = 0u;
}

// w -= sum_i h2_i V_i, ||w||; the last block updates the least-squares problem
template <typename T>
__global__ void __launch_bounds__(FC_THREADS) fc_norm_kernel(const T* __restrict__ V, long long ld, T* __restrict__ w,
                                                            long long n, int j, int steps, FcState* st,
                                                            double* __restrict__ partial)
{
    if (st->stop) return;
    using A = FcAcc<T>;
    __shared__ A h[FC_MAX + 1];
    if (threadIdx.x <= j) h[threadIdx.x] = (A)st->h2[threadIdx.x];
    __syncthreads();
    A acc[1] = {A(0)};
    for (long long r = (long long)blockIdx.x * FC_THREADS + threadIdx.x; r < n; r += (long long)gridDim.x * FC_THREADS) {
        A wr = (A)w[r];
#pragma unroll
        for (int i = 0; i <= FC_MAX; ++i)
            if (i <= j) wr = fma(-h[i], (A)V[(long long)i * ld + r], wr);
        w[r] = (T)wr;
        const A wt = (A)w[r];
        acc[0] = fma(wt, wt, acc[0]);
    }
    __shared__ double fin[1];
    if (!fc_block_partials<1>(acc, 1, partial, &st->ticket)) return;   // block-uniform
    fc_finish_sums(partial, gridDim.x, 1, fin);
    if (threadIdx.x == 0) {
        const double hn = sqrt(fin[0]);
        const int ldh = FC_MAX + 1;
        double* col = st->H + (long long)j * ldh;
        for (int i = 0; i <= j; ++i) col[i] = st->h1[i] + st->h2[i];
        col[j + 1] = hn;
        for (int i = 0; i < j; ++i) {   // earlier rotations
            const double a = col[i], b = col[i + 1];
            col[i] = st->cs[i] * a + st->sn[i] * b;
            col[i + 1] = -st->sn[i] * a + st->cs[i] * b;
        }
        const double a = col[j], b = col[j + 1];
        const double rho = hypot(a, b);
        st->ticket = 0u;
        if (rho == 0.0) {   // degenerate column: breakdown, the step is dropped
            st->stop = 1;
            return;
        }
        st->cs[j] = a / rho;
        st->sn[j] = b / rho;
        col[j] = rho;
        col[j + 1] = 0.0;
        st->g[j + 1] = -st->sn[j] * st->g[j];
        st->g[j] = st->cs[j] * st->g[j];
        st->J = j + 1;
        st->hnext = hn;
        if (st->g[j + 1] == 0.0 || j + 1 >= steps || hn <= 1e-14 * sqrt(st->h1[FC_MAX + 1])) st->stop = 1;
    }
}

// V_{j+1} = w / h_{j+1,j} in place
template <typename T>
__global__ void fc_vscale_kernel(T* __restrict__ w, long long n, const FcState* st)
{
    if (st->stop) return;
    const FcAcc<T> inv = (FcAcc<T>)(1.0 / st->hnext);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        w[i] = (T)((FcAcc<T>)w[i] * inv);
}

// y = R^{-1} g over the J kept columns
__global__ void fc_backsolve_kernel(FcState* st)
{
    if (threadIdx.x != 0 || st->skip) return;
    const int ldh = FC_MAX + 1;
    const int J = st->J;
    for (int i = J - 1; i >= 0; --i) {
        double s = st->g[i];
        for (int c = i + 1; c < J; ++c) s -= st->H[(long long)c * ldh + i] * st->y[c];
        st->y[i] = s / st->H[(long long)i * ldh + i];
    }
}

// d = sum_{i<J} y_i Z_i
template <typename T>
__global__ void fc_combine_kernel(const T* __restrict__ Z, long long ld, T* __restrict__ d, long long n,
                                  const FcState* st)
{
    if (st->skip) return;
    using A = FcAcc<T>;
    __shared__ A ys[FC_MAX];
    const int J = st->J;
    if (threadIdx.x < J) ys[threadIdx.x] = (A)st->y[threadIdx.x];
    __syncthreads();
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        A s = A(0);
        for (int i = 0; i < J; ++i) s = fma(ys[i], (A)Z[(long long)i * ld + r], s);
        d[r] = (T)s;
    }
}

// accept iff ||r - q|| < beta (q = K d)
template <typename T>
__global__ void __launch_bounds__(FC_THREADS) fc_accept_kernel(const T* __restrict__ r, const T* __restrict__ q,
                                                              long long n, FcState* st, double* __restrict__ partial)
{
    if (st->skip) return;
    using A = FcAcc<T>;
    A acc[1] = {A(0)};
    for (long long i = (long long)blockIdx.x * FC_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * FC_THREADS) {
        const A e = (A)r[i] - (A)q[i];
        acc[0] = fma(e, e, acc[0]);
    }
    __shared__ double fin[1];
    if (!fc_block_partials<1>(acc, 1, partial, &st->ticket)) return;   // block-uniform
    fc_finish_sums(partial, gridDim.x, 1, fin);
    if (threadIdx.x == 0) {
        st->accept = sqrt(fin[0]) < st->beta ? 1 : 0;
        st->ticket = 0u;
    }
}

// z += d when accepted
template <typename T>
__global__ void fc_apply_kernel(double* __restrict__ z, const T* __restrict__ d, long long n, const FcState* st)
{
    if (st->skip || !st->accept) return;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        z[i] += (double)d[i];
}

}  // namespace gf
