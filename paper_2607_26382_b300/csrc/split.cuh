// FP64-class matrix-free K*u without FP64 multiply-adds ("split-integer" operator).
//
// B300 runs FP64 at 1/64 of the FP32 rate, and the dense element product costs 576
// FP64 FMAs per node. The hex8 element stiffness is K0 = s * M with M an integer
// matrix (|M| <= 88 for nu = 0.3), so the product can be formed exactly in FP32:
//
//  1. per node tile, every u value of the tile and its halo is written as
//     u = sign * U * 2^(xmax - 1022 - P), U < 2^P (P = 48 bits kept below the tile's
//     largest exponent xmax), and U is cut into 4 signed digits of 12 bits;
//  2. per digit slice, t = sum_j M_ij d_j over an element's 24 DOFs is an integer of
//     at most 24 * 88 * 4095 < 2^24, so FP32 FMAs compute it exactly;
//  3. the slices are recombined, T = sum_k t_k 2^(12(3-k)), in double-float
//     arithmetic (about 48 bits of the exact integer);
//  4. T is weighted by s*E_e (held as a float pair) and summed over the node's 8
//     elements in double-float arithmetic, then scaled by the tile's power of two
//     into FP64.
// No step uses an FP64 multiply-add or an integer/float conversion instruction in
// the inner loops: on B300 both run on the slow FP64 pipe.
//
// The error is ~2^-44 of the tile's largest |u| times |M|, within a few bits of
// FP64 element-by-element rounding. The acceptance guard keeps the native FP64 kernel.
#pragma once
#include <cuda_runtime.h>

namespace gf {

constexpr int SPX = 16, SPY = 4, SPZ = 2;                  // nodes per tile (128 threads)
constexpr int SPHX = SPX + 2, SPHY = SPY + 2, SPHZ = SPZ + 2;
constexpr int SPHN = SPHX * SPHY * SPHZ;                   // halo nodes (432)
constexpr int SPLIT_P = 48, SPLIT_B = 12, SPLIT_K = 4;
constexpr int SPLIT_VALS = (SPHN * 3 + 127) / 128;         // halo values held per thread

struct MParam {
    float m[576];   // integer matrix M = K0 / s, row-major 24x24
};

// E as a float pair (hi + lo = s * E_e to ~48 bits).
__global__ void edf_kernel(const double* __restrict__ E, double s, float2* __restrict__ out, long long n)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double v = s * E[e];
    const float hi = (float)v;
    out[e] = make_float2(hi, (float)(v - (double)hi));
}

__device__ __forceinline__ void two_sum_acc(float& ah, float& al, float ph, float pl)
{
    const float s = ah + ph;
    const float bb = s - ah;
    const float err = (ah - (s - bb)) + (ph - bb);
    ah = s;
    al += pl + err;
}

// 2^k as a float for k in [-126, 127], from its exponent bits
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

// DD = false: y (FP64). DD = true: yd, the result as a normalised double-float pair
// (hi + lo), for the double-float Gram-Schmidt passes.
template <bool DD>
__global__ void __launch_bounds__(128)
apply_split_kernel(const double* __restrict__ u, double* __restrict__ y, float2* __restrict__ yd,
                   const float2* __restrict__ Edf, GridDims d, const __grid_constant__ MParam M,
                   const int* __restrict__ halt)
{
    if (halt != nullptr && *halt != 0) return;
    __shared__ float dig[SPLIT_K][SPHN * 3];
    __shared__ int wmax[4];
    const int NX = d.nx + 1, NY = d.ny + 1, NZ = d.nz + 1;
    const int i0 = blockIdx.x * SPX, j0 = blockIdx.y * SPY, k0 = blockIdx.z * SPZ;
    const int tid = threadIdx.x + SPX * (threadIdx.y + SPY * threadIdx.z);

    // pass 1: the tile's halo values and their largest biased exponent
    long long bits[SPLIT_VALS];
    int emax = 0;
#pragma unroll
    for (int r = 0; r < SPLIT_VALS; ++r) {
        const int q = tid + 128 * r;
        bits[r] = 0;
        if (q < SPHN * 3) {
            const int c = q % 3, hn = q / 3;
            const int hx = hn % SPHX, hy = (hn / SPHX) % SPHY, hz = hn / (SPHX * SPHY);
            const int gi = i0 - 1 + hx, gj = j0 - 1 + hy, gk = k0 - 1 + hz;
            if (gi >= 1 && gi < NX && gj >= 0 && gj < NY && gk >= 0 && gk < NZ) {
                bits[r] = __double_as_longlong(u[3 * ((long long)gi + (long long)NX * (gj + (long long)NY * gk)) + c]);
                emax = max(emax, (int)((bits[r] >> 52) & 0x7ff));
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    if ((tid & 31) == 0) wmax[tid >> 5] = emax;
    __syncthreads();
    const int xmax = max(max(wmax[0], wmax[1]), max(wmax[2], wmax[3]));

    // pass 2: signed 12-bit digits on the common exponent
#pragma unroll
    for (int r = 0; r < SPLIT_VALS; ++r) {
        const int q = tid + 128 * r;
        if (q < SPHN * 3) {
            const long long b = bits[r];
            const int e = (int)((b >> 52) & 0x7ff);
            const long long mant = (b & 0xFFFFFFFFFFFFFLL) | (e ? (1LL << 52) : 0LL);
            const int shift = xmax - (e ? e : 1) + 53 - SPLIT_P;
            const long long U = (shift >= 63) ? 0LL : (mant >> shift);
            const float sg = (b < 0) ? -1.f : 1.f;
            // 0 <= digit < 2^12: (2^23 | digit) as a float is 2^23 + digit exactly, so the
            // digit becomes a float without an integer-to-float conversion instruction
#pragma unroll
            for (int k = 0; k < SPLIT_K; ++k) {
                const int dgt = (int)((U >> (SPLIT_B * (SPLIT_K - 1 - k))) & ((1 << SPLIT_B) - 1));
                dig[k][q] = sg * (__int_as_float(0x4B000000 | dgt) - 8388608.0f);
            }
        }
    }
    __syncthreads();

    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    const int gi = i0 + tx, gj = j0 + ty, gk = k0 + tz;
    if (gi >= NX || gj >= NY || gk >= NZ) return;
    const long long n = gi + (long long)NX * (gj + (long long)NY * gk);
    if (gi == 0) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            if (DD) yd[3 * n + r] = make_float2(0.f, 0.f);
            else y[3 * n + r] = 0.0;
        }
        return;
    }

    // pass 3: exact integer element products, slice by slice. Each digit of the 27
    // neighbouring nodes feeds every (element, row) accumulator that uses it, so the
    // 24 accumulators form independent FMA chains.
    // T = sum_k t_k 2^(12 (3-k)) kept as a float pair (Horner: T <- 4096 T + t_k, the
    // scaling exact and the addition by TwoSum), ~48 bits of the exact integer
    float Th[8][3], Tl[8][3];
#pragma unroll
    for (int e = 0; e < 8; ++e)
#pragma unroll
        for (int r = 0; r < 3; ++r) Th[e][r] = Tl[e][r] = 0.f;
#pragma unroll 1
    for (int k = 0; k < SPLIT_K; ++k) {
        float t[8][3];
#pragma unroll
        for (int e = 0; e < 8; ++e)
#pragma unroll
            for (int r = 0; r < 3; ++r) t[e][r] = 0.f;
#pragma unroll
        for (int oz = 0; oz < 3; ++oz)
#pragma unroll
            for (int oy = 0; oy < 3; ++oy)
#pragma unroll
                for (int ox = 0; ox < 3; ++ox) {
                    const int hn = (tx + ox) + SPHX * ((ty + oy) + SPHY * (tz + oz));
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float dv = dig[k][3 * hn + c];
#pragma unroll
                        for (int ez = 0; ez < 2; ++ez)
#pragma unroll
                            for (int ey = 0; ey < 2; ++ey)
#pragma unroll
                                for (int ex = 0; ex < 2; ++ex) {
                                    const int bx = ox - ex, by = oy - ey, bz = oz - ez;
                                    if (bx < 0 || bx > 1 || by < 0 || by > 1 || bz < 0 || bz > 1) continue;
                                    const int e = ex + 2 * (ey + 2 * ez);
                                    const int a = local_index(1 - ex, 1 - ey, 1 - ez);
                                    const int bl = local_index(bx, by, bz);
#pragma unroll
                                    for (int r = 0; r < 3; ++r)
                                        t[e][r] = fmaf(M.m[(3 * a + r) * 24 + 3 * bl + c], dv, t[e][r]);
                                }
                    }
                }
#pragma unroll
        for (int e = 0; e < 8; ++e)
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const float a = Th[e][r] * 4096.0f, b = Tl[e][r] * 4096.0f, tv = t[e][r];
                const float s = a + tv;
                const float bb = s - a;
                Th[e][r] = s;
                Tl[e][r] = b + ((a - (s - bb)) + (tv - bb));
            }
    }

    // pass 4: weight by s*E_e and sum over the elements in double-float
    float ah[3] = {0.f, 0.f, 0.f}, al[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int ez = 0; ez < 2; ++ez)
#pragma unroll
        for (int ey = 0; ey < 2; ++ey)
#pragma unroll
            for (int ex = 0; ex < 2; ++ex) {
                const int e = ex + 2 * (ey + 2 * ez);
                const int cx = gi - 1 + ex, cy = gj - 1 + ey, cz = gk - 1 + ez;
                if (cx < 0 || cx >= d.nx || cy < 0 || cy >= d.ny || cz < 0 || cz >= d.nz) continue;
                const float2 E = Edf[cx + (long long)d.nx * (cy + (long long)d.ny * cz)];
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    const float th = Th[e][r], tl = Tl[e][r];
                    const float ph = th * E.x;
                    float pl = fmaf(th, E.x, -ph);
                    pl = fmaf(th, E.y, pl);
                    pl = fmaf(tl, E.x, pl);
                    two_sum_acc(ah[r], al[r], ph, pl);
                }
            }
    if (DD) {
        // scale by 2^(xmax - 1022 - P) in two exact power-of-two steps (the factor
        // itself may lie outside the float range while the result does not), then
        // renormalise the pair (Fast2Sum; |hi| >= |lo|)
        const int k = xmax - 1022 - SPLIT_P;
        const int k1 = k / 2, k2 = k - k1;
        const float f1 = pow2f(max(-126, min(127, k1))), f2 = pow2f(max(-126, min(127, k2)));
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float h0 = ah[r] * f1 * f2, l0 = al[r] * f1 * f2;
            const float h = h0 + l0;
            yd[3 * n + r] = make_float2(h, l0 - (h - h0));
        }
        return;
    }
    // 2^(xmax - 1022 - P) built from its exponent bits when it is a normal number
    const int sexp = xmax - 1022 - SPLIT_P + 1023;
    const double scale = (sexp >= 1) ? __longlong_as_double((long long)sexp << 52) : scalbn(1.0, sexp - 1023);
#pragma unroll
    for (int r = 0; r < 3; ++r) y[3 * n + r] = ((double)ah[r] + (double)al[r]) * scale;
}

}  // namespace gf
