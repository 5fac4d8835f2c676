// Split-integer FP64-class K*u with the element products on the tensor cores.
//
// Same number format as apply_split_kernel (split.cuh): K0 = s * M with integer M
// (|M| <= 88), every u value written on a common exponent of its region as a
// P = 55-bit integer, cut into 5 signed 11-bit digits. A digit is an exact fp16
// number and M is exact in fp16, and an element's 24-term digit product is below
// 24 * 88 * 2047 < 2^24, so an fp16 MMA with FP32 accumulation forms every
// slice's element product M d_e exactly. The batched contraction per element layer
// of a tile is a (16 elements x 32) x (32 x 24) product per warp and slice
// (mma.sync m16n8k16, K and N padded from 24; the D fragments stay in registers).
//
// Work per CTA: an (x, y) tile of 16 x 8 elements walking a chunk of element layers
// in z. For each element layer:
//   1. the next node layer's u values -> 5 digit slices in shared memory, stored as
//      x-adjacent pairs (the A fragments load whole 32-bit pairs);
//   2. each warp (one row of 16 elements) runs 5 slices x 3 output components x
//      2 K-steps of MMAs; slice k's exact result t_k times 2^(11(4-k)) is an exact
//      float, so s E_e sum_k t_k 2^(11(4-k)) is accumulated in registers as a
//      double-float: slices 0..2 through exact products (FMA) and TwoSum, slices 3
//      and 4 (below 2^-33 of slice 0) into the low word;
//   3. the 24 weighted element rows go to shared memory, and every node of the tile
//      whose 8 elements are now all done sums them in a fixed order (deterministic)
//      and writes y (FP64) or the normalised pair (for the double-float CGS2).
// Node tile: 15 x 7 nodes (x, y) per 16 x 8 elements; neighbouring tiles recompute
// one shared element column/row.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>

namespace gf {

constexpr int TC_EX = 16, TC_EY = 8;                 // elements per layer of a tile
constexpr int TC_NX = TC_EX - 1, TC_NY = TC_EY - 1;  // nodes written per layer
constexpr int TC_CZ = 7;                             // node layers per CTA
constexpr int TC_P = 55, TC_B = 11, TC_K = 5;        // bits kept, digit bits, slices
constexpr int TC_WX = TC_EX + 1, TC_WY = TC_EY + 1;  // node window per layer
constexpr int TC_PAIRS = TC_EX;                      // x-pairs (wx, wx+1), wx < 16
// pair words of one slot: [slice][comp][wy][pair]; the slot stride is padded so the
// four (y, z) lanes of an A-fragment load fall in distinct banks
constexpr int TC_SLOT_WORDS = TC_K * 3 * TC_WY * TC_PAIRS + 8;
constexpr int TC_THREADS = 32 * TC_EY;

struct TcBFrag {
    unsigned int w[12][32];   // [t = out comp][kstep][2] packed half2 of M', by lane (device memory)
};

// Shared-memory layout (dynamic): two digit slots, two element-result layers.
struct TcSmem {
    unsigned int pairs[2][TC_SLOT_WORDS];
    float2 R[2][TC_EX * TC_EY][24];   // s E_e T, row a' * 3 + comp, a' = x + 2y + 4z
    unsigned int bfrag[12][32];       // B fragments, lane-major (conflict-free per lane)
    int wmax[TC_THREADS / 32];
};

// values of one node layer's window held by a thread between load and digit split
constexpr int TC_LAYER_VALS = TC_WX * TC_WY * 3;                       // 459
constexpr int TC_PER_THREAD = (TC_LAYER_VALS + TC_THREADS - 1) / TC_THREADS;   // 2

__device__ __forceinline__ void mma_f16_16816(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                              unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// biased exponent of a double's bits (0 for zero / denormal)
__device__ __forceinline__ int tc_exp(long long b) { return (int)((b >> 52) & 0x7ff); }

// The 5 signed 11-bit digits of u on the common exponent xmax, as fp16 bit patterns.
__device__ __forceinline__ void tc_digits(long long b, int xmax, unsigned short (&h)[TC_K])
{
    const int e = tc_exp(b);
    const long long mant = (b & 0xFFFFFFFFFFFFFLL) | (e ? (1LL << 52) : 0LL);
    const int shift = xmax - (e ? e : 1) + 53 - TC_P;   // may be -2 .. 63+
    const long long U = shift >= 63 ? 0LL : (shift >= 0 ? (mant >> shift) : (mant << (-shift)));
    const unsigned short sg = (b < 0) ? 0x8000 : 0;
#pragma unroll
    for (int k = 0; k < TC_K; ++k) {
        const int dgt = (int)((U >> (TC_B * (TC_K - 1 - k))) & ((1 << TC_B) - 1));
        // the digit as a float without a conversion instruction ((2^23 | d) - 2^23); its
        // fp16 pattern is the float's exponent rebiased (127 -> 15) and top 10 mantissa
        // bits, exact for d < 2^11
        const unsigned fb = __float_as_uint(__int_as_float(0x4B000000 | dgt) - 8388608.0f);
        h[k] = dgt ? (unsigned short)(((fb >> 13) - (112u << 10)) | sg) : (unsigned short)0;
    }
}

template <bool DD>
__global__ void __launch_bounds__(TC_THREADS, 3)
apply_split_tc_kernel(const double* __restrict__ u, double* __restrict__ y, float2* __restrict__ yd,
                      const float2* __restrict__ Edf, GridDims d, const TcBFrag* __restrict__ B,
                      const int* __restrict__ halt)
{
    if (halt != nullptr && *halt != 0) return;
    extern __shared__ __align__(16) unsigned char tc_smem_raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(tc_smem_raw);
    const int NX = d.nx + 1, NY = d.ny + 1, NZ = d.nz + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ex0 = blockIdx.x * TC_NX - 1, ey0 = blockIdx.y * TC_NY - 1;   // first element (may be -1)
    const int kz0 = blockIdx.z * TC_CZ;                                   // first node layer written
    const int kz1 = min(kz0 + TC_CZ, NZ);                                 // one past the last

    // ---- region exponent: node window x layers kz0-1 .. kz1 (free nodes only)
    // (lane-indexed reads of a kernel parameter would serialise in the constant cache)
    for (int q = tid; q < 12 * 32; q += TC_THREADS) S.bfrag[q / 32][q % 32] = B->w[q / 32][q % 32];
    int emax = 0;
    {
        // only the high words (sign, exponent) are read, 9 in flight per thread
        const int* uhi = reinterpret_cast<const int*>(u) + 1;
        const int nv = TC_LAYER_VALS * (kz1 - kz0 + 2);
        constexpr int UNR = 9;
        for (int q0 = tid; q0 < nv; q0 += UNR * TC_THREADS) {
            int hw[UNR];
#pragma unroll
            for (int v = 0; v < UNR; ++v) {
                const int q = q0 + v * TC_THREADS;
                hw[v] = 0;
                if (q < nv) {
                    const int c = q % 3, r = q / 3;
                    const int wx = r % TC_WX, wy = (r / TC_WX) % TC_WY, l = r / (TC_WX * TC_WY);
                    const int gi = ex0 + wx, gj = ey0 + wy, gk = kz0 - 1 + l;
                    if (gi >= 1 && gi < NX && gj >= 0 && gj < NY && gk >= 0 && gk < NZ)
                        hw[v] = uhi[2 * (3 * ((long long)gi + (long long)NX * (gj + (long long)NY * gk)) + c)];
                }
            }
#pragma unroll
            for (int v = 0; v < UNR; ++v) emax = max(emax, (hw[v] >> 20) & 0x7ff);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        if (lane == 0) S.wmax[warp] = emax;
        __syncthreads();
        emax = S.wmax[0];
#pragma unroll
        for (int w = 1; w < TC_THREADS / 32; ++w) emax = max(emax, S.wmax[w]);
    }
    const int xmax = emax;

    // node layer gk's window values into registers (issued early, used after the MMAs)
    auto load_layer = [&](int gk, long long (&bits)[TC_PER_THREAD]) {
#pragma unroll
        for (int v = 0; v < TC_PER_THREAD; ++v) {
            const int q = tid + v * TC_THREADS;
            bits[v] = 0;
            if (q < TC_LAYER_VALS) {
                const int c = q % 3, r = q / 3;
                const int wx = r % TC_WX, wy = r / TC_WX;
                const int gi = ex0 + wx, gj = ey0 + wy;
                if (gi >= 1 && gi < NX && gj >= 0 && gj < NY && gk >= 0 && gk < NZ)
                    bits[v] = __double_as_longlong(u[3 * ((long long)gi + (long long)NX * (gj + (long long)NY * gk)) + c]);
            }
        }
    };
    // their digits into slot s (pairs (wx, wx+1) of the window row)
    auto store_digits = [&](const long long (&bits)[TC_PER_THREAD], int s) {
        unsigned short* P = reinterpret_cast<unsigned short*>(S.pairs[s]);
#pragma unroll
        for (int v = 0; v < TC_PER_THREAD; ++v) {
            const int q = tid + v * TC_THREADS;
            if (q >= TC_LAYER_VALS) continue;
            const int c = q % 3, r = q / 3;
            const int wx = r % TC_WX, wy = r / TC_WX;
            unsigned short h[TC_K];
            tc_digits(bits[v], xmax, h);
#pragma unroll
            for (int k = 0; k < TC_K; ++k) {
                const int row = ((k * 3 + c) * TC_WY + wy) * TC_PAIRS;
                if (wx < TC_PAIRS) P[2 * (row + wx) + 0] = h[k];          // low half of pair wx
                if (wx >= 1) P[2 * (row + wx - 1) + 1] = h[k];            // high half of pair wx-1
            }
        }
    };

    const int g = lane >> 2, cq = lane & 3;
    const int ly = warp;                       // this warp's element row
    const int yo = cq & 1, zo = cq >> 1;       // A-fragment node offsets of this lane
    // s E_e of this lane's two elements (g, g+8 of row ly) in element layer ez
    auto load_e = [&](int ez, float2 (&E)[2]) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int ex = ex0 + g + 8 * half, ey = ey0 + ly;
            E[half] = make_float2(0.f, 0.f);
            if (ez >= 0 && ez < d.nz && ex >= 0 && ex < d.nx && ey >= 0 && ey < d.ny)
                E[half] = Edf[ex + (long long)d.nx * (ey + (long long)d.ny * ez)];
        }
    };
    float2 Ew[2];
    load_e(kz0 - 1, Ew);
    __syncthreads();                           // bfrag staged
    unsigned int bw[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) bw[q] = S.bfrag[q][lane];

    // prologue: digits of node layers kz0-1 and kz0
    {
        long long bits[TC_PER_THREAD];
        load_layer(kz0 - 1, bits);
        store_digits(bits, (kz0 - 1) & 1);
        load_layer(kz0, bits);
        store_digits(bits, kz0 & 1);
    }
    __syncthreads();

    for (int ez = kz0 - 1; ez < kz1; ++ez) {
        // slots hold node layers ez and ez+1; layer ez+2 is fetched now and split after
        // the MMAs (into the slot of layer ez)
        long long nxt[TC_PER_THREAD];
        const bool more = ez + 1 < kz1;
        if (more) load_layer(ez + 2, nxt);
        float2 Enext[2];
        load_e(ez + 1, Enext);   // one layer ahead: used by the next iteration's MMAs

        float2* R = S.R[ez & 1][0];
        const bool layer_exists = (ez >= 0 && ez < d.nz);
        if (layer_exists) {
            // accumulator (double-float) of this lane's 12 outputs: [t][v], v = 0,1 -> element
            // g (a' = 2cq + v), v = 2,3 -> element g+8
            float Ah[3][4], Al[3][4];
#pragma unroll
            for (int k = 0; k < TC_K; ++k) {
                const unsigned* p0 = S.pairs[(ez + zo) & 1];
                // A fragments: row g / g+8 = element x, cols = (x-pair) at (y = yo, z = zo)
                unsigned a[3][2];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int base = ((k * 3 + c) * TC_WY + (ly + yo)) * TC_PAIRS;
                    a[c][0] = p0[base + g];
                    a[c][1] = p0[base + g + 8];
                }
                // s E_e 2^(11 (4 - k)) as a float pair (exact power-of-two scaling)
                const float sk = __int_as_float((127 + TC_B * (TC_K - 1 - k)) << 23);
                const float eh0 = Ew[0].x * sk, el0 = Ew[0].y * sk, eh1 = Ew[1].x * sk, el1 = Ew[1].y * sk;
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    float acc[4] = {0.f, 0.f, 0.f, 0.f};
                    // K-step 0: cols 0..7 = comp 0, cols 8..15 = comp 1; K-step 1: comp 2, padding
                    mma_f16_16816(acc, a[0][0], a[0][1], a[1][0], a[1][1], bw[4 * t + 0], bw[4 * t + 1]);
                    mma_f16_16816(acc, a[2][0], a[2][1], 0u, 0u, bw[4 * t + 2], bw[4 * t + 3]);
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const float eh = v < 2 ? eh0 : eh1, el = v < 2 ? el0 : el1;
                        const float tv = acc[v];
                        if (k == 0) {
                            const float p = tv * eh;
                            Ah[t][v] = p;
                            Al[t][v] = fmaf(tv, el, fmaf(tv, eh, -p));
                        } else if (k <= 2) {
                            const float p = tv * eh;
                            const float e = fmaf(tv, el, fmaf(tv, eh, -p));
                            const float hs = Ah[t][v] + p;
                            const float bb = hs - Ah[t][v];
                            const float r = (Ah[t][v] - (hs - bb)) + (p - bb);
                            Ah[t][v] = hs;
                            Al[t][v] += r + e;
                        } else {
                            Al[t][v] = fmaf(tv, eh, Al[t][v]);
                        }
                    }
                }
            }
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float2* Re = R + (ly * TC_EX + g + 8 * half) * 24;
#pragma unroll
                for (int t = 0; t < 3; ++t)
#pragma unroll
                    for (int v = 0; v < 2; ++v)
                        Re[(2 * cq + v) * 3 + t] = make_float2(Ah[t][2 * half + v], Al[t][2 * half + v]);
            }
        } else {
            for (int q = tid; q < TC_EX * TC_EY * 24; q += TC_THREADS) R[q] = make_float2(0.f, 0.f);
        }
        __syncthreads();

        // node layer gk = ez (elements ez-1 and ez both done)
        const int gk = ez;
        if (gk >= kz0 && gk < kz1) {
            const float2* Rc = S.R[ez & 1][0];
            const float2* Rp = S.R[(ez + 1) & 1][0];   // element layer ez-1
            for (int o = tid; o < TC_NX * TC_NY * 3; o += TC_THREADS) {
                const int c = o % 3, nn = o / 3;
                const int li = nn % TC_NX, lj = nn / TC_NX;
                const int gi = ex0 + 1 + li, gj = ey0 + 1 + lj;
                if (gi >= NX || gj >= NY) continue;
                const long long n = gi + (long long)NX * (gj + (long long)NY * gk);
                float h = 0.f, l = 0.f;
                if (gi >= 1) {
#pragma unroll
                    for (int z = 0; z < 2; ++z)
#pragma unroll
                        for (int yy = 0; yy < 2; ++yy)
#pragma unroll
                            for (int x = 0; x < 2; ++x) {
                                const float2* Rz = z ? Rp : Rc;   // node at offset z of element layer gk - z
                                const float2 v = Rz[((lj + 1 - yy) * TC_EX + (li + 1 - x)) * 24 + (x + 2 * yy + 4 * z) * 3 + c];
                                dd_add(h, l, v.x, v.y);
                            }
                }
                if (DD) {
                    const int kk = xmax - 1022 - TC_P;
                    const int k1 = kk / 2, k2 = kk - k1;
                    const float f1 = pow2f(max(-126, min(127, k1))), f2 = pow2f(max(-126, min(127, k2)));
                    const float h0 = h * f1 * f2, l0 = l * f1 * f2;
                    const float hs = h0 + l0;
                    yd[3 * n + c] = make_float2(hs, l0 - (hs - h0));
                } else {
                    const int sexp = xmax - 1022 - TC_P + 1023;
                    const double scale = (sexp >= 1) ? __longlong_as_double((long long)sexp << 52)
                                                     : scalbn(1.0, sexp - 1023);
                    y[3 * n + c] = ((double)h + (double)l) * scale;
                }
            }
        }
        if (more) store_digits(nxt, ez & 1);    // layer ez's slot is free after the MMAs
        Ew[0] = Enext[0];
        Ew[1] = Enext[1];
        __syncthreads();
    }
}

}  // namespace gf
