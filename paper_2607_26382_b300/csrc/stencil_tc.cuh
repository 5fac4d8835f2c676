// FP32-class V-cycle stencil (K x, b - K x, one node-block Jacobi sweep) with the
// element products on the tensor cores.
//
// The operator is the same as node_stencil_kernel's (Eq. frozen_operator on one level:
// y_n = sum over the 8 elements around node n of E_e (K0 u_e) restricted to n's rows).
// K0 = s M with small integers M (|M| <= 170, exact in TF32), so per element layer of a
// tile the products M u_e form one dense contraction, (16 elements x 24) x (24 x 24)
// per warp, run as mma.sync m16n8k8 on TF32 operands. TF32 keeps 11 significant bits,
// so a node value u is split into its TF32 rounding and the TF32-rounded remainder and
// each product is M u_hi + M u_lo (~2^-22 of |M||u|, against 2^-24 per FMA of the FP32
// kernel). A node value is split once, when its layer is staged in shared memory, and
// serves the 8 elements that share it.
//
// Work per CTA (256 threads): an (x, y) tile of 16 x 8 elements walking cz node layers
// in z. For element layer ez:
//   1. warp w (element row w) loads its A fragments from the (hi, lo) node window of
//      layers ez and ez+1 and runs 3 output x 3 input components x 2 parts of MMAs;
//      the accumulators (M u_e) go to shared memory;
//   2. the 105 nodes of node layer ez (15 x 7 per tile: neighbouring tiles recompute one
//      shared element row and column) sum s E_e (M u_e) over their 8 elements in a fixed
//      order and finish the mode's output; the other 151 threads split node layer ez+2
//      into the window and scale the moduli of element layer ez+1.
// The raw node layers and moduli arrive by cp.async into a 4-deep ring, requested four
// layers ahead, so a CTA waits for global memory once instead of once per layer.
// K-step c of the contraction is input component c; its 8 columns are the element's
// local nodes a' = x + 2y + 4z. Output tile t is output component t; its 8 columns are
// the output local nodes.
#pragma once
#include <cuda_runtime.h>

namespace gf {

constexpr int S3_EX = 16, S3_EY = 8;                 // elements per layer of a tile
constexpr int S3_NX = S3_EX - 1, S3_NY = S3_EY - 1;  // nodes written per layer
constexpr int S3_WX = S3_EX + 1, S3_WY = S3_EY + 1;  // node window per layer
constexpr int S3_RS = 24;                            // window row stride (float2): conflict-free A loads
constexpr int S3_ERS = 25;                           // element row stride of R (floats)
constexpr int S3_THREADS = 32 * S3_EY;
constexpr int S3_NODES = S3_NX * S3_NY;              // 105 gather threads
constexpr int S3_STAGERS = S3_THREADS - S3_NODES;    // 151 staging threads
constexpr int S3_LAYER_VALS = S3_WX * S3_WY * 3;     // 459
constexpr int S3_PER_STAGER = (S3_LAYER_VALS + S3_STAGERS - 1) / S3_STAGERS;   // 4
constexpr int S3_TILE_E = S3_EX * S3_EY;             // 128 moduli per element layer
constexpr int S3_RING = 4;                           // raw layers in flight

// B fragments of M, lane-major: [(t * 3 + c) * 2 + {b0, b1}][lane]
struct S3BFrag {
    float w[18][32];
};

struct S3Smem {
    float2 win[2][3][S3_WY][S3_RS];        // (hi, lo) of node values; slot = node layer & 1
    float R[2][S3_TILE_E][S3_ERS];         // (M u_e)[3 a' + t]; slot = element layer & 1
    float Es[3][S3_TILE_E];                // s E_e; slot = element layer mod 3
    float rawx[S3_RING][S3_STAGERS * S3_PER_STAGER];   // node layer L in slot L mod 4, by stager
    float rawe[S3_RING][S3_TILE_E];        // moduli of element layer L - 1 with node layer L
};

// TF32 rounding of an FP32 value (nearest, ties away from zero), in an FP32 register
__host__ __device__ __forceinline__ float tf32_round(float x)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
#else
    unsigned int b;
    static_assert(sizeof(b) == sizeof(x), "32-bit float");
    __builtin_memcpy(&b, &x, 4);
    b = (b + 0x1000u) & 0xFFFFE000u;
    float r;
    __builtin_memcpy(&r, &b, 4);
    return r;
#endif
}

__device__ __forceinline__ void mma_tf32_1688(float (&d)[4], float a0, float a1, float a2, float a3, float b0,
                                              float b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(__float_as_uint(a0)), "r"(__float_as_uint(a1)), "r"(__float_as_uint(a2)), "r"(__float_as_uint(a3)),
          "r"(__float_as_uint(b0)), "r"(__float_as_uint(b1)));
}

__device__ __forceinline__ int s3_mod3(int v) { return ((v % 3) + 3) % 3; }
__device__ __forceinline__ int s3_mod4(int v) { return v & 3; }

// 4-byte asynchronous copy global -> shared; ok == false writes 0 and reads nothing
__device__ __forceinline__ void s3_cp4(float* dst, const float* src, bool ok)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void s3_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void s3_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// MODE, out, b as in stencil_node: APPLY out = K x, RESID out = b - K x,
// SWEEP out = x + omega D_n^{-1} (b - K x); fixed nodes (i == 0) get 0.
// E: the level's moduli; s: K0 = s M; B: build_s3_bfrag's fragments in device memory.
// Grid: (ceil(NX / 15), ceil(NY / 7), ceil(NZ / cz)) CTAs of S3_THREADS, sizeof(S3Smem)
// bytes of dynamic shared memory.
template <int MODE, typename BT, typename OT>
__global__ void __launch_bounds__(S3_THREADS, 3)
stencil_tc32_kernel(const float* __restrict__ x, const BT* __restrict__ b, OT* __restrict__ out,
                    const float* __restrict__ E, GridDims d, const __grid_constant__ MParam M,
                    const S3BFrag* __restrict__ B, float s, float omega, int cz, const int* __restrict__ halt)
{
    if (halt != nullptr && *halt != 0) return;
    extern __shared__ __align__(16) unsigned char s3_smem_raw[];
    S3Smem& S = *reinterpret_cast<S3Smem*>(s3_smem_raw);
    const int NX = d.nx + 1, NY = d.ny + 1, NZ = d.nz + 1;
    const long long layer = (long long)NX * NY;                           // nodes per node layer
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ex0 = blockIdx.x * S3_NX - 1, ey0 = blockIdx.y * S3_NY - 1;   // first element (may be -1)
    const int kz0 = blockIdx.z * cz;                                      // first node layer written
    const int kz1 = min(kz0 + cz, NZ);                                    // one past the last

    // ---- staging threads: fixed (layer-independent) window positions
    const int st = tid - S3_NODES;
    int woff[S3_PER_STAGER];          // DOF offset within a node layer, -1 = reads 0
    int wdst[S3_PER_STAGER];          // float2 index into win[slot], -1 = none
#pragma unroll
    for (int v = 0; v < S3_PER_STAGER; ++v) {
        const int q = st + v * S3_STAGERS;
        woff[v] = -1;
        wdst[v] = -1;
        if (st >= 0 && q < S3_LAYER_VALS) {
            const int c = q % 3, r = q / 3;
            const int wx = r % S3_WX, wy = r / S3_WX;
            const int gi = ex0 + wx, gj = ey0 + wy;
            wdst[v] = (c * S3_WY + wy) * S3_RS + wx;
            if (gi >= 1 && gi < NX && gj >= 0 && gj < NY) woff[v] = 3 * (gi + NX * gj) + c;
        }
    }
    int eoff = -1;                    // element offset within an element layer (st < 128)
    if (st >= 0 && st < S3_TILE_E) {
        const int ex = ex0 + st % S3_EX, ey = ey0 + st / S3_EX;
        if (ex >= 0 && ex < d.nx && ey >= 0 && ey < d.ny) eoff = ex + d.nx * ey;
    }
    // request node layer L (and the moduli of element layer L - 1) into ring slot L mod 4;
    // every thread commits one group per layer, empty or not
    auto request = [&](int L) {
        if (st >= 0 && L <= kz1) {
            const bool in = L >= 0 && L < NZ;
            const float* xl = x + 3 * layer * (in ? L : 0);
            float* rx = &S.rawx[s3_mod4(L)][st * S3_PER_STAGER];
#pragma unroll
            for (int q = 0; q < S3_PER_STAGER; ++q)
                if (wdst[q] >= 0) s3_cp4(rx + q, in && woff[q] >= 0 ? xl + woff[q] : x, in && woff[q] >= 0);
            if (st < S3_TILE_E) {
                const int el = L - 1;
                const bool ein = eoff >= 0 && el >= 0 && el < d.nz;
                s3_cp4(&S.rawe[s3_mod4(L)][st], ein ? E + (long long)d.nx * d.ny * el + eoff : E, ein);
            }
        }
        s3_commit();
    };
    // node layer L from the ring into window slot L & 1; moduli of element layer L - 1
    auto split = [&](int L) {
        if (st >= 0) {
            const float* rx = &S.rawx[s3_mod4(L)][st * S3_PER_STAGER];
            float2* w = &S.win[L & 1][0][0][0];
#pragma unroll
            for (int q = 0; q < S3_PER_STAGER; ++q)
                if (wdst[q] >= 0) {
                    const float v = rx[q];
                    const float hi = tf32_round(v);
                    w[wdst[q]] = make_float2(hi, tf32_round(v - hi));
                }
            if (st < S3_TILE_E) S.Es[s3_mod3(L - 1)][st] = s * S.rawe[s3_mod4(L)][st];
        }
    };

    // ---- gather threads: fixed node of the tile
    const int li = tid % S3_NX, lj = tid / S3_NX;
    const int gi = ex0 + 1 + li, gj = ey0 + 1 + lj;
    const bool gather = tid < S3_NODES && gi < NX && gj < NY;
    const long long n0 = gi + (long long)NX * gj;                         // node index in layer 0

    // prologue: node layers kz0-1 .. kz0+2 requested; kz0-1 and kz0 split (with the
    // moduli of element layers kz0-2, unused, and kz0-1), their slots requested again
    // for kz0+3 and kz0+4. A stager only ever reads the ring entries it copied itself.
#pragma unroll
    for (int L = 0; L < S3_RING; ++L) request(kz0 - 1 + L);
    float bw[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) bw[q] = B->w[q][lane];
    s3_wait<S3_RING - 2>();
    split(kz0 - 1);
    request(kz0 + 3);
    split(kz0);
    request(kz0 + 4);
    __syncthreads();
    const int g = lane >> 2, cq = lane & 3;
    const int ly = warp;                         // this warp's element row
    const int aoff = (ly + (cq >> 1)) * S3_RS + g + (cq & 1);   // A-fragment window position

    for (int ez = kz0 - 1; ez < kz1; ++ez) {

        // ---- 1. element layer ez: M u_e on the tensor cores
        {
            float acc[3][4];
#pragma unroll
            for (int t = 0; t < 3; ++t)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[t][v] = 0.f;
            const float2* w0 = &S.win[ez & 1][0][0][0] + aoff;         // node layer ez (z = 0)
            const float2* w1 = &S.win[(ez + 1) & 1][0][0][0] + aoff;   // node layer ez+1 (z = 1)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float2 p0 = w0[c * S3_WY * S3_RS], p1 = w0[c * S3_WY * S3_RS + 8];
                const float2 p2 = w1[c * S3_WY * S3_RS], p3 = w1[c * S3_WY * S3_RS + 8];
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    const float b0 = bw[(t * 3 + c) * 2], b1 = bw[(t * 3 + c) * 2 + 1];
                    mma_tf32_1688(acc[t], p0.y, p1.y, p2.y, p3.y, b0, b1);   // remainder first
                    mma_tf32_1688(acc[t], p0.x, p1.x, p2.x, p3.x, b0, b1);
                }
            }
            // D rows g / g+8 = elements, cols 2cq, 2cq+1 = output local nodes
            float* R = &S.R[ez & 1][0][0];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float* Re = R + (ly * S3_EX + g + 8 * h) * S3_ERS;
#pragma unroll
                for (int t = 0; t < 3; ++t)
#pragma unroll
                    for (int v = 0; v < 2; ++v) Re[(2 * cq + v) * 3 + t] = acc[t][2 * h + v];
            }
        }
        __syncthreads();

        // ---- 2. node layer gk = ez (element layers ez-1 and ez are done)
        const int gk = ez;
        if (gather && gk >= kz0) {
            const long long n = n0 + layer * gk;
            if (gi == 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) out[3 * n + c] = OT(0);
            } else {
                const float* Rc = &S.R[ez & 1][0][0];          // element layer ez   (node at z = 0)
                const float* Rp = &S.R[(ez + 1) & 1][0][0];    // element layer ez-1 (node at z = 1)
                const float* Ec = S.Es[s3_mod3(ez)];
                const float* Ep = S.Es[s3_mod3(ez - 1)];
                float a0 = 0.f, a1 = 0.f, a2 = 0.f;
                float d00 = 0.f, d11 = 0.f, d22 = 0.f, d01 = 0.f, d02 = 0.f, d12 = 0.f;
#pragma unroll
                for (int oz = 0; oz < 2; ++oz)
#pragma unroll
                    for (int oy = 0; oy < 2; ++oy)
#pragma unroll
                        for (int ox = 0; ox < 2; ++ox) {
                            // element (gi-1+ox, gj-1+oy, gk-1+oz) = tile element (li+ox, lj+oy)
                            const int e = (lj + oy) * S3_EX + li + ox;
                            const int ap = (1 - ox) + 2 * (1 - oy) + 4 * (1 - oz);
                            const float* Re = (oz ? Rc : Rp) + e * S3_ERS + 3 * ap;
                            const float Ee = (oz ? Ec : Ep)[e];
                            a0 = fmaf(Ee, Re[0], a0);
                            a1 = fmaf(Ee, Re[1], a1);
                            a2 = fmaf(Ee, Re[2], a2);
                            if (MODE == ST_SWEEP) {
                                const int a = local_index(1 - ox, 1 - oy, 1 - oz);
                                d00 = fmaf(Ee, M.m[(3 * a + 0) * 24 + 3 * a + 0], d00);
                                d11 = fmaf(Ee, M.m[(3 * a + 1) * 24 + 3 * a + 1], d11);
                                d22 = fmaf(Ee, M.m[(3 * a + 2) * 24 + 3 * a + 2], d22);
                                d01 = fmaf(Ee, M.m[(3 * a + 0) * 24 + 3 * a + 1], d01);
                                d02 = fmaf(Ee, M.m[(3 * a + 0) * 24 + 3 * a + 2], d02);
                                d12 = fmaf(Ee, M.m[(3 * a + 1) * 24 + 3 * a + 2], d12);
                            }
                        }
                if (MODE == ST_APPLY) {
                    out[3 * n + 0] = OT(a0);
                    out[3 * n + 1] = OT(a1);
                    out[3 * n + 2] = OT(a2);
                } else {
                    const float r0 = float(b[3 * n + 0]) - a0;
                    const float r1 = float(b[3 * n + 1]) - a1;
                    const float r2 = float(b[3 * n + 2]) - a2;
                    if (MODE == ST_RESID) {
                        out[3 * n + 0] = OT(r0);
                        out[3 * n + 1] = OT(r1);
                        out[3 * n + 2] = OT(r2);
                    } else {
                        const float c00 = d11 * d22 - d12 * d12;
                        const float c01 = d02 * d12 - d01 * d22;
                        const float c02 = d01 * d12 - d02 * d11;
                        const float c11 = d00 * d22 - d02 * d02;
                        const float c12 = d01 * d02 - d00 * d12;
                        const float c22 = d00 * d11 - d01 * d01;
                        const float det = d00 * c00 + d01 * c01 + d02 * c02;
                        const float sc = omega / det;
                        out[3 * n + 0] = OT(x[3 * n + 0] + sc * (c00 * r0 + c01 * r1 + c02 * r2));
                        out[3 * n + 1] = OT(x[3 * n + 1] + sc * (c01 * r0 + c11 * r1 + c12 * r2));
                        out[3 * n + 2] = OT(x[3 * n + 2] + sc * (c02 * r0 + c12 * r1 + c22 * r2));
                    }
                }
            }
        }
        // staging: node layer ez's window slot is free after the MMAs, and the moduli slot
        // of element layer ez+1 is neither of the two the gather reads. Groups committed so
        // far run to node layer ez+5; layer ez+2's is complete when at most 3 are pending.
        // Its ring slot then takes node layer ez+6. No copy is left in flight at the end:
        // layers past kz1 are empty groups, and layer kz1 is split at ez = kz1 - 2.
        if (ez + 2 <= kz1) {
            s3_wait<3>();
            split(ez + 2);
        }
        request(ez + 6);
        __syncthreads();
    }
}

}  // namespace gf
