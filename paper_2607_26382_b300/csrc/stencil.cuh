// Matrix-free hex8 elasticity stencils on a structured grid (node-centric gather).
//
// y_n = sum over the (up to) 8 elements e touching node n of E_e * K0[3a:3a+3, :] u_e,
// where a is n's local index in e -- the frozen operator K = sum_e E_e K_e of
// Eq. (frozen_operator) (arXiv 2607.26382), evaluated one output node per thread so
// that no atomics and no zero-fill pass are needed. K0 (24x24, E0 applied, edge 1)
// is a kernel parameter: after full unrolling every K0 entry is a compile-time
// offset into the constant parameter bank and feeds the FMA directly.
//
// The same gather also yields the node's 3x3 diagonal block sum_e E_e K0[3a:3a+3,
// 3a:3a+3], which the damped node-block Jacobi smoother inverts in closed form.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "cvt.cuh"

namespace gf {

template <typename T>
struct K0Param {
    T k[576];   // row-major 24x24
};

// Local index of the element node at offset (x,y,z) in {0,1}^3: bottom face
// counter-clockwise (0..3), then top face (4..7).
__host__ __device__ constexpr int local_index(int x, int y, int z) {
    return 4 * z + (y ? (x ? 2 : 3) : (x ? 1 : 0));
}

enum StencilMode { ST_APPLY = 0, ST_RESID = 1, ST_SWEEP = 2 };

struct GridDims {
    int nx, ny, nz;                 // elements per axis
    const uint8_t* fix = nullptr;   // per node, bit c set: component c fixed (device); null: every
                                    // DOF of the nodes on the clamped face x = 0 (the cantilever)
};

// Fixed components of node n (i: its x index) as bits 0..2.
__device__ __forceinline__ unsigned fix_bits(const GridDims& d, long long n, int i)
{
    return d.fix ? (unsigned)__ldg(d.fix + n) : (i == 0 ? 7u : 0u);
}

// Is DOF q (= 3n + c) fixed?
__device__ __forceinline__ bool fix_dof(const GridDims& d, long long q)
{
    const long long n = q / 3;
    return d.fix ? ((__ldg(d.fix + n) >> (int)(q - 3 * n)) & 1) != 0 : (n % (d.nx + 1)) == 0;
}

// The node block of a partly fixed node: identity rows and columns on its fixed components.
template <typename T>
__device__ __forceinline__ void mask_block(unsigned fb, T& d00, T& d11, T& d22, T& d01, T& d02, T& d12)
{
    if (fb & 1u) { d00 = T(1); d01 = T(0); d02 = T(0); }
    if (fb & 2u) { d11 = T(1); d01 = T(0); d12 = T(0); }
    if (fb & 4u) { d22 = T(1); d02 = T(0); d12 = T(0); }
}

// (i, j, k) of node n = i + NX (j + NY k). Grids hold fewer than 2^31 nodes
// (gf_create_grid checks), so 32-bit unsigned division suffices.
__device__ __forceinline__ void node_coords(long long n, int NX, int NY, int& i, int& j, int& k) {
    const unsigned u = (unsigned)n;
    const unsigned t = u / (unsigned)NX;
    i = (int)(u - t * (unsigned)NX);
    j = (int)(t % (unsigned)NY);
    k = (int)(t / (unsigned)NY);
}

// Damped node-block Jacobi update out = x + omega * D_n^{-1} r, D_n solved by its adjugate.
// Every product and sum is an explicit fma or a single rounded operation, so each stencil
// kernel that calls this rounds the update identically, whatever contractions the
// compiler picks around it.
template <typename T, typename OT>
__device__ __forceinline__ void node_block_update(T d00, T d11, T d22, T d01, T d02, T d12, T r0, T r1, T r2,
                                                  const T* __restrict__ x, OT* __restrict__ out, T omega)
{
    const T c00 = fma(d11, d22, -(d12 * d12));
    const T c01 = fma(d02, d12, -(d01 * d22));
    const T c02 = fma(d01, d12, -(d02 * d11));
    const T c11 = fma(d00, d22, -(d02 * d02));
    const T c12 = fma(d01, d02, -(d00 * d12));
    const T c22 = fma(d00, d11, -(d01 * d01));
    const T det = fma(d00, c00, fma(d01, c01, d02 * c02));
    const T s = omega / det;
    out[0] = convert<OT>(fma(s, fma(c00, r0, fma(c01, r1, c02 * r2)), x[0]));
    out[1] = convert<OT>(fma(s, fma(c01, r0, fma(c11, r1, c12 * r2)), x[1]));
    out[2] = convert<OT>(fma(s, fma(c02, r0, fma(c12, r1, c22 * r2)), x[2]));
}

// MODE == ST_APPLY: out = K x
// MODE == ST_RESID: out = b - K x
// MODE == ST_SWEEP: out = x + omega * D_n^{-1} (b - K x)     (D_n: 3x3 node block)
// Fixed nodes (i == 0) read as 0 and are written as 0. Element moduli E are
// already multiplied by the element edge h (K_e(h) = h K_e(1) in 3D).
// MASK: fixed components from d.fix (any supports); otherwise the clamped face x = 0
// by the node index (the cantilever code, unchanged).
template <typename T, typename ET, int MODE, typename BT, typename OT, bool MASK = false>
__device__ __forceinline__ void stencil_node(long long n, const T* __restrict__ x, const BT* __restrict__ b,
                                             OT* __restrict__ out, const ET* __restrict__ E, GridDims d,
                                             const K0Param<T>& K0, T omega)
{
    const int NX = d.nx + 1, NY = d.ny + 1;
    int i, j, k;
    node_coords(n, NX, NY, i, j, k);
    const unsigned fb = MASK ? (unsigned)__ldg(d.fix + n) : (i == 0 ? 7u : 0u);
    if (fb == 7u) {
        out[3 * n + 0] = OT(0);
        out[3 * n + 1] = OT(0);
        out[3 * n + 2] = OT(0);
        return;
    }
    T a0 = 0, a1 = 0, a2 = 0;
    T d00 = 0, d11 = 0, d22 = 0, d01 = 0, d02 = 0, d12 = 0;
    // FP32: the 27 neighbour nodes are loaded once into registers (a node shared by
    // several elements would otherwise be re-read per element); the FMAs below run in
    // the same order either way. Out-of-domain and fixed neighbours read as 0.
    // The node planes are loaded as needed (planes z-1, z for the lower elements, plane
    // z+1 before the upper ones), so at most two planes are live.
    constexpr bool REGS = sizeof(T) == 4;
    T nb[REGS ? 3 : 1][REGS ? 3 : 1][REGS ? 3 : 1][3];
    auto load_plane = [&](int dz) {
        if constexpr (REGS) {
            const int NZ = d.nz + 1;
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const int ni = i - 1 + dx, nj = j - 1 + dy, nk = k - 1 + dz;
                    const long long m = n + (dx - 1) + (long long)NX * ((dy - 1) + (long long)NY * (dz - 1));
                    if constexpr (MASK) {
                        const bool in = ni >= 0 && ni < NX && nj >= 0 && nj < NY && nk >= 0 && nk < NZ;
                        const unsigned mb = in ? (unsigned)__ldg(d.fix + m) : 7u;
#pragma unroll
                        for (int c = 0; c < 3; ++c) nb[dz][dy][dx][c] = ((mb >> c) & 1u) ? T(0) : x[3 * m + c];
                    } else {
                        const bool ok = ni >= 1 && ni < NX && nj >= 0 && nj < NY && nk >= 0 && nk < NZ;
#pragma unroll
                        for (int c = 0; c < 3; ++c) nb[dz][dy][dx][c] = ok ? x[3 * m + c] : T(0);
                    }
                }
        }
    };
    load_plane(0);
    load_plane(1);
#pragma unroll
    for (int oz = 0; oz < 2; ++oz) {
        if (oz == 1) load_plane(2);
#pragma unroll
        for (int oy = 0; oy < 2; ++oy) {
#pragma unroll
            for (int ox = 0; ox < 2; ++ox) {
                const int ex = i - 1 + ox, ey = j - 1 + oy, ez = k - 1 + oz;
                if (ex < 0 || ex >= d.nx || ey < 0 || ey >= d.ny || ez < 0 || ez >= d.nz) continue;
                const T Ee = (T)E[ex + (long long)d.nx * (ey + (long long)d.ny * ez)];
                const int a = local_index(1 - ox, 1 - oy, 1 - oz);
                T t0 = 0, t1 = 0, t2 = 0;
#pragma unroll
                for (int bz = 0; bz < 2; ++bz) {
#pragma unroll
                    for (int by = 0; by < 2; ++by) {
#pragma unroll
                        for (int bx = 0; bx < 2; ++bx) {
                            const int bl = local_index(bx, by, bz);
                            const int ni = ex + bx;
                            T u0 = 0, u1 = 0, u2 = 0;
                            if constexpr (REGS) {
                                u0 = nb[oz + bz][oy + by][ox + bx][0];
                                u1 = nb[oz + bz][oy + by][ox + bx][1];
                                u2 = nb[oz + bz][oy + by][ox + bx][2];
                            } else if constexpr (MASK) {
                                const long long m = ni + (long long)NX * ((ey + by) + (long long)NY * (ez + bz));
                                const unsigned mb = (unsigned)__ldg(d.fix + m);
                                u0 = (mb & 1u) ? T(0) : x[3 * m + 0];
                                u1 = (mb & 2u) ? T(0) : x[3 * m + 1];
                                u2 = (mb & 4u) ? T(0) : x[3 * m + 2];
                            } else if (ni != 0) {
                                const long long m = ni + (long long)NX * ((ey + by) + (long long)NY * (ez + bz));
                                u0 = x[3 * m + 0];
                                u1 = x[3 * m + 1];
                                u2 = x[3 * m + 2];
                            }
                            const T* r0 = &K0.k[(3 * a + 0) * 24 + 3 * bl];
                            const T* r1 = &K0.k[(3 * a + 1) * 24 + 3 * bl];
                            const T* r2 = &K0.k[(3 * a + 2) * 24 + 3 * bl];
                            t0 = fma(r0[0], u0, fma(r0[1], u1, fma(r0[2], u2, t0)));
                            t1 = fma(r1[0], u0, fma(r1[1], u1, fma(r1[2], u2, t1)));
                            t2 = fma(r2[0], u0, fma(r2[1], u1, fma(r2[2], u2, t2)));
                        }
                    }
                }
                a0 = fma(Ee, t0, a0);
                a1 = fma(Ee, t1, a1);
                a2 = fma(Ee, t2, a2);
                if (MODE == ST_SWEEP) {
                    d00 = fma(Ee, K0.k[(3 * a + 0) * 24 + 3 * a + 0], d00);
                    d11 = fma(Ee, K0.k[(3 * a + 1) * 24 + 3 * a + 1], d11);
                    d22 = fma(Ee, K0.k[(3 * a + 2) * 24 + 3 * a + 2], d22);
                    d01 = fma(Ee, K0.k[(3 * a + 0) * 24 + 3 * a + 1], d01);
                    d02 = fma(Ee, K0.k[(3 * a + 0) * 24 + 3 * a + 2], d02);
                    d12 = fma(Ee, K0.k[(3 * a + 1) * 24 + 3 * a + 2], d12);
                }
            }
        }
    }
    if constexpr (MASK) {   // a partly fixed node: its fixed components stay 0
        if (fb & 1u) a0 = T(0);
        if (fb & 2u) a1 = T(0);
        if (fb & 4u) a2 = T(0);
    }
    if (MODE == ST_APPLY) {
        out[3 * n + 0] = OT(a0);
        out[3 * n + 1] = OT(a1);
        out[3 * n + 2] = OT(a2);
        return;
    }
    T r0 = T(b[3 * n + 0]) - a0;
    T r1 = T(b[3 * n + 1]) - a1;
    T r2 = T(b[3 * n + 2]) - a2;
    if constexpr (MASK) {
        if (fb & 1u) r0 = T(0);
        if (fb & 2u) r1 = T(0);
        if (fb & 4u) r2 = T(0);
    }
    if (MODE == ST_RESID) {
        out[3 * n + 0] = OT(r0);
        out[3 * n + 1] = OT(r1);
        out[3 * n + 2] = OT(r2);
        return;
    }
    if constexpr (MASK) {
        if (fb) {   // identity rows and columns on the fixed components; their output stays 0
            mask_block<T>(fb, d00, d11, d22, d01, d02, d12);
            const T xm[3] = {(fb & 1u) ? T(0) : x[3 * n + 0], (fb & 2u) ? T(0) : x[3 * n + 1],
                             (fb & 4u) ? T(0) : x[3 * n + 2]};
            node_block_update<T, OT>(d00, d11, d22, d01, d02, d12, r0, r1, r2, xm, out + 3 * n, omega);
            return;
        }
    }
    node_block_update<T, OT>(d00, d11, d22, d01, d02, d12, r0, r1, r2, x + 3 * n, out + 3 * n, omega);
}

// FP32: at most 80 registers (3 blocks of 256 per SM), which the plane-wise neighbour
// loads allow with a few bytes of spill; measured 17.3 -> 14.7 us (96x48x48) and
// 92.8 -> 74.5 us (192x96x96) against the unbounded 108-120-register build.
template <typename T, typename ET, int MODE, typename BT = T, typename OT = T, bool MASK = false>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
node_stencil_kernel(const T* __restrict__ x, const BT* __restrict__ b, OT* __restrict__ out,
                    const ET* __restrict__ E, GridDims d, const __grid_constant__ K0Param<T> K0,
                    T omega, const int* __restrict__ halt)
{
    if (halt != nullptr && *halt != 0) return;
    const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    stencil_node<T, ET, MODE, BT, OT, MASK>(n, x, b, out, E, d, K0, omega);
}

// ---- FP32 node stencil with paired FMAs (fma.rn.f32x2) ------------------------------
// K0 rows 3a and 3a+1 stored as adjacent pairs, so one paired FMA advances the x and y
// output chains of an element together; the z chain stays scalar. Every K*u chain keeps
// the order of stencil_node (K*u bit-identical to node_stencil_kernel<float>; the sweep's
// node-block solve may round differently in its last bit). The FP32 V-cycle default.
struct K0Pair {
    float2 p[8][8][3];   // (K0[3a][3b+k], K0[3a+1][3b+k]), a = output node, b = input node
    float s[8][8][3];    // K0[3a+2][3b+k]
};

__device__ __forceinline__ void fma_f32x2(float& d0, float& d1, float2 a, float b)
{
    asm("{\n .reg .b64 ra, rb, rc;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %4};\n mov.b64 rc, {%0, %1};\n"
        " fma.rn.f32x2 rc, ra, rb, rc;\n mov.b64 {%0, %1}, rc;\n}\n"
        : "+f"(d0), "+f"(d1) : "f"(a.x), "f"(a.y), "f"(b));
}

template <int MODE, typename BT, typename OT, bool MASK = false>
__device__ __forceinline__ void stencil_node_f32x2(long long n, const float* __restrict__ x, const BT* __restrict__ b,
                                                   OT* __restrict__ out, const float* __restrict__ E, GridDims d,
                                                   const K0Pair& K0, float omega)
{
    const int NX = d.nx + 1, NY = d.ny + 1;
    int i, j, k;
    node_coords(n, NX, NY, i, j, k);
    const unsigned fb = MASK ? (unsigned)__ldg(d.fix + n) : (i == 0 ? 7u : 0u);
    if (fb == 7u) {
        out[3 * n + 0] = OT(0);
        out[3 * n + 1] = OT(0);
        out[3 * n + 2] = OT(0);
        return;
    }
    float a0 = 0, a1 = 0, a2 = 0;
    float d00 = 0, d11 = 0, d22 = 0, d01 = 0, d02 = 0, d12 = 0;
    float nb[3][3][3][3];
    auto load_plane = [&](int dz) {
        const int NZ = d.nz + 1;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const int ni = i - 1 + dx, nj = j - 1 + dy, nk = k - 1 + dz;
                const long long m = n + (dx - 1) + (long long)NX * ((dy - 1) + (long long)NY * (dz - 1));
                if constexpr (MASK) {
                    const bool in = ni >= 0 && ni < NX && nj >= 0 && nj < NY && nk >= 0 && nk < NZ;
                    const unsigned mb = in ? (unsigned)__ldg(d.fix + m) : 7u;
#pragma unroll
                    for (int c = 0; c < 3; ++c) nb[dz][dy][dx][c] = ((mb >> c) & 1u) ? 0.f : x[3 * m + c];
                } else {
                    const bool ok = ni >= 1 && ni < NX && nj >= 0 && nj < NY && nk >= 0 && nk < NZ;
#pragma unroll
                    for (int c = 0; c < 3; ++c) nb[dz][dy][dx][c] = ok ? x[3 * m + c] : 0.f;
                }
            }
    };
    load_plane(0);
    load_plane(1);
#pragma unroll
    for (int oz = 0; oz < 2; ++oz) {
        if (oz == 1) load_plane(2);
#pragma unroll
        for (int oy = 0; oy < 2; ++oy) {
#pragma unroll
            for (int ox = 0; ox < 2; ++ox) {
                const int ex = i - 1 + ox, ey = j - 1 + oy, ez = k - 1 + oz;
                if (ex < 0 || ex >= d.nx || ey < 0 || ey >= d.ny || ez < 0 || ez >= d.nz) continue;
                const float Ee = E[ex + (long long)d.nx * (ey + (long long)d.ny * ez)];
                const int a = local_index(1 - ox, 1 - oy, 1 - oz);
                float t0 = 0, t1 = 0, t2 = 0;
#pragma unroll
                for (int bz = 0; bz < 2; ++bz) {
#pragma unroll
                    for (int by = 0; by < 2; ++by) {
#pragma unroll
                        for (int bx = 0; bx < 2; ++bx) {
                            const int bl = local_index(bx, by, bz);
                            const float u0 = nb[oz + bz][oy + by][ox + bx][0];
                            const float u1 = nb[oz + bz][oy + by][ox + bx][1];
                            const float u2 = nb[oz + bz][oy + by][ox + bx][2];
                            fma_f32x2(t0, t1, K0.p[a][bl][2], u2);
                            fma_f32x2(t0, t1, K0.p[a][bl][1], u1);
                            fma_f32x2(t0, t1, K0.p[a][bl][0], u0);
                            t2 = fmaf(K0.s[a][bl][0], u0, fmaf(K0.s[a][bl][1], u1, fmaf(K0.s[a][bl][2], u2, t2)));
                        }
                    }
                }
                a0 = fmaf(Ee, t0, a0);
                a1 = fmaf(Ee, t1, a1);
                a2 = fmaf(Ee, t2, a2);
                if (MODE == ST_SWEEP) {
                    d00 = fmaf(Ee, K0.p[a][a][0].x, d00);
                    d11 = fmaf(Ee, K0.p[a][a][1].y, d11);
                    d22 = fmaf(Ee, K0.s[a][a][2], d22);
                    d01 = fmaf(Ee, K0.p[a][a][1].x, d01);
                    d02 = fmaf(Ee, K0.p[a][a][2].x, d02);
                    d12 = fmaf(Ee, K0.p[a][a][2].y, d12);
                }
            }
        }
    }
    if constexpr (MASK) {
        if (fb & 1u) a0 = 0.f;
        if (fb & 2u) a1 = 0.f;
        if (fb & 4u) a2 = 0.f;
    }
    if (MODE == ST_APPLY) {
        out[3 * n + 0] = OT(a0);
        out[3 * n + 1] = OT(a1);
        out[3 * n + 2] = OT(a2);
        return;
    }
    float r0 = float(b[3 * n + 0]) - a0;
    float r1 = float(b[3 * n + 1]) - a1;
    float r2 = float(b[3 * n + 2]) - a2;
    if constexpr (MASK) {
        if (fb & 1u) r0 = 0.f;
        if (fb & 2u) r1 = 0.f;
        if (fb & 4u) r2 = 0.f;
    }
    if (MODE == ST_RESID) {
        out[3 * n + 0] = OT(r0);
        out[3 * n + 1] = OT(r1);
        out[3 * n + 2] = OT(r2);
        return;
    }
    if constexpr (MASK) {
        if (fb) {
            mask_block<float>(fb, d00, d11, d22, d01, d02, d12);
            const float xm[3] = {(fb & 1u) ? 0.f : x[3 * n + 0], (fb & 2u) ? 0.f : x[3 * n + 1],
                                 (fb & 4u) ? 0.f : x[3 * n + 2]};
            node_block_update<float, OT>(d00, d11, d22, d01, d02, d12, r0, r1, r2, xm, out + 3 * n, omega);
            return;
        }
    }
    node_block_update<float, OT>(d00, d11, d22, d01, d02, d12, r0, r1, r2, x + 3 * n, out + 3 * n, omega);
}

template <int MODE, typename BT, typename OT, bool MASK = false>
__global__ void __launch_bounds__(256, 3)
node_stencil_f32x2_kernel(const float* __restrict__ x, const BT* __restrict__ b, OT* __restrict__ out,
                          const float* __restrict__ E, GridDims d, const __grid_constant__ K0Pair K0, float omega,
                          const int* __restrict__ halt)
{
    if (halt != nullptr && *halt != 0) return;
    const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    stencil_node_f32x2<MODE, BT, OT, MASK>(n, x, b, out, E, d, K0, omega);
}

// First smoothing sweep from x = 0: out = omega * D_n^{-1} b, b_n = (r0, r1, r2).
template <typename T, typename ET>
__device__ __forceinline__ void first_sweep_vals(long long n, T r0, T r1, T r2, T* __restrict__ out,
                                                 const ET* __restrict__ E, GridDims d, const K0Param<T>& K0,
                                                 T omega)
{
    const int NX = d.nx + 1, NY = d.ny + 1;
    int i, j, k;
    node_coords(n, NX, NY, i, j, k);
    const unsigned fb = fix_bits(d, n, i);
    if (fb == 7u) {
        out[3 * n + 0] = T(0);
        out[3 * n + 1] = T(0);
        out[3 * n + 2] = T(0);
        return;
    }
    T d00 = 0, d11 = 0, d22 = 0, d01 = 0, d02 = 0, d12 = 0;
#pragma unroll
    for (int oz = 0; oz < 2; ++oz)
#pragma unroll
        for (int oy = 0; oy < 2; ++oy)
#pragma unroll
            for (int ox = 0; ox < 2; ++ox) {
                const int ex = i - 1 + ox, ey = j - 1 + oy, ez = k - 1 + oz;
                if (ex < 0 || ex >= d.nx || ey < 0 || ey >= d.ny || ez < 0 || ez >= d.nz) continue;
                const T Ee = (T)E[ex + (long long)d.nx * (ey + (long long)d.ny * ez)];
                const int a = local_index(1 - ox, 1 - oy, 1 - oz);
                d00 = fma(Ee, K0.k[(3 * a + 0) * 24 + 3 * a + 0], d00);
                d11 = fma(Ee, K0.k[(3 * a + 1) * 24 + 3 * a + 1], d11);
                d22 = fma(Ee, K0.k[(3 * a + 2) * 24 + 3 * a + 2], d22);
                d01 = fma(Ee, K0.k[(3 * a + 0) * 24 + 3 * a + 1], d01);
                d02 = fma(Ee, K0.k[(3 * a + 0) * 24 + 3 * a + 2], d02);
                d12 = fma(Ee, K0.k[(3 * a + 1) * 24 + 3 * a + 2], d12);
            }
    if (fb) {   // a partly fixed node: identity rows and columns, zero right-hand side there
        mask_block<T>(fb, d00, d11, d22, d01, d02, d12);
        if (fb & 1u) r0 = T(0);
        if (fb & 2u) r1 = T(0);
        if (fb & 4u) r2 = T(0);
    }
    const T c00 = d11 * d22 - d12 * d12;
    const T c01 = d02 * d12 - d01 * d22;
    const T c02 = d01 * d12 - d02 * d11;
    const T c11 = d00 * d22 - d02 * d02;
    const T c12 = d01 * d02 - d00 * d12;
    const T c22 = d00 * d11 - d01 * d01;
    const T det = d00 * c00 + d01 * c01 + d02 * c02;
    const T s = omega / det;
    out[3 * n + 0] = s * (c00 * r0 + c01 * r1 + c02 * r2);
    out[3 * n + 1] = s * (c01 * r0 + c11 * r1 + c12 * r2);
    out[3 * n + 2] = s * (c02 * r0 + c12 * r1 + c22 * r2);
}

// The same with b read from memory. BT is b's type.
template <typename T, typename ET, typename BT>
__device__ __forceinline__ void first_sweep_node(long long n, const BT* __restrict__ b, T* __restrict__ out,
                                                 const ET* __restrict__ E, GridDims d, const K0Param<T>& K0,
                                                 T omega)
{
    first_sweep_vals<T, ET>(n, (T)b[3 * n + 0], (T)b[3 * n + 1], (T)b[3 * n + 2], out, E, d, K0, omega);
}

template <typename T, typename ET, typename BT>
__global__ void __launch_bounds__(256)
first_sweep_kernel(const BT* __restrict__ b, T* __restrict__ out, const ET* __restrict__ E,
                   GridDims d, const __grid_constant__ K0Param<T> K0, T omega,
                   const int* __restrict__ halt)
{
    if (halt != nullptr && *halt != 0) return;
    const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    first_sweep_node<T, ET, BT>(n, b, out, E, d, K0, omega);
}

// The same, storing the right-hand side converted to T once (bout) for the level's later
// sweeps and residual: they then read T instead of converting BT at every read.
template <typename T, typename ET, typename BT>
__global__ void __launch_bounds__(256)
first_sweep_store_kernel(const BT* __restrict__ b, T* __restrict__ bout, T* __restrict__ out,
                         const ET* __restrict__ E, GridDims d, const __grid_constant__ K0Param<T> K0, T omega,
                         const int* __restrict__ halt)
{
    if (halt != nullptr && *halt != 0) return;
    const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    const T r0 = convert<T>(b[3 * n + 0]), r1 = convert<T>(b[3 * n + 1]), r2 = convert<T>(b[3 * n + 2]);
    bout[3 * n + 0] = r0;
    bout[3 * n + 1] = r1;
    bout[3 * n + 2] = r2;
    first_sweep_vals<T, ET>(n, r0, r1, r2, out, E, d, K0, omega);
}

// Restriction = transpose of trilinear prolongation, then mask: coarse node (I,J,K)
// gathers the fine nodes (2I+di, 2J+dj, 2K+dk), di,dj,dk in {-1,0,1}, with weight
// prod (1 if offset 0 else 1/2). `cd` are the coarse element counts.
template <typename T>
__device__ __forceinline__ void restrict_vals(long long n, const T* __restrict__ r, GridDims cd, T& s0, T& s1, T& s2)
{
    const int CX = cd.nx + 1, CY = cd.ny + 1;
    int I, J, K;
    node_coords(n, CX, CY, I, J, K);
    s0 = s1 = s2 = T(0);
    const unsigned fb = fix_bits(cd, n, I);
    if (fb == 7u) return;
    const int FX = 2 * cd.nx + 1, FY = 2 * cd.ny + 1, FZ = 2 * cd.nz + 1;
#pragma unroll
    for (int dk = -1; dk <= 1; ++dk) {
        const int fk = 2 * K + dk;
        if (fk < 0 || fk >= FZ) continue;
#pragma unroll
        for (int dj = -1; dj <= 1; ++dj) {
            const int fj = 2 * J + dj;
            if (fj < 0 || fj >= FY) continue;
#pragma unroll
            for (int di = -1; di <= 1; ++di) {
                const int fi = 2 * I + di;
                if (fi < 0 || fi >= FX) continue;   // (fi < 0 only on supports other than the clamped face)
                const T w = T((di ? 0.5 : 1.0) * (dj ? 0.5 : 1.0) * (dk ? 0.5 : 1.0));
                const long long m = fi + (long long)FX * (fj + (long long)FY * fk);
                s0 = fma(w, r[3 * m + 0], s0);
                s1 = fma(w, r[3 * m + 1], s1);
                s2 = fma(w, r[3 * m + 2], s2);
            }
        }
    }
    if (fb & 1u) s0 = T(0);
    if (fb & 2u) s1 = T(0);
    if (fb & 4u) s2 = T(0);
}

template <typename T>
__device__ __forceinline__ void restrict_node(long long n, const T* __restrict__ r, T* __restrict__ bc, GridDims cd)
{
    T s0, s1, s2;
    restrict_vals<T>(n, r, cd, s0, s1, s2);
    bc[3 * n + 0] = s0;
    bc[3 * n + 1] = s1;
    bc[3 * n + 2] = s2;
}

template <typename T>
__global__ void __launch_bounds__(256)
restrict_kernel(const T* __restrict__ r, T* __restrict__ bc, GridDims cd, const int* __restrict__ halt)
{
    if (halt != nullptr && *halt != 0) return;
    const long long nn = (long long)(cd.nx + 1) * (cd.ny + 1) * (cd.nz + 1);
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    restrict_node<T>(n, r, bc, cd);
}

// Restriction into a coarse level fused with that level's first sweep from x = 0:
// the sweep needs b only at its own node, so the thread that forms b_n sweeps it.
// Stores b (for the level's later sweeps and residual) and x. Same arithmetic as
// restrict_kernel followed by first_sweep_kernel.
template <typename T>
__global__ void __launch_bounds__(256)
restrict_first_sweep_kernel(const T* __restrict__ r, T* __restrict__ bc, T* __restrict__ xc,
                            const T* __restrict__ Ec, GridDims cd, const __grid_constant__ K0Param<T> K0, T omega,
                            const int* __restrict__ halt)
{
    if (halt != nullptr && *halt != 0) return;
    const long long nn = (long long)(cd.nx + 1) * (cd.ny + 1) * (cd.nz + 1);
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    T s0, s1, s2;
    restrict_vals<T>(n, r, cd, s0, s1, s2);
    bc[3 * n + 0] = s0;
    bc[3 * n + 1] = s1;
    bc[3 * n + 2] = s2;
    first_sweep_vals<T, T>(n, s0, s1, s2, xc, Ec, cd, K0, omega);
}

// x += P xc (trilinear interpolation, fine nodes on the fixed face untouched).
template <typename T, typename CT>
__device__ __forceinline__ void prolong_node(long long n, T* __restrict__ x, const CT* __restrict__ xc, GridDims fd)
{
    const int FX = fd.nx + 1, FY = fd.ny + 1;
    int i, j, k;
    node_coords(n, FX, FY, i, j, k);
    const unsigned fb = fix_bits(fd, n, i);
    if (fb == 7u) return;
    const int CX = fd.nx / 2 + 1, CY = fd.ny / 2 + 1;
    int Is[2], Js[2], Ks[2];
    T wi[2], wj[2], wk[2];
    int ni, nj, nk;
    if (i & 1) { Is[0] = (i - 1) / 2; Is[1] = (i + 1) / 2; wi[0] = wi[1] = T(0.5); ni = 2; }
    else { Is[0] = i / 2; wi[0] = T(1); ni = 1; }
    if (j & 1) { Js[0] = (j - 1) / 2; Js[1] = (j + 1) / 2; wj[0] = wj[1] = T(0.5); nj = 2; }
    else { Js[0] = j / 2; wj[0] = T(1); nj = 1; }
    if (k & 1) { Ks[0] = (k - 1) / 2; Ks[1] = (k + 1) / 2; wk[0] = wk[1] = T(0.5); nk = 2; }
    else { Ks[0] = k / 2; wk[0] = T(1); nk = 1; }
    T s0 = 0, s1 = 0, s2 = 0;
    for (int c = 0; c < nk; ++c)
        for (int bb = 0; bb < nj; ++bb)
            for (int a = 0; a < ni; ++a) {
                const T w = wi[a] * wj[bb] * wk[c];
                const long long m = Is[a] + (long long)CX * (Js[bb] + (long long)CY * Ks[c]);
                s0 = fma(w, (T)xc[3 * m + 0], s0);
                s1 = fma(w, (T)xc[3 * m + 1], s1);
                s2 = fma(w, (T)xc[3 * m + 2], s2);
            }
    if (!(fb & 1u)) x[3 * n + 0] += s0;
    if (!(fb & 2u)) x[3 * n + 1] += s1;
    if (!(fb & 4u)) x[3 * n + 2] += s2;
}

template <typename T, typename CT>
__global__ void __launch_bounds__(256)
prolong_add_kernel(T* __restrict__ x, const CT* __restrict__ xc, GridDims fd, const int* __restrict__ halt)
{
    if (halt != nullptr && *halt != 0) return;
    const long long nn = (long long)(fd.nx + 1) * (fd.ny + 1) * (fd.nz + 1);
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    prolong_node<T, CT>(n, x, xc, fd);
}

// ---------------------------------------------------------------- setup -------

// E_e = (rho_min + (1 - rho_min) rho_hat_e^p) * scale  (Eq. floor_scaling; scale = E0*h
// is folded in by the caller). Integer p by repeated multiplication.
__global__ void modulus_fp64_kernel(const double* __restrict__ rho, double* __restrict__ E, long long n,
                                    double rho_min, double p, int p_int, double scale)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double r = rho[e];
    double rp;
    if (p_int > 0) {
        rp = r;
        for (int q = 1; q < p_int; ++q) rp *= r;
    } else {
        rp = pow(r, p);
    }
    E[e] = (rho_min + (1.0 - rho_min) * rp) * scale;
}

// FP32 modulus from the BF16-stored density (the mixed-precision V-cycle's fine level).
__global__ void modulus_fp32_kernel(const __nv_bfloat16* __restrict__ rho, float* __restrict__ E, long long n,
                                    float rho_min, float p, int p_int, float scale)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float r = __bfloat162float(rho[e]);
    float rp;
    if (p_int > 0) {
        rp = r;
        for (int q = 1; q < p_int; ++q) rp *= r;
    } else {
        rp = powf(r, p);
    }
    E[e] = (rho_min + (1.0f - rho_min) * rp) * scale;
}

// Coarse scaled modulus: E_c h_c = mean(E_children) * 2 h_f = sum(E_children h_f) / 4.
template <typename ET>
__global__ void coarsen_kernel(const ET* __restrict__ Ef, ET* __restrict__ Ec, GridDims cd)
{
    const long long nc = (long long)cd.nx * cd.ny * cd.nz;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nc) return;
    const int ex = (int)(e % cd.nx);
    const long long t = e / cd.nx;
    const int ey = (int)(t % cd.ny), ez = (int)(t / cd.ny);
    const int fx = 2 * cd.nx, fy = 2 * cd.ny;
    ET s = 0;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx)
                s += Ef[(2 * ex + dx) + (long long)fx * ((2 * ey + dy) + (long long)fy * (2 * ez + dz))];
    Ec[e] = s * ET(0.25);
}

// Density check (finite, in [0,1]) and BF16 copy. bad[0] is set to 1 on a violation.
__global__ void density_check_kernel(const double* __restrict__ rho, __nv_bfloat16* __restrict__ r16,
                                     double* __restrict__ r64, long long n, int* __restrict__ bad)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double r = rho[e];
    if (!(r >= 0.0 && r <= 1.0)) atomicExch(bad, 1);   // NaN fails both comparisons
    r64[e] = r;
    r16[e] = __double2bfloat16(r);
}

// Per-block [count of rho == 0, sum rho, sum rho^2] for the selector's density inputs.
__global__ void __launch_bounds__(256)
density_stats_kernel(const double* __restrict__ rho, long long n, double* __restrict__ partial)
{
    __shared__ double red[3][8];
    const long long chunk = (n + gridDim.x - 1) / gridDim.x;
    const long long r0 = (long long)blockIdx.x * chunk;
    const long long r1 = r0 + chunk < n ? r0 + chunk : n;
    double a[3] = {0.0, 0.0, 0.0};
    for (long long e = r0 + threadIdx.x; e < r1; e += blockDim.x) {
        const double r = rho[e];
        a[0] += (r == 0.0) ? 1.0 : 0.0;
        a[1] += r;
        a[2] = fma(r, r, a[2]);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        double v = a[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
        partial[3 * blockIdx.x + threadIdx.x] = s;
    }
}

// Entry t of a dense coarsest matrix: row r and column c among all ndof DOFs (idx null,
// layout ndof x ndof), or among the free DOFs idx[0 .. m-1] (compact layout m x m).
__device__ __forceinline__ bool coarse_entry(long long t, long long ndof, const int* __restrict__ idx, int m,
                                             long long& r, long long& c)
{
    if (idx) {
        if (t >= (long long)m * m) return false;
        r = idx[t / m];
        c = idx[t % m];
        return true;
    }
    if (t >= ndof * ndof) return false;
    r = t / ndof;
    c = t % ndof;
    return true;
}

// Dense coarsest operator (row-major, over all DOFs of the coarsest level or, with idx,
// over its free DOFs only), one thread per entry: A[r][c] = sum over the elements e
// containing both nodes of E_e h K0[3 a_r + c_r][3 a_c + c_c], summed in a fixed element
// order so that the matrix (and its inverse) is bit-reproducible.
__global__ void coarse_assemble_kernel(const double* __restrict__ E, double* __restrict__ A, GridDims d,
                                       const __grid_constant__ K0Param<double> K0, const int* __restrict__ idx = nullptr,
                                       int m = 0)
{
    const int NX = d.nx + 1, NY = d.ny + 1, NZ = d.nz + 1;
    const long long ndof = 3LL * NX * NY * NZ;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long r, c;
    if (!coarse_entry(t, ndof, idx, m, r, c)) return;
    const long long nr = r / 3, nc = c / 3;
    const int cr = (int)(r % 3), cc = (int)(c % 3);
    const int ir = (int)(nr % NX), jr = (int)((nr / NX) % NY), kr = (int)(nr / ((long long)NX * NY));
    const int ic = (int)(nc % NX), jc = (int)((nc / NX) % NY), kc = (int)(nc / ((long long)NX * NY));
    double s = 0.0;
    if (abs(ir - ic) <= 1 && abs(jr - jc) <= 1 && abs(kr - kc) <= 1) {
        const int x0 = max(max(ir, ic) - 1, 0), x1 = min(min(ir, ic), d.nx - 1);
        const int y0 = max(max(jr, jc) - 1, 0), y1 = min(min(jr, jc), d.ny - 1);
        const int z0 = max(max(kr, kc) - 1, 0), z1 = min(min(kr, kc), d.nz - 1);
        for (int ez = z0; ez <= z1; ++ez)
            for (int ey = y0; ey <= y1; ++ey)
                for (int ex = x0; ex <= x1; ++ex) {
                    const int ar = local_index(ir - ex, jr - ey, kr - ez);
                    const int ac = local_index(ic - ex, jc - ey, kc - ez);
                    s = fma(E[ex + (long long)d.nx * (ey + (long long)d.ny * ez)],
                            K0.k[(3 * ar + cr) * 24 + 3 * ac + cc], s);
                }
    }
    A[t] = s;
}

// The free DOFs of a level in ascending order (idx[0 .. m-1]), each DOF's position among
// them (pos[q], -1 for a fixed DOF), and m (*m_out). One warp.
// Order of the coarsest level's free DOFs: nodes run along the axis with the fewest nodes
// first and the one with the most last (ties in x, y, z order), the three components of a
// node together. Neighbouring nodes then differ by at most 1 + N_a + N_a N_b positions
// (N_a <= N_b the two smallest node counts), which bounds the operator's band at
// 3 (1 + N_a + N_a N_b) + 2; at 13 x 7 x 7 nodes that is 173 against 317 in x-fastest
// order. ax[0] is the fastest axis (0 = x, 1 = y, 2 = z).
__host__ __device__ inline void coarse_axes(const GridDims& d, int ax[3])
{
    const int N[3] = {d.nx + 1, d.ny + 1, d.nz + 1};
    ax[0] = 0, ax[1] = 1, ax[2] = 2;
    for (int i = 1; i < 3; ++i)   // stable insertion sort by node count
        for (int j = i; j > 0 && N[ax[j]] < N[ax[j - 1]]; --j) {
            const int t = ax[j];
            ax[j] = ax[j - 1];
            ax[j - 1] = t;
        }
}

__host__ __device__ inline int coarse_band(const GridDims& d)
{
    const int N[3] = {d.nx + 1, d.ny + 1, d.nz + 1};
    int ax[3];
    coarse_axes(d, ax);
    return 3 * (1 + N[ax[0]] + N[ax[0]] * N[ax[1]]) + 2;
}

// pos[q]: the compact index of DOF q (-1 when fixed); idx[i]: the DOF at compact index i;
// *m_out: the free DOF count. One warp, in the order of coarse_axes.
__global__ void coarse_map_kernel(GridDims d, int* __restrict__ pos, int* __restrict__ idx, int* __restrict__ m_out)
{
    const int N[3] = {d.nx + 1, d.ny + 1, d.nz + 1};
    int ax[3];
    coarse_axes(d, ax);
    const long long ndof = 3LL * N[0] * N[1] * N[2];
    const unsigned lane = threadIdx.x;
    int base = 0;
    for (long long t0 = 0; t0 < ndof; t0 += 32) {
        const long long t = t0 + lane;
        long long q = -1;
        if (t < ndof) {
            int v[3];
            long long r = t / 3;
            v[ax[0]] = (int)(r % N[ax[0]]);
            r /= N[ax[0]];
            v[ax[1]] = (int)(r % N[ax[1]]);
            v[ax[2]] = (int)(r / N[ax[1]]);
            q = 3 * (v[0] + (long long)N[0] * (v[1] + (long long)N[1] * v[2])) + t % 3;
        }
        const bool fr = q >= 0 && !fix_dof(d, q);
        const unsigned bal = __ballot_sync(0xffffffffu, fr);
        const int at = base + __popc(bal & ((1u << lane) - 1u));
        if (q >= 0) pos[q] = fr ? at : -1;
        if (fr) idx[at] = (int)q;
        base += __popc(bal);
    }
    if (lane == 0) *m_out = base;
}

// Fixed DOFs: zero row and column, unit diagonal.
__global__ void coarse_fix_kernel(double* __restrict__ A, GridDims d)
{
    const int NX = d.nx + 1, NY = d.ny + 1, NZ = d.nz + 1;
    const long long ndof = 3LL * NX * NY * NZ;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ndof * ndof) return;
    const long long r = t / ndof, c = t % ndof;
    const bool fr = fix_dof(d, r), fc = fix_dof(d, c);
    if (fr || fc) A[t] = (r == c) ? 1.0 : 0.0;
}

// Cantilever load and free mask.
__global__ void cantilever_load_kernel(double* __restrict__ f, GridDims d)
{
    const long long ndof = 3LL * (d.nx + 1) * (d.ny + 1) * (d.nz + 1);
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ndof) return;
    const long long nl = d.nx + (long long)(d.nx + 1) * (d.ny / 2 + (long long)(d.ny + 1) * (d.nz / 2));
    f[t] = (t == 3 * nl + 2) ? -1.0 : 0.0;
}

__global__ void free_mask_kernel(uint8_t* __restrict__ mask, GridDims d)
{
    const long long ndof = 3LL * (d.nx + 1) * (d.ny + 1) * (d.nz + 1);
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ndof) return;
    mask[t] = !fix_dof(d, t);
}

// The bridge's load: a unit pressure on the top face y = ny h, pointing down (-y), as
// consistent nodal forces -p h^2 / 4 from each of the (up to four) top faces around a
// node (the bilinear face integral of a uniform pressure); 0 on fixed DOFs. h2 = h^2.
__global__ void bridge_load_kernel(double* __restrict__ f, GridDims d, double h2)
{
    const int NX = d.nx + 1, NY = d.ny + 1;
    const long long ndof = 3LL * NX * NY * (d.nz + 1);
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ndof) return;
    const long long n = t / 3;
    const int c = (int)(t - 3 * n);
    int i, j, k;
    node_coords(n, NX, NY, i, j, k);
    double v = 0.0;
    if (c == 1 && j == d.ny && !fix_dof(d, t)) {
        const int fx = (i > 0) + (i < d.nx), fz = (k > 0) + (k < d.nz);   // top faces touching the node
        v = -0.25 * h2 * (double)(fx * fz);
    }
    f[t] = v;
}

// Per-node fixed components of the bridge's supports on level l of a hierarchy whose
// fine grid has nz_f elements in z: fine node (i, j, k) is fixed in every component at
// (0, 0, k) and in y and z at (nx_f, 0, k) for k in {0, nz_f/2, nz_f}; coarse node
// (I, J, K) takes the components of fine node (2^l I, 2^l J, 2^l K) (injection).
__global__ void bridge_fix_kernel(uint8_t* __restrict__ fix, GridDims d, int level, int nx_f, int nz_f)
{
    const int NX = d.nx + 1, NY = d.ny + 1;
    const long long nn = (long long)NX * NY * (d.nz + 1);
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    int I, J, K;
    node_coords(n, NX, NY, I, J, K);
    const int i = I << level, j = J << level, k = K << level;
    unsigned b = 0;
    if (j == 0 && (k == 0 || 2 * k == nz_f || k == nz_f)) {
        if (i == 0) b = 7u;
        else if (i == nx_f) b = 6u;
    }
    fix[n] = (uint8_t)b;
}

// dc_e = -p (1 - rho_min) rho_e^(p-1) u_e^T K0 u_e * E0 h (scale folded in K0/caller).
__global__ void __launch_bounds__(256)
sensitivity_kernel(const double* __restrict__ u, const double* __restrict__ rho, double* __restrict__ dc,
                   GridDims d, const __grid_constant__ K0Param<double> K0, double coef, double pm1,
                   int pm1_int)
{
    const long long ne = (long long)d.nx * d.ny * d.nz;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const int ex = (int)(e % d.nx);
    const long long t = e / d.nx;
    const int ey = (int)(t % d.ny), ez = (int)(t / d.ny);
    const int NX = d.nx + 1, NY = d.ny + 1;
    double ue[24];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int ox = (a == 1 || a == 2 || a == 5 || a == 6), oy = (a == 2 || a == 3 || a == 6 || a == 7), oz = a >= 4;
        const int ni = ex + ox;
        const long long m = ni + (long long)NX * ((ey + oy) + (long long)NY * (ez + oz));
        const unsigned mb = fix_bits(d, m, ni);
#pragma unroll
        for (int c = 0; c < 3; ++c) ue[3 * a + c] = ((mb >> c) & 1u) ? 0.0 : u[3 * m + c];
    }
    double energy = 0.0;
#pragma unroll
    for (int p = 0; p < 24; ++p) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < 24; ++q) s = fma(K0.k[p * 24 + q], ue[q], s);
        energy = fma(ue[p], s, energy);
    }
    const double r = rho[e];
    double rp;
    if (pm1_int >= 0) {
        rp = 1.0;
        for (int q = 0; q < pm1_int; ++q) rp *= r;
    } else {
        rp = pow(r, pm1);
    }
    dc[e] = coef * rp * energy;
}

}  // namespace gf

namespace gf {

// FP32 node stencils on a shared-memory tile (the V-cycle's level operators).
// A CTA stages the tile's nodes plus a one-node halo of x and the tile's elements
// plus a one-element halo of E; each thread then reads its 27 neighbouring nodes
// once and feeds every value to the (element, row) accumulators that use it, so
// the inner loop is shared-memory loads and FMAs with K0 from the parameter bank.
constexpr int TSX = 16, TSY = 4, TSZ = 2;                      // nodes per tile (128 threads)
constexpr int THX = TSX + 2, THY = TSY + 2, THZ = TSZ + 2;      // node halo
constexpr int TEX = TSX + 1, TEY = TSY + 1, TEZ = TSZ + 1;      // element halo

template <int MODE, typename BT, typename OT>
__global__ void __launch_bounds__(128)
tiled_stencil_f32_kernel(const float* __restrict__ x, const BT* __restrict__ b, OT* __restrict__ out,
                         const float* __restrict__ E, GridDims d, const __grid_constant__ K0Param<float> K0,
                         float omega, const int* __restrict__ halt)
{
    if (halt != nullptr && *halt != 0) return;
    __shared__ float sx[THX * THY * THZ * 3];
    __shared__ float sE[TEX * TEY * TEZ];
    const int NX = d.nx + 1, NY = d.ny + 1, NZ = d.nz + 1;
    const int i0 = blockIdx.x * TSX, j0 = blockIdx.y * TSY, k0 = blockIdx.z * TSZ;
    const int tid = threadIdx.x + TSX * (threadIdx.y + TSY * threadIdx.z);
    for (int q = tid; q < THX * THY * THZ * 3; q += 128) {
        const int c = q % 3, hn = q / 3;
        const int hx = hn % THX, hy = (hn / THX) % THY, hz = hn / (THX * THY);
        const int gi = i0 - 1 + hx, gj = j0 - 1 + hy, gk = k0 - 1 + hz;
        float v = 0.f;
        if (gi >= 1 && gi < NX && gj >= 0 && gj < NY && gk >= 0 && gk < NZ)
            v = x[3 * ((long long)gi + (long long)NX * (gj + (long long)NY * gk)) + c];
        sx[q] = v;
    }
    for (int q = tid; q < TEX * TEY * TEZ; q += 128) {
        const int ex = q % TEX, ey = (q / TEX) % TEY, ez = q / (TEX * TEY);
        const int ge = i0 - 1 + ex, gey = j0 - 1 + ey, gez = k0 - 1 + ez;
        float v = 0.f;
        if (ge >= 0 && ge < d.nx && gey >= 0 && gey < d.ny && gez >= 0 && gez < d.nz)
            v = E[ge + (long long)d.nx * (gey + (long long)d.ny * gez)];
        sE[q] = v;
    }
    __syncthreads();
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    const int gi = i0 + tx, gj = j0 + ty, gk = k0 + tz;
    if (gi >= NX || gj >= NY || gk >= NZ) return;
    const long long n = gi + (long long)NX * (gj + (long long)NY * gk);
    if (gi == 0) {
        out[3 * n + 0] = OT(0);
        out[3 * n + 1] = OT(0);
        out[3 * n + 2] = OT(0);
        return;
    }
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
                const int hn = (tx + ox) + THX * ((ty + oy) + THY * (tz + oz));
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float v = sx[3 * hn + c];
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
                                    t[e][r] = fmaf(K0.k[(3 * a + r) * 24 + 3 * bl + c], v, t[e][r]);
                            }
                }
            }
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    float d00 = 0.f, d11 = 0.f, d22 = 0.f, d01 = 0.f, d02 = 0.f, d12 = 0.f;
#pragma unroll
    for (int ez = 0; ez < 2; ++ez)
#pragma unroll
        for (int ey = 0; ey < 2; ++ey)
#pragma unroll
            for (int ex = 0; ex < 2; ++ex) {
                const int e = ex + 2 * (ey + 2 * ez);
                const float Ee = sE[(tx + ex) + TEX * ((ty + ey) + TEY * (tz + ez))];
                a0 = fmaf(Ee, t[e][0], a0);
                a1 = fmaf(Ee, t[e][1], a1);
                a2 = fmaf(Ee, t[e][2], a2);
                if (MODE == ST_SWEEP) {
                    const int a = local_index(1 - ex, 1 - ey, 1 - ez);
                    d00 = fmaf(Ee, K0.k[(3 * a + 0) * 24 + 3 * a + 0], d00);
                    d11 = fmaf(Ee, K0.k[(3 * a + 1) * 24 + 3 * a + 1], d11);
                    d22 = fmaf(Ee, K0.k[(3 * a + 2) * 24 + 3 * a + 2], d22);
                    d01 = fmaf(Ee, K0.k[(3 * a + 0) * 24 + 3 * a + 1], d01);
                    d02 = fmaf(Ee, K0.k[(3 * a + 0) * 24 + 3 * a + 2], d02);
                    d12 = fmaf(Ee, K0.k[(3 * a + 1) * 24 + 3 * a + 2], d12);
                }
            }
    if (MODE == ST_APPLY) {
        out[3 * n + 0] = OT(a0);
        out[3 * n + 1] = OT(a1);
        out[3 * n + 2] = OT(a2);
        return;
    }
    const float r0 = (float)b[3 * n + 0] - a0;
    const float r1 = (float)b[3 * n + 1] - a1;
    const float r2 = (float)b[3 * n + 2] - a2;
    if (MODE == ST_RESID) {
        out[3 * n + 0] = OT(r0);
        out[3 * n + 1] = OT(r1);
        out[3 * n + 2] = OT(r2);
        return;
    }
    const float c00 = d11 * d22 - d12 * d12;
    const float c01 = d02 * d12 - d01 * d22;
    const float c02 = d01 * d12 - d02 * d11;
    const float c11 = d00 * d22 - d02 * d02;
    const float c12 = d01 * d02 - d00 * d12;
    const float c22 = d00 * d11 - d01 * d01;
    const float det = d00 * c00 + d01 * c01 + d02 * c02;
    const float s = omega / det;
    const int hc = (tx + 1) + THX * ((ty + 1) + THY * (tz + 1));
    out[3 * n + 0] = OT(sx[3 * hc + 0] + s * (c00 * r0 + c01 * r1 + c02 * r2));
    out[3 * n + 1] = OT(sx[3 * hc + 1] + s * (c01 * r0 + c11 * r1 + c12 * r2));
    out[3 * n + 2] = OT(sx[3 * hc + 2] + s * (c02 * r0 + c12 * r1 + c22 * r2));
}

}  // namespace gf

namespace gf {

// Node stencil that reads each of the 27 neighbouring nodes once (81 loads, 32-bit
// offsets from the node's own address) and feeds every value to the (element, row)
// accumulators that use it. Same modes and types as node_stencil_kernel.
template <typename T, int MODE, typename BT, typename OT>
__global__ void __launch_bounds__(256)
node_stencil27_kernel(const T* __restrict__ x, const BT* __restrict__ b, OT* __restrict__ out,
                      const T* __restrict__ E, GridDims d, const __grid_constant__ K0Param<T> K0, T omega,
                      const int* __restrict__ halt)
{
    if (halt != nullptr && *halt != 0) return;
    const int NX = d.nx + 1, NY = d.ny + 1;
    const int nn = NX * NY * (d.nz + 1);
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    const int i = n % NX, j = (n / NX) % NY, k = n / (NX * NY);
    if (i == 0) {
        out[3 * (long long)n + 0] = OT(0);
        out[3 * (long long)n + 1] = OT(0);
        out[3 * (long long)n + 2] = OT(0);
        return;
    }
    const T* xn = x + 3 * (long long)n;
    const int sy = 3 * NX, sz = 3 * NX * NY;
    T t[8][3];
#pragma unroll
    for (int e = 0; e < 8; ++e)
#pragma unroll
        for (int r = 0; r < 3; ++r) t[e][r] = T(0);
#pragma unroll
    for (int oz = 0; oz < 3; ++oz) {
        const bool okz = (oz != 0 || k > 0) && (oz != 2 || k < d.nz);
#pragma unroll
        for (int oy = 0; oy < 3; ++oy) {
            const bool oky = okz && (oy != 0 || j > 0) && (oy != 2 || j < d.ny);
#pragma unroll
            for (int ox = 0; ox < 3; ++ox) {
                // the clamped face (i - 1 + ox == 0) reads as zero
                const bool ok = oky && (ox != 0 || i > 1) && (ox != 2 || i < d.nx);
                const T* p = xn + (ox - 1) * 3 + (oy - 1) * sy + (oz - 1) * sz;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const T v = ok ? p[c] : T(0);
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
                                for (int r = 0; r < 3; ++r) t[e][r] = fma(K0.k[(3 * a + r) * 24 + 3 * bl + c], v, t[e][r]);
                            }
                }
            }
        }
    }
    T a0 = 0, a1 = 0, a2 = 0;
    T d00 = 0, d11 = 0, d22 = 0, d01 = 0, d02 = 0, d12 = 0;
#pragma unroll
    for (int ez = 0; ez < 2; ++ez)
#pragma unroll
        for (int ey = 0; ey < 2; ++ey)
#pragma unroll
            for (int ex = 0; ex < 2; ++ex) {
                const int cx = i - 1 + ex, cy = j - 1 + ey, cz = k - 1 + ez;
                if (cx < 0 || cx >= d.nx || cy < 0 || cy >= d.ny || cz < 0 || cz >= d.nz) continue;
                const int e = ex + 2 * (ey + 2 * ez);
                const T Ee = E[cx + d.nx * (cy + d.ny * cz)];
                a0 = fma(Ee, t[e][0], a0);
                a1 = fma(Ee, t[e][1], a1);
                a2 = fma(Ee, t[e][2], a2);
                if (MODE == ST_SWEEP) {
                    const int a = local_index(1 - ex, 1 - ey, 1 - ez);
                    d00 = fma(Ee, K0.k[(3 * a + 0) * 24 + 3 * a + 0], d00);
                    d11 = fma(Ee, K0.k[(3 * a + 1) * 24 + 3 * a + 1], d11);
                    d22 = fma(Ee, K0.k[(3 * a + 2) * 24 + 3 * a + 2], d22);
                    d01 = fma(Ee, K0.k[(3 * a + 0) * 24 + 3 * a + 1], d01);
                    d02 = fma(Ee, K0.k[(3 * a + 0) * 24 + 3 * a + 2], d02);
                    d12 = fma(Ee, K0.k[(3 * a + 1) * 24 + 3 * a + 2], d12);
                }
            }
    const long long o = 3 * (long long)n;
    if (MODE == ST_APPLY) {
        out[o + 0] = OT(a0);
        out[o + 1] = OT(a1);
        out[o + 2] = OT(a2);
        return;
    }
    const T r0 = T(b[o + 0]) - a0, r1 = T(b[o + 1]) - a1, r2 = T(b[o + 2]) - a2;
    if (MODE == ST_RESID) {
        out[o + 0] = OT(r0);
        out[o + 1] = OT(r1);
        out[o + 2] = OT(r2);
        return;
    }
    const T c00 = d11 * d22 - d12 * d12;
    const T c01 = d02 * d12 - d01 * d22;
    const T c02 = d01 * d12 - d02 * d11;
    const T c11 = d00 * d22 - d02 * d02;
    const T c12 = d01 * d02 - d00 * d12;
    const T c22 = d00 * d11 - d01 * d01;
    const T det = d00 * c00 + d01 * c01 + d02 * c02;
    const T s = omega / det;
    out[o + 0] = OT(xn[0] + s * (c00 * r0 + c01 * r1 + c02 * r2));
    out[o + 1] = OT(xn[1] + s * (c01 * r0 + c11 * r1 + c12 * r2));
    out[o + 2] = OT(xn[2] + s * (c02 * r0 + c12 * r1 + c22 * r2));
}

}  // namespace gf
