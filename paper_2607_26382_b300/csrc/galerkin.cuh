// Galerkin coarse operators (Table solver-config): K_{l+1} = P^T K_l P with the 2:1
// trilinear prolongation P, held as one dense 24x24 matrix per coarse element.
//
// A fine element lies inside one coarse element, and there P is a fixed map T_c from
// the coarse element's 24 DOFs to the 24 DOFs of its child c: child-local node a takes
// coarse-local node b with the trilinear weight W_c[a][b] (products of 1, 1/2 per axis),
// the same for each displacement component. So P^T K P assembles element by element,
//   K_C = sum_{c < 8} T_c^T K_c T_c,   (T_c^T K T_c)[3b+i][3b'+j] = sum_{a,a'} W_c[a][b] K[3a+i][3a'+j] W_c[a'][b'],
// with K_c = E_c K0 on the finest level (E_c carries the element edge h).
// Fixed DOFs: a fine node on the clamped x = 0 face interpolates only from coarse nodes
// on that face, so the masked prolongation M_f P M_c equals P M_c, and on free coarse
// DOFs M_c P^T M_f K M_f P M_c is the element-wise sum above of the unmasked matrices.
// The matrices are kept unmasked; the kernels read fixed nodes as 0 and write them as 0.
#pragma once
#include <cuda_runtime.h>
#include <type_traits>

namespace gf {

constexpr int GAL_FIRST = 3;   // out = omega D_n^{-1} b: the first sweep from x = 0
constexpr int GAL_CHEB = 4;    // Chebyshev step: d = c1 d + c2 D_n^{-1} (b - K x), out = x + d (x may be null)
constexpr int GAL_KE = 576;    // 24 x 24 entries per element, row-major

// (x, y, z) offsets of element-local node a (inverse of local_index)
__host__ __device__ inline void local_xyz(int a, int& x, int& y, int& z)
{
    z = a >> 2;
    const int r = a & 3;
    x = (r == 1 || r == 2) ? 1 : 0;
    y = (r >= 2) ? 1 : 0;
}

// W_c[a][b]: weight of coarse-local node b at node a of child c. Per axis, the fine
// node sits at s = c + a half-steps of the coarse element: weight 1 - s/2 for b = 0,
// s/2 for b = 1.
__host__ __device__ inline double gal_weight(int c, int a, int b)
{
    int cx, cy, cz, ax, ay, az, bx, by, bz;
    local_xyz(c, cx, cy, cz);
    local_xyz(a, ax, ay, az);
    local_xyz(b, bx, by, bz);
    const int sx = cx + ax, sy = cy + ay, sz = cz + az;
    const double wx = bx ? 0.5 * sx : 1.0 - 0.5 * sx;
    const double wy = by ? 0.5 * sy : 1.0 - 0.5 * sy;
    const double wz = bz ? 0.5 * sz : 1.0 - 0.5 * sz;
    return wx * wy * wz;
}

// fine element index of child c of coarse element (X, Y, Z); cd = coarse dims
__device__ __forceinline__ long long gal_child(long long e, int c, GridDims cd)
{
    const long long X = e % cd.nx, Y = (e / cd.nx) % cd.ny, Z = e / ((long long)cd.nx * cd.ny);
    int cx, cy, cz;
    local_xyz(c, cx, cy, cz);
    const long long fnx = 2LL * cd.nx, fny = 2LL * cd.ny;
    return (2 * X + cx) + fnx * ((2 * Y + cy) + fny * (2 * Z + cz));
}

// First coarse level from the finest: K_C[q] = sum_c E[child c] G[c][q], G_c = T_c^T K0 T_c
// (host-built, FP64). One thread per entry; the FP64 result, and optionally its FP32
// rounding.
template <typename ET>
__global__ void gal_first_level_kernel(const ET* __restrict__ Ef, const double* __restrict__ G,
                                       double* __restrict__ Kc, float* __restrict__ Kc32, GridDims cd)
{
    const long long ne = (long long)cd.nx * cd.ny * cd.nz;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ne * GAL_KE) return;
    const long long e = t / GAL_KE;
    const int q = (int)(t % GAL_KE);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s = fma((double)Ef[gal_child(e, c, cd)], G[c * GAL_KE + q], s);
    if (Kc) Kc[t] = s;
    if (Kc32) Kc32[t] = (float)s;
}

// Next coarse level from element matrices: K_C = sum_c T_c^T K_c T_c, skipping the
// zero weights, in a fixed (c, a, a') order. One thread per entry.
__global__ void gal_coarsen_kernel(const double* __restrict__ Kf, double* __restrict__ Kc,
                                   float* __restrict__ Kc32, GridDims cd)
{
    const long long ne = (long long)cd.nx * cd.ny * cd.nz;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ne * GAL_KE) return;
    const long long e = t / GAL_KE;
    const int q = (int)(t % GAL_KE);
    const int R = q / 24, S = q % 24;
    const int b = R / 3, i = R % 3, bp = S / 3, j = S % 3;
    double s = 0.0;
    for (int c = 0; c < 8; ++c) {
        const double* K = Kf + gal_child(e, c, cd) * GAL_KE;
        for (int a = 0; a < 8; ++a) {
            const double wa = gal_weight(c, a, b);
            if (wa == 0.0) continue;
            double u = 0.0;
            for (int ap = 0; ap < 8; ++ap) {
                const double wp = gal_weight(c, ap, bp);
                if (wp == 0.0) continue;
                u = fma(wp, K[(3 * a + i) * 24 + 3 * ap + j], u);
            }
            s = fma(wa, u, s);
        }
    }
    if (Kc) Kc[t] = s;
    if (Kc32) Kc32[t] = (float)s;
}

// The level operator from element matrices (node_stencil_kernel's modes, plus
// GAL_FIRST), eight threads per node: thread el of a node's group takes the adjacent
// element (i - 1 + (el & 1), j - 1 + (el >> 1 & 1), k - 1 + (el >> 2)), where the node is
// local node a, and forms rows 3a..3a+2 of that element's matrix times its node values
// (fixed nodes read as 0) and, to smooth, the element's 3x3 block at (a, a). A xor
// butterfly over the eight lanes sums the elements in a fixed order, and the group's
// first lane writes the node. Coarse levels have few nodes; eight threads per node
// keep several blocks on every SM and the element rows' loads in parallel.
template <typename T, int MODE, typename BT, typename OT>
__global__ void __launch_bounds__(256)
gal_node_kernel(const T* __restrict__ x, const BT* __restrict__ b, OT* __restrict__ out,
                const T* __restrict__ Ke, GridDims d, T omega, const int* __restrict__ halt,
                T* __restrict__ dv, const double* __restrict__ coef)
{
    if (halt != nullptr && *halt != 0) return;   // uniform over the grid
    const int NX = d.nx + 1, NY = d.ny + 1;
    const long long nn = (long long)NX * NY * (d.nz + 1);
    const long long n = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int el = threadIdx.x & 7;
    const bool active = n < nn;                  // uniform over the node's eight lanes
    int i = 0, j = 0, k = 0;
    if (active) node_coords(n, NX, NY, i, j, k);
    T a0 = 0, a1 = 0, a2 = 0;
    T d00 = 0, d11 = 0, d22 = 0, d01 = 0, d02 = 0, d12 = 0;
    const int ox = el & 1, oy = (el >> 1) & 1, oz = el >> 2;
    const int ex = i - 1 + ox, ey = j - 1 + oy, ez = k - 1 + oz;
    if (active && i != 0 && ex >= 0 && ex < d.nx && ey >= 0 && ey < d.ny && ez >= 0 && ez < d.nz) {
        const int a = local_index(1 - ox, 1 - oy, 1 - oz);
        const T* Kr = Ke + (ex + (long long)d.nx * (ey + (long long)d.ny * ez)) * GAL_KE + 3 * a * 24;
        if (MODE != GAL_FIRST && !(MODE == GAL_CHEB && x == nullptr)) {
            T u[24];   // the element's node values, local node order (fixed nodes read as 0)
#pragma unroll
            for (int bl = 0; bl < 8; ++bl) {
                int bx, by, bz;
                local_xyz(bl, bx, by, bz);
                const bool fixed = ex + bx == 0;
                const long long m = (ex + bx) + (long long)NX * ((ey + by) + (long long)NY * (ez + bz));
#pragma unroll
                for (int c = 0; c < 3; ++c) u[3 * bl + c] = fixed ? T(0) : x[3 * m + c];
            }
            // rows 3a..3a+2 as 16-byte vectors: the element's 576 values start on a 16-byte
            // boundary (cudaMalloc base), and 72 a and 24 r values are multiples of 16 bytes
            using V = typename std::conditional<sizeof(T) == sizeof(float), float4, double2>::type;
            constexpr int PER = (int)(sizeof(V) / sizeof(T));
            T acc[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const V* row = reinterpret_cast<const V*>(Kr + 24 * r);
                T s = 0;
#pragma unroll
                for (int q = 0; q < 24 / PER; ++q) {
                    const V kv = row[q];
                    if constexpr (PER == 4) {
                        s = fma(kv.x, u[4 * q + 0], s);
                        s = fma(kv.y, u[4 * q + 1], s);
                        s = fma(kv.z, u[4 * q + 2], s);
                        s = fma(kv.w, u[4 * q + 3], s);
                    } else {
                        s = fma(kv.x, u[2 * q + 0], s);
                        s = fma(kv.y, u[2 * q + 1], s);
                    }
                }
                acc[r] = s;
            }
            a0 = acc[0];
            a1 = acc[1];
            a2 = acc[2];
        }
        if (MODE == ST_SWEEP || MODE == GAL_FIRST || MODE == GAL_CHEB) {
            d00 = Kr[3 * a + 0];
            d01 = Kr[3 * a + 1];
            d02 = Kr[3 * a + 2];
            d11 = Kr[24 + 3 * a + 1];
            d12 = Kr[24 + 3 * a + 2];
            d22 = Kr[48 + 3 * a + 2];
        }
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        if (MODE == ST_SWEEP || MODE == GAL_FIRST || MODE == GAL_CHEB) {
            d00 += __shfl_xor_sync(0xffffffffu, d00, o);
            d11 += __shfl_xor_sync(0xffffffffu, d11, o);
            d22 += __shfl_xor_sync(0xffffffffu, d22, o);
            d01 += __shfl_xor_sync(0xffffffffu, d01, o);
            d02 += __shfl_xor_sync(0xffffffffu, d02, o);
            d12 += __shfl_xor_sync(0xffffffffu, d12, o);
        }
    }
    if (!active || el != 0) return;
    if (i == 0) {
        out[3 * n + 0] = OT(0);
        out[3 * n + 1] = OT(0);
        out[3 * n + 2] = OT(0);
        if (MODE == GAL_CHEB) dv[3 * n + 0] = dv[3 * n + 1] = dv[3 * n + 2] = T(0);
        return;
    }
    if (MODE == GAL_CHEB) {   // z = D^{-1} (b - K x), d = c1 d + c2 z, out = x + d
        const T zero[3] = {T(0), T(0), T(0)};
        T z[3];
        node_block_update<T, T>(d00, d11, d22, d01, d02, d12, T(b[3 * n + 0]) - a0, T(b[3 * n + 1]) - a1,
                                T(b[3 * n + 2]) - a2, zero, z, T(1));
        const T c1 = (T)coef[0], c2 = (T)coef[1];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T dn = (coef[0] != 0.0) ? c1 * dv[3 * n + c] + c2 * z[c] : c2 * z[c];
            dv[3 * n + c] = dn;
            out[3 * n + c] = OT((x != nullptr ? x[3 * n + c] : T(0)) + dn);
        }
        return;
    }
    if (MODE == ST_APPLY) {
        out[3 * n + 0] = OT(a0);
        out[3 * n + 1] = OT(a1);
        out[3 * n + 2] = OT(a2);
        return;
    }
    const T r0 = T(b[3 * n + 0]) - a0;
    const T r1 = T(b[3 * n + 1]) - a1;
    const T r2 = T(b[3 * n + 2]) - a2;
    if (MODE == ST_RESID) {
        out[3 * n + 0] = OT(r0);
        out[3 * n + 1] = OT(r1);
        out[3 * n + 2] = OT(r2);
        return;
    }
    const T zero[3] = {T(0), T(0), T(0)};
    node_block_update<T, OT>(d00, d11, d22, d01, d02, d12, r0, r1, r2, MODE == GAL_FIRST ? zero : x + 3 * n,
                             out + 3 * n, omega);
}

// Dense coarsest operator from element matrices (coarse_assemble_kernel's layouts and
// element order): A[r][c] = sum over the elements holding both nodes of K_e[3 a_r + c_r][3 a_c + c_c].
__global__ void gal_assemble_kernel(const double* __restrict__ Ke, double* __restrict__ A, GridDims d,
                                    const int* __restrict__ idx = nullptr, int m = 0)
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
                    s += Ke[(ex + (long long)d.nx * (ey + (long long)d.ny * ez)) * GAL_KE + (3 * ar + cr) * 24 +
                            3 * ac + cc];
                }
    }
    A[t] = s;
}

}  // namespace gf
