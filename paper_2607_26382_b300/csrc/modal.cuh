// FP64 matrix-free K*u through the modal (sum/difference) factorisation of K0.
//
// The frozen operator of Eq. (frozen_operator) (arXiv 2607.26382) is
// y = sum_e E_e P_e^T K0 P_e u with one 24x24 hex8 stiffness K0. Write the trilinear
// field of an element in the product basis P_beta = p_bx(x) p_by(y) p_bz(z),
// p_0 = 1, p_1 = 2s - 1 on the unit cube. Its coefficients are the unnormalised
// sums and differences m = H u_e (H: the 8x8 matrix of signs prod_k s_k^beta_k,
// s = -1 at offset 0, +1 at offset 1), so K0 = H^T Km H / 64. In that basis the 1D
// mass, stiffness and mixed integrals are diag(1, 1/3), diag(0, 4) and one entry 2,
// so Km = a(P_alpha e_d, P_beta e_c) has 45 non-zeros of 9 kinds (lambda, mu, and
// powers of 1/3):
//   diagonal (c, beta):  4 (lam + mu) b_c 3^-n + 4 mu (b_c 3^-n + n 3^-(b_c + n - 1))
//                        with b_c = beta_c and n = number of other axes with beta = 1;
//   cross (c, d != c):   beta_c = 1, beta_d = 0:  4 lam w(beta_o) m_d[beta ^ e_c ^ e_d]
//                        beta_c = 0, beta_d = 1:  4 mu  w(beta_o) m_d[beta ^ e_c ^ e_d]
//                        (o the third axis, w(0) = 1, w(1) = 1/3).
// (Checked numerically against the Gauss-integrated K0 on the host: both are the
// exact integral, and they agree to rounding.)
//
// Cost per element: the sum/difference network forward (45 FP64 adds, a face of
// the column's next node plane transformed once and reused by the element above; the
// constant mode is never formed), 45 multiply-adds in modal space with the element's 9
// coefficients E_e C (scaled once per floor, modal_scale_kernel), the transposed network
// back (54: the constant mode, a rigid translation, carries no force), and the 9 adds of
// the node gather -- 153 FP64 instructions against the 576 FMAs of the dense 24x24
// product. B300 issues FP64 at 1/64 of the FP32 rate, so this count, not memory, bounds
// the kernel.
//
// Layout of the work: a CTA owns a tile of BX x BY element columns (32 x 16 or 16 x 32,
// whichever wastes fewer warps on the grid; the tiles do not overlap) and walks them up
// a run of node planes. At each step every thread forms its element's forces, sums its
// bottom face with the top face of the element below (carried in registers, in modal
// form), transforms the face back to its four nodes and stores them in shared memory;
// after a barrier each of the (BX-1) x (BY-1) nodes inside the tile adds the four
// columns around it in a fixed order. A node on a tile boundary has columns in two or
// four tiles: each column writes its corner to that node's slot in a side buffer, and
// modal_fixup_kernel adds the four slots in the same fixed order. No atomics: the result
// does not depend on the launch shape. (The FP32 fine-level kernel below keeps tiles
// that overlap by one element column on the low x and y sides and needs no side buffer:
// its smoothing update of a node needs the node's complete residual, and a fix-up launch
// per sweep costs more there than the overlap.)
#pragma once
#include <cuda_runtime.h>
#include <algorithm>
#include <vector>
#include "stencil.cuh"

namespace gf {

struct ModalCoef {
    double diag[6];    // [b_c * 3 + n], entry 0 (the constant mode) unused; already / 64
    double cross[4];   // [lam w=1, lam w=1/3, mu w=1, mu w=1/3], already / 64
};

__host__ inline ModalCoef modal_coef(double E0, double nu)
{
    const double lam = E0 * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    const double mu = E0 / (2.0 * (1.0 + nu));
    ModalCoef c{};
    const double inv3[3] = {1.0, 1.0 / 3.0, 1.0 / 9.0};
    for (int bc = 0; bc < 2; ++bc)
        for (int n = 0; n < 3; ++n) {
            double v = 4.0 * (lam + mu) * bc * inv3[n] + 4.0 * mu * bc * inv3[n];
            if (n >= 1) v += 4.0 * mu * n * (bc ? inv3[n] : inv3[n - 1]);
            c.diag[bc * 3 + n] = v / 64.0;
        }
    c.cross[0] = 4.0 * lam / 64.0;
    c.cross[1] = 4.0 * lam / 3.0 / 64.0;
    c.cross[2] = 4.0 * mu / 64.0;
    c.cross[3] = 4.0 * mu / 3.0 / 64.0;
    return c;
}

// Element columns per CTA of the full-SM tile shapes, 32 x 16 or 16 x 32 (one CTA fills
// an SM's registers); the 16 x 16 shape takes half of them, so that kernels of other
// streams (the FP32 V-cycle of a concurrent solve) can share the SM.
constexpr int MODAL_THREADS = 512;

// Dynamic shared memory of the modal kernels: two buffers of 12 corner forces per column
// (and, for the FP32 kernel, three layers of element moduli).
template <typename T, int BX, int BY>
constexpr int modal_smem_bytes()
{
    return (int)(sizeof(T) * (2 * 12 + (sizeof(T) == 4 ? 3 : 0)) * BX * BY);
}

// Work items of the modal kernels for a grid of nx x ny x nz elements on `slots`
// concurrent CTAs: x = tile column, y = tile row, [z, w) = node planes. halo = true:
// tiles of (bx-1) x (by-1) output nodes whose bx x by element columns start one column
// and one row below the tile (the FP32 kernel); halo = false: tiles of bx x by element
// columns that do not overlap (apply_modal_kernel). A CTA step costs the busiest of the SM's four sub-partitions (warp w
// runs on w mod 4), counting the warps that hold at least one element column inside
// the grid (a warp issues its FP64 instructions for 32 lanes whatever its active mask):
// far-edge tiles whose whole warps fall outside are cheaper and take longer runs of
// node planes, while a tile cut by the x edge costs as much as a full one. The planes of
// every tile are cut into near-equal runs, and the run lengths are chosen to minimise
// waves x (largest item cost), with (planes + 1) steps per run. *cost receives that
// product. Plain host arithmetic, deterministic.
inline std::vector<int4> modal_plan(int nx, int ny, int nz, int bx, int by, int slots, int forced_planes,
                                    double* cost, bool halo = true)
{
    const int NX = nx + 1, NY = ny + 1, NZ = nz + 1;
    const int tx = halo ? (NX + bx - 2) / (bx - 1) : (nx + bx - 1) / bx;
    const int ty = halo ? (NY + by - 2) / (by - 1) : (ny + by - 1) / by;
    std::vector<long long> v(tx * ty);
    for (int b = 0; b < ty; ++b)
        for (int a = 0; a < tx; ++a) {
            long long per_smsp[4] = {0, 0, 0, 0};
            for (int w = 0; w < bx * by / 32; ++w) {
                bool any = false;
                for (int l = 0; l < 32 && !any; ++l) {
                    const int t = 32 * w + l;
                    const int ex = halo ? a * (bx - 1) - 1 + t % bx : a * bx + t % bx;
                    const int ey = halo ? b * (by - 1) - 1 + t / bx : b * by + t / bx;
                    any = ex >= 0 && ex < nx && ey >= 0 && ey < ny;
                }
                per_smsp[w % 4] += any;
            }
            v[b * tx + a] = 4 * std::max(std::max(per_smsp[0], per_smsp[1]), std::max(per_smsp[2], per_smsp[3]));
        }
    auto runs_for = [&](long long vt, long long cap) -> int {   // planes per run within the cap
        if (forced_planes > 0) return std::min(forced_planes, NZ);
        if (vt <= 0) return NZ;
        return (int)std::max<long long>(1, std::min<long long>(NZ, cap / vt - 1));
    };
    auto count = [&](long long cap, long long* maxcost) {
        long long n = 0, mc = 0;
        for (long long vt : v) {
            const int L = runs_for(vt, cap);
            const int pieces = (NZ + L - 1) / L;
            const int len = (NZ + pieces - 1) / pieces;
            n += pieces;
            mc = std::max(mc, std::max<long long>(vt, 1) * (len + 1));
        }
        *maxcost = mc;
        return n;
    };
    long long best_cap = 0, vmax = 1;
    double best = 1e300;
    for (long long vt : v) vmax = std::max(vmax, vt);
    for (int waves = 1; waves <= 16; ++waves) {
        // smallest cap whose item count fits in `waves` rounds of the slots
        long long lo = 2 * vmax, hi = vmax * (long long)(NZ + 1), mc;
        if (count(hi, &mc) > (long long)waves * slots) continue;
        while (lo < hi) {
            const long long mid = (lo + hi) / 2;
            if (count(mid, &mc) <= (long long)waves * slots) hi = mid;
            else lo = mid + 1;
        }
        const long long n = count(hi, &mc);
        const double t = (double)((n + slots - 1) / slots) * mc;
        if (t < best) {
            best = t;
            best_cap = hi;
        }
        if (forced_planes > 0) break;
    }
    if (best_cap == 0) best_cap = vmax * (long long)(NZ + 1);
    long long mc;
    const long long n = count(best_cap, &mc);
    if (cost) *cost = (double)((n + slots - 1) / slots) * mc;
    std::vector<int4> items;
    for (int b = 0; b < ty; ++b)
        for (int a = 0; a < tx; ++a) {
            const int L = runs_for(v[b * tx + a], best_cap);
            const int pieces = (NZ + L - 1) / L;
            for (int p = 0; p < pieces; ++p) {
                const int z0 = (int)((long long)NZ * p / pieces), z1 = (int)((long long)NZ * (p + 1) / pieces);
                items.push_back(make_int4(a, b, z0, z1));
            }
        }
    return items;
}

// The 9 scaled modal coefficients of every element, E_e C.diag[1..5] then E_e C.cross[0..3],
// as 9 arrays of nel (Es[k * nel + e]): the element's only coupling to its modulus in
// apply_modal_kernel, formed once per floor (the same FP64 products the kernel would form).
__global__ void modal_scale_kernel(const double* __restrict__ E, ModalCoef C, double* __restrict__ Es, long long nel)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nel) return;
    const double s = E[e];
#pragma unroll
    for (int k = 1; k < 6; ++k) Es[(k - 1) * nel + e] = s * C.diag[k];
#pragma unroll
    for (int k = 0; k < 4; ++k) Es[(5 + k) * nel + e] = s * C.cross[k];
}

// 2D sum/difference transform of a face: v[x + 2y] -> f[bx + 2by] = sum s_x^bx s_y^by v.
template <typename T>
__device__ __forceinline__ void face_fwd(const T v[4], T f[4])
{
    const T sx0 = v[1] + v[0], dx0 = v[1] - v[0];
    const T sx1 = v[3] + v[2], dx1 = v[3] - v[2];
    f[0] = sx0 + sx1;
    f[2] = sx1 - sx0;
    f[1] = dx0 + dx1;
    f[3] = dx1 - dx0;
}

// Its transpose: f[bx + 2by] -> v[x + 2y] = sum_beta s_x^bx s_y^by f[beta].
template <typename T>
__device__ __forceinline__ void face_inv(const T f[4], T v[4])
{
    const T lo0 = f[0] - f[2], hi0 = f[0] + f[2];   // bx = 0: y offset 0 / 1
    const T lo1 = f[1] - f[3], hi1 = f[1] + f[3];   // bx = 1
    v[0] = lo0 - lo1;
    v[1] = lo0 + lo1;
    v[2] = hi0 - hi1;
    v[3] = hi0 + hi1;
}

// Side buffer of apply_modal_kernel<BX, BY>: for every node on a tile boundary, the
// corner forces of the four element columns around it, 12 doubles [slot q][component],
// slot q = qx + 2 qy holding corner q of column (ni - qx, nj - qy). Nodes with ni a
// multiple of BX come first ("x lines", (nz + 1) x (nx / BX + 1) x (ny + 1) of them),
// then nodes with nj a multiple of BY ("y lines", (nz + 1) x (ny / BY + 1) x (nx + 1)
// entries; those that also lie on an x line stay unused).
struct ModalSide {
    int bx, by, nxl, nyl;   // tile shape; x lines nx / bx + 1, y lines ny / by + 1
    long long xn;           // entries of the x lines
    __host__ __device__ long long entries(const GridDims& d) const
    {
        return xn + (long long)(d.nz + 1) * nyl * (d.nx + 1);
    }
    __host__ __device__ long long slot_x(const GridDims& d, int ix, int nj, int kz) const
    {
        return ((long long)kz * nxl + ix) * (d.ny + 1) + nj;
    }
    __host__ __device__ long long slot_y(const GridDims& d, int iy, int ni, int kz) const
    {
        return xn + ((long long)kz * nyl + iy) * (d.nx + 1) + ni;
    }
};

__host__ inline ModalSide modal_side(const GridDims& d, int bx, int by)
{
    ModalSide m;
    m.bx = bx;
    m.by = by;
    m.nxl = d.nx / bx + 1;
    m.nyl = d.ny / by + 1;
    m.xn = (long long)(d.nz + 1) * m.nxl * (d.ny + 1);
    return m;
}

// After a step's barrier: the corners of the tile's columns at the nodes on its boundary,
// from shared memory (part[corner * 3 + comp][row][column]) to their side-buffer slots.
// Thread r < 4 BY + 4 (BX - 1) takes one column corner and its three components: columns
// (0, j) corners 0 and 2 and (BX-1, j) corners 1 and 3 (the x lines, tile corners
// included), then row 0's columns i < BX-1 corner 1 and i > 0 corner 0, and row BY-1's
// corners 3 and 2 likewise (the y lines). Columns outside the grid write nothing.
template <typename T, int BX, int BY>
__device__ __forceinline__ void modal_ring_store(const T (*__restrict__ part)[BY][BX], T* __restrict__ side,
                                                 const ModalSide& sd, const GridDims& d, int4 it, int ez, int r)
{
    constexpr int NR = 4 * BY + 4 * (BX - 1);
    if (r >= NR) return;
    int i, j, q;
    if (r < 2 * BY) {
        i = 0, j = r >> 1, q = (r & 1) ? 2 : 0;
    } else if (r < 4 * BY) {
        const int u = r - 2 * BY;
        i = BX - 1, j = u >> 1, q = (u & 1) ? 3 : 1;
    } else {
        const int u = r - 4 * BY;
        const bool top = u >= 2 * (BX - 1);
        const int v = top ? u - 2 * (BX - 1) : u;
        j = top ? BY - 1 : 0;
        if (v < BX - 1) {
            i = v, q = top ? 3 : 1;
        } else {
            i = v - (BX - 1) + 1, q = top ? 2 : 0;
        }
    }
    const int ex = it.x * BX + i, ey = it.y * BY + j;
    if (ex >= d.nx || ey >= d.ny) return;
    const int lx = i + (q & 1), ly = j + (q >> 1);
    const long long sl = (lx == 0 || lx == BX) ? sd.slot_x(d, it.x + (lx == BX ? 1 : 0), ey + (q >> 1), ez)
                                               : sd.slot_y(d, it.y + (ly == BY ? 1 : 0), ex + (q & 1), ez);
#pragma unroll
    for (int c = 0; c < 3; ++c) side[sl * 12 + q * 3 + c] = part[q * 3 + c][j][i];
}

// One CTA per work item: element tile (x, y) of BX x BY columns and node planes [z, w).
// The host balances the items (modal_plan, halo = false): tiles at the far edges of the
// grid hold fewer element columns and take longer runs of planes, so that every CTA costs
// about the same. Writes y at the nodes inside the tile and the side buffer for the
// nodes on its boundary (modal_fixup_kernel completes those).
// MASK: fixed components from d.fix (any supports); otherwise the clamped face x = 0.
template <int BX, int BY, bool MASK = false>
__global__ void __launch_bounds__(BX * BY, MODAL_THREADS / (BX * BY))
apply_modal_kernel(const double* __restrict__ u, double* __restrict__ y, const double* __restrict__ Es,
                   GridDims d, const int4* __restrict__ items, double* __restrict__ side, ModalSide sd_,
                   const int* __restrict__ halt)
{
    if (halt != nullptr && *halt != 0) return;
    // two buffers of corner forces [corner * 3 + comp][column], by step parity (dynamic
    // shared memory, modal_smem_bytes<double, BX, BY>): one barrier per step
    extern __shared__ __align__(16) unsigned char modal_smem[];
    double(*partb)[12][BY][BX] = reinterpret_cast<double(*)[12][BY][BX]>(modal_smem);
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int NX = d.nx + 1, NY = d.ny + 1, NZ = d.nz + 1;
    const int4 it = items[blockIdx.x];
    const int i0 = it.x * BX, j0 = it.y * BY;
    const int k0 = it.z;
    const int k1 = min(NZ, it.w);
    const int ex = i0 + tx, ey = j0 + ty;                 // this thread's element column
    const bool col = ex < d.nx && ey < d.ny;
    const long long plane = (long long)NX * NY;

    // face transform of node plane kz for this column (zero outside the domain; the
    // clamped face x = 0 reads as 0)
    auto load_face = [&](int kz, double f[3][4]) {
        double v[3][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int ni = ex + (q & 1), nj = ey + (q >> 1);
            const long long n = ni + (long long)NX * nj + plane * kz;
            if constexpr (MASK) {
                const bool in = col && kz >= 0 && kz < NZ;
                const unsigned mb = in ? (unsigned)__ldg(d.fix + n) : 7u;
#pragma unroll
                for (int c = 0; c < 3; ++c) v[c][q] = ((mb >> c) & 1u) ? 0.0 : __ldg(u + 3 * n + c);
            } else {
                const bool ok = col && kz >= 0 && kz < NZ && ni >= 1;
#pragma unroll
                for (int c = 0; c < 3; ++c) v[c][q] = ok ? __ldg(u + 3 * n + c) : 0.0;
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) face_fwd<double>(v[c], f[c]);
    };

    double bot[3][4];     // modal face of the current element's bottom node plane
    double carry[3][4];   // modal face forces of the element below at that plane
    load_face(k0 - 1, bot);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q) carry[c][q] = 0.0;

    for (int ez = k0 - 1; ez < k1; ++ez) {
        double top[3][4];
        load_face(ez + 1, top);
        double face[3][4];    // modal forces of node plane ez from this column
        if (col && ez >= 0 && ez < d.nz) {
            // m[c][beta], beta = bx + 2 by + 4 bz: z stage of the sum/difference network
            double m[3][8];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    m[c][q] = top[c][q] + bot[c][q];
                    m[c][q + 4] = top[c][q] - bot[c][q];
                }
            // the element's scaled modal coefficients E_e C (modal_scale_kernel, once per floor)
            const long long e = ex + (long long)d.nx * (ey + (long long)d.ny * ez);
            const long long nel = (long long)d.nx * d.ny * d.nz;
            double sd[6], sc[4];
#pragma unroll
            for (int k = 1; k < 6; ++k) sd[k] = __ldg(Es + (k - 1) * nel + e);
#pragma unroll
            for (int k = 0; k < 4; ++k) sc[k] = __ldg(Es + (5 + k) * nel + e);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double G[8];
#pragma unroll
                for (int beta = 1; beta < 8; ++beta) {
                    const int bc = (beta >> c) & 1;
                    const int n = ((beta >> ((c + 1) % 3)) & 1) + ((beta >> ((c + 2) % 3)) & 1);
                    double t = (bc == 0 && n == 0) ? 0.0 : sd[bc * 3 + n] * m[c][beta];
#pragma unroll
                    for (int dd = 1; dd < 3; ++dd) {
                        const int dc = (c + dd) % 3;
                        const int o = 3 - c - dc;
                        const int bd = (beta >> dc) & 1;
                        if (bc != bd) {
                            const int alpha = beta ^ (1 << c) ^ (1 << dc);
                            const int k = (bc ? 0 : 2) + ((beta >> o) & 1);
                            t = fma(sc[k], m[dc][alpha], t);
                        }
                    }
                    G[beta] = t;
                }
                // z stage of the transposed network: bottom face G0 - G1, top face G0 + G1
                // (the constant mode beta = 0 carries no force: a rigid translation)
                face[c][0] = carry[c][0] - G[4];
                carry[c][0] = G[4];
#pragma unroll
                for (int q = 1; q < 4; ++q) {
                    face[c][q] = carry[c][q] + (G[q] - G[q + 4]);
                    carry[c][q] = G[q] + G[q + 4];
                }
            }
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    face[c][q] = carry[c][q];
                    carry[c][q] = 0.0;
                }
        }
        // node plane ez: this column's four corner forces, then the gather (the buffer of
        // this parity was last read by the gather two steps back, which every thread
        // finished before the previous step's barrier)
        double(*part)[BY][BX] = partb[(ez - k0 + 1) & 1];
        const bool out = ez >= k0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double v[4];
            face_inv<double>(face[c], v);
#pragma unroll
            for (int q = 0; q < 4; ++q) part[q * 3 + c][ty][tx] = v[q];
        }
        __syncthreads();
        if (out) modal_ring_store<double, BX, BY>(part, side, sd_, d, it, ez, tx + BX * ty);
        const int ni = i0 + tx + 1, nj = j0 + ty + 1;   // the node inside the tile at this column's corner 3
        if (out && tx < BX - 1 && ty < BY - 1 && ni < NX && nj < NY) {
            const long long n = ni + (long long)NX * nj + plane * ez;
            const unsigned ob = MASK ? (unsigned)__ldg(d.fix + n) : (ni == 0 ? 7u : 0u);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                // node (ni, nj) is corner 3 (1,1) of column (tx, ty), 2 (0,1) of (tx+1, ty),
                // 1 (1,0) of (tx, ty+1) and 0 (0,0) of (tx+1, ty+1)
                double acc = part[3 * 3 + c][ty][tx] + part[2 * 3 + c][ty][tx + 1];
                acc += part[1 * 3 + c][ty + 1][tx];
                acc += part[0 * 3 + c][ty + 1][tx + 1];
                y[3 * n + c] = ((ob >> c) & 1u) ? 0.0 : acc;
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int q = 0; q < 4; ++q) bot[c][q] = top[c][q];
    }
}

// The nodes on tile boundaries: the four corner forces from the side buffer, added in the
// order of the gather inside a tile (columns outside the grid read as zero there too), so
// every node of K*u has the same arithmetic wherever the tiles fall. One thread per
// side-buffer entry.
template <bool MASK = false>
__global__ void modal_fixup_kernel(const double* __restrict__ side, ModalSide sd_, double* __restrict__ y,
                                   GridDims d, const int* __restrict__ halt)
{
    if (halt != nullptr && *halt != 0) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int NX = d.nx + 1, NY = d.ny + 1;
    if (t >= sd_.entries(d)) return;
    int ni, nj, kz;
    if (t < sd_.xn) {
        nj = (int)(t % NY);
        const long long r = t / NY;
        ni = (int)(r % sd_.nxl) * sd_.bx;
        kz = (int)(r / sd_.nxl);
    } else {
        const long long u = t - sd_.xn;
        ni = (int)(u % NX);
        const long long r = u / NX;
        nj = (int)(r % sd_.nyl) * sd_.by;
        kz = (int)(r / sd_.nyl);
        if (ni % sd_.bx == 0) return;   // on an x line: its entry is there
    }
    if (ni >= NX || nj >= NY) return;
    const long long n = ni + (long long)NX * nj + (long long)NX * NY * kz;
    const unsigned ob = MASK ? (unsigned)__ldg(d.fix + n) : (ni == 0 ? 7u : 0u);
    bool in[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int ex = ni - (q & 1), ey = nj - (q >> 1);
        in[q] = ex >= 0 && ex < d.nx && ey >= 0 && ey < d.ny;
    }
    const double* s = side + t * 12;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double p3 = in[3] ? s[9 + c] : 0.0, p2 = in[2] ? s[6 + c] : 0.0;
        const double p1 = in[1] ? s[3 + c] : 0.0, p0 = in[0] ? s[c] : 0.0;
        double acc = p3 + p2;
        acc += p1;
        acc += p0;
        y[3 * n + c] = ((ob >> c) & 1u) ? 0.0 : acc;
    }
}

// ---- the FP32 V-cycle's fine-level operator in the same basis ------------------------
// A pair of FP32 values, the x and y components of one quantity, added and subtracted by
// the packed f32x2 instructions: each lane rounds to nearest like the scalar instruction,
// so the pair gives bit for bit the scalar results at half the instructions.
struct f32x2 {
    float x, y;
};
__device__ __forceinline__ f32x2 operator+(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("{\n .reg .b64 ra, rb, rc;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " add.rn.f32x2 rc, ra, rb;\n mov.b64 {%0, %1}, rc;\n}\n"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ f32x2 operator-(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("{\n .reg .b64 ra, rb, rc;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " sub.rn.f32x2 rc, ra, rb;\n mov.b64 {%0, %1}, rc;\n}\n"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

// The level-0 smoothing sweeps and residual of the mixed V-cycle (and the FP32 K*u) with
// the modal K0 in FP32: the column walk of apply_modal_kernel (on tiles that overlap by one
// element column, modal_plan with halo = true, so no side buffer), with the next
// node plane's values and element modulus loaded one step ahead, and at the gather each
// node also sums its 3x3 diagonal block from the moduli of its eight elements (kept in
// shared memory for the current and the previous element layer) for the damped
// node-block Jacobi update:
//   MODE ST_APPLY: out = K x;  ST_RESID: out = b - K x;  ST_SWEEP: out = x + omega D_n^-1 (b - K x).
// Fixed nodes (the clamped face x = 0) read as 0 and are written as 0. FP32 arithmetic
// (the V-cycle's precision); K*u rounds differently from the node stencil, within FP32.
struct ModalCoefF {
    float diag[6], cross[4];
    float blk[8][6];   // the 3x3 diagonal block of K0 at local node a: d00 d11 d22 d01 d02 d12
};

template <int MODE, typename BT, typename OT, int BX, int BY>
__global__ void __launch_bounds__(BX * BY, MODAL_THREADS / (BX * BY))
modal_stencil_f32_kernel(const float* __restrict__ x, const BT* __restrict__ b, OT* __restrict__ out,
                         const float* __restrict__ E, GridDims d, const __grid_constant__ ModalCoefF C,
                         float omega, const int4* __restrict__ items, const int* __restrict__ halt)
{
    if (halt != nullptr && *halt != 0) return;
    // corner forces [corner][column] in two buffers by step parity, the x and y components
    // as pairs (partb) and z apart (partz), and the column's element moduli in three by
    // layer (the gather reads this layer's and the previous one's): dynamic shared memory,
    // modal_smem_bytes<float, BX, BY>; one barrier per step. The x and y components run
    // through the transforms, the face recurrence and the gather as f32x2 pairs; the
    // modal-space products, whose index pattern differs by component, stay scalar.
    extern __shared__ __align__(16) unsigned char modal_smem[];
    f32x2(*partb)[4][BY][BX] = reinterpret_cast<f32x2(*)[4][BY][BX]>(modal_smem);
    float(*partz)[4][BY][BX] = reinterpret_cast<float(*)[4][BY][BX]>(modal_smem + sizeof(float) * 2 * 8 * BY * BX);
    float(*Es)[BY][BX] = reinterpret_cast<float(*)[BY][BX]>(modal_smem + sizeof(float) * 2 * 12 * BY * BX);
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int NX = d.nx + 1, NY = d.ny + 1, NZ = d.nz + 1;
    const int4 it = items[blockIdx.x];
    const int i0 = it.x * (BX - 1), j0 = it.y * (BY - 1);
    const int k0 = it.z;
    const int k1 = min(NZ, it.w);
    const int ex = i0 - 1 + tx, ey = j0 - 1 + ty;
    const bool col = ex >= 0 && ex < d.nx && ey >= 0 && ey < d.ny;
    const long long plane = (long long)NX * NY;
    const int ni = i0 + tx, nj = j0 + ty;   // this thread's output node column
    const bool outnode = tx < BX - 1 && ty < BY - 1 && ni < NX && nj < NY;

    auto load_raw = [&](int kz, f32x2 v[4], float vz[4]) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int qi = ex + (q & 1), qj = ey + (q >> 1);
            const bool ok = col && kz >= 0 && kz < NZ && qi >= 1;
            const long long n = qi + (long long)NX * qj + plane * kz;
            v[q].x = ok ? __ldg(x + 3 * n + 0) : 0.f;
            v[q].y = ok ? __ldg(x + 3 * n + 1) : 0.f;
            vz[q] = ok ? __ldg(x + 3 * n + 2) : 0.f;
        }
    };
    auto load_E = [&](int kz) -> float {
        return (col && kz >= 0 && kz < d.nz) ? __ldg(E + ex + (long long)d.nx * (ey + (long long)d.ny * kz)) : 0.f;
    };

    f32x2 bot[4], carry[4], raw[4];         // x and y components
    float botz[4], carryz[4], rawz[4];      // z
    load_raw(k0 - 1, raw, rawz);
    face_fwd<f32x2>(raw, bot);
    face_fwd<float>(rawz, botz);
    load_raw(k0, raw, rawz);                // the next top face, untransformed
    float Ecur = load_E(k0 - 1);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        carry[q] = f32x2{0.f, 0.f};
        carryz[q] = 0.f;
    }

    for (int ez = k0 - 1; ez < k1; ++ez) {
        // loads one step ahead: the plane after next, the next element's modulus, and this
        // step's node values for the update
        f32x2 rawn[4];
        float rawnz[4];
        load_raw(ez + 2, rawn, rawnz);
        const float Enext = load_E(ez + 1);
        float xn[3] = {0.f, 0.f, 0.f}, bn[3] = {0.f, 0.f, 0.f};
        long long nn = 0;
        if (ez >= k0 && outnode) {
            nn = ni + (long long)NX * nj + plane * ez;
            if (MODE != ST_APPLY) {
#pragma unroll
                for (int c = 0; c < 3; ++c) bn[c] = convert<float>(b[3 * nn + c]);
            }
            if (MODE == ST_SWEEP) {
#pragma unroll
                for (int c = 0; c < 3; ++c) xn[c] = x[3 * nn + c];
            }
        }
        f32x2 top[4];
        float topz[4];
        face_fwd<f32x2>(raw, top);
        face_fwd<float>(rawz, topz);
        f32x2 face[4];
        float facez[4];
        if (col && ez >= 0 && ez < d.nz) {
            f32x2 m[8];   // modes of the x and y components
            float mz[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                m[q] = top[q] + bot[q];
                m[q + 4] = top[q] - bot[q];
                mz[q] = topz[q] + botz[q];
                mz[q + 4] = topz[q] - botz[q];
            }
            // component dc's mode beta
            auto mode = [&](int dc, int beta) -> float { return dc == 0 ? m[beta].x : dc == 1 ? m[beta].y : mz[beta]; };
            const float s = Ecur;
            float sd[6], sc[4];
#pragma unroll
            for (int k = 1; k < 6; ++k) sd[k] = s * C.diag[k];
#pragma unroll
            for (int k = 0; k < 4; ++k) sc[k] = s * C.cross[k];
            f32x2 G[8];
            float Gz[8];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
#pragma unroll
                for (int beta = 1; beta < 8; ++beta) {   // beta = 0 (a rigid translation) carries no force
                    const int bc = (beta >> c) & 1;
                    const int n = ((beta >> ((c + 1) % 3)) & 1) + ((beta >> ((c + 2) % 3)) & 1);
                    float t = (bc == 0 && n == 0) ? 0.f : sd[bc * 3 + n] * mode(c, beta);
#pragma unroll
                    for (int dd = 1; dd < 3; ++dd) {
                        const int dc = (c + dd) % 3;
                        const int o = 3 - c - dc;
                        const int bdd = (beta >> dc) & 1;
                        if (bc != bdd) {
                            const int alpha = beta ^ (1 << c) ^ (1 << dc);
                            const int k = (bc ? 0 : 2) + ((beta >> o) & 1);
                            t = fmaf(sc[k], mode(dc, alpha), t);
                        }
                    }
                    if (c == 0) G[beta].x = t;
                    else if (c == 1) G[beta].y = t;
                    else Gz[beta] = t;
                }
            }
            face[0] = carry[0] - G[4];
            carry[0] = G[4];
            facez[0] = carryz[0] - Gz[4];
            carryz[0] = Gz[4];
#pragma unroll
            for (int q = 1; q < 4; ++q) {
                face[q] = carry[q] + (G[q] - G[q + 4]);
                carry[q] = G[q] + G[q + 4];
                facez[q] = carryz[q] + (Gz[q] - Gz[q + 4]);
                carryz[q] = Gz[q] + Gz[q + 4];
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                face[q] = carry[q];
                carry[q] = f32x2{0.f, 0.f};
                facez[q] = carryz[q];
                carryz[q] = 0.f;
            }
        }
        // buffers of this step: part by parity, Es by step mod 3 (last read by the gathers
        // three and two steps back, finished before the previous step's barrier)
        const int step = ez - k0 + 1;
        const int cur = step % 3, prv = (step + 2) % 3;
        f32x2(*part)[BY][BX] = partb[step & 1];
        float(*pz)[BY][BX] = partz[step & 1];
        {
            f32x2 v[4];
            float vz[4];
            face_inv<f32x2>(face, v);
            face_inv<float>(facez, vz);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                part[q][ty][tx] = v[q];
                pz[q][ty][tx] = vz[q];
            }
        }
        Es[cur][ty][tx] = Ecur;
        __syncthreads();
        if (ez >= k0 && outnode) {
            f32x2 axy = part[3][ty][tx] + part[2][ty][tx + 1];
            axy = axy + part[1][ty + 1][tx];
            axy = axy + part[0][ty + 1][tx + 1];
            float az = pz[3][ty][tx] + pz[2][ty][tx + 1];
            az += pz[1][ty + 1][tx];
            az += pz[0][ty + 1][tx + 1];
            const float a[3] = {axy.x, axy.y, az};
            if (ni == 0) {
                out[3 * nn + 0] = OT(0);
                out[3 * nn + 1] = OT(0);
                out[3 * nn + 2] = OT(0);
            } else if (MODE == ST_APPLY) {
#pragma unroll
                for (int c = 0; c < 3; ++c) out[3 * nn + c] = convert<OT>(a[c]);
            } else if (MODE == ST_RESID) {
#pragma unroll
                for (int c = 0; c < 3; ++c) out[3 * nn + c] = convert<OT>(bn[c] - a[c]);
            } else {
                // the node's 3x3 diagonal block from its eight elements (previous layer: the
                // node at local z offset 1; current layer: offset 0), in a fixed order
                float db[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int lz = 0; lz < 2; ++lz) {
                    const int layer = lz == 0 ? prv : cur;   // ez - 1, then ez
                    const int oz = lz == 0 ? 1 : 0;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int cx = q & 1, cy = q >> 1;            // column (tx + cx, ty + cy)
                        const float Ee = Es[layer][ty + cy][tx + cx];
                        const int la = local_index(1 - cx, 1 - cy, oz);
#pragma unroll
                        for (int k = 0; k < 6; ++k) db[k] = fmaf(Ee, C.blk[la][k], db[k]);
                    }
                }
                const float r0 = bn[0] - a[0], r1 = bn[1] - a[1], r2 = bn[2] - a[2];
                node_block_update<float, OT>(db[0], db[1], db[2], db[3], db[4], db[5], r0, r1, r2, xn, out + 3 * nn,
                                             omega);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            bot[q] = top[q];
            raw[q] = rawn[q];
            botz[q] = topz[q];
            rawz[q] = rawnz[q];
        }
        Ecur = Enext;
    }
}

}  // namespace gf
