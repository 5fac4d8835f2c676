// C ABI of the guarded floor-selection state solver (see include/gf.h).
//
// Host side: the grid handle, hierarchy set-up, the V-cycle schedule, the FGMRES
// driver (device-resident Arnoldi/Givens state, host polls a mapped stop flag with
// at most two steps in flight) and Algorithm 1 of arXiv 2607.26382.
#include "../../include/gf.h"
#include "stencil.cuh"
#include "krylov.cuh"
#include "ddgs.cuh"
#include "oc.cuh"
#include "split.cuh"
#include "split_tc.cuh"
#include "stencil_tc.cuh"
#include "cheb.cuh"
#include "vcycle_cluster.cuh"
#include "lanczos.cuh"
#include "linesearch.cuh"
#include "finecorr.cuh"
#include "galerkin.cuh"
#include "coarse_krylov.cuh"
#include "modal.cuh"
#include "ldl.cuh"

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cfloat>
#include <cstring>
#include <cstdlib>
#include <string>
#include <vector>
#include <algorithm>
#include <utility>
#include <mutex>
#include <functional>
#include <thread>

namespace {

thread_local std::string g_err;

int set_err(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return set_err(e_ == cudaErrorMemoryAllocation ? GF_ERR_OOM : GF_ERR_CUDA,  \
                           std::string(#call) + ": " + cudaGetErrorString(e_));        \
    } while (0)

#define RET(call)                      \
    do {                               \
        int r_ = (call);               \
        if (r_ != GF_OK) return r_;    \
    } while (0)

inline unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

struct Level {
    int nx, ny, nz;
    double h;
    long long nodes, ndof, nel;
    double* E64 = nullptr;
    float* E32 = nullptr;
    double *b64 = nullptr, *x64 = nullptr, *t64 = nullptr, *r64 = nullptr;
    float *b32 = nullptr, *x32 = nullptr, *t32 = nullptr, *r32 = nullptr;
    double* q64 = nullptr;            // line-searched coarse correction: K c (allocated on first use)
    float* q32 = nullptr;
    double* Ke64 = nullptr;           // Galerkin levels (l >= 1): 24x24 element matrices, FP64 moduli
    float* Ke32 = nullptr;            //   and from the BF16-density moduli, rounded to FP32
    uint8_t* fix = nullptr;           // per-node fixed components (bridge supports); null: clamped face x = 0
    gf::GridDims dims() const { return gf::GridDims{nx, ny, nz, fix}; }
};

// Element stiffness of the unit cube (E = 1 scaled by E0 by the caller) from the
// exact 1D integrals of linear hats: S_ab[i,j] = int d_a N_i d_b N_j factorises
// into m = int phi phi, k = int phi' phi', c = int phi' phi per axis, and
// K[3i+al][3j+be] = lam S_{al be} + mu S_{be al} + mu delta_{al be} sum_g S_gg.
void build_k0(double E0, double nu, double* K)
{
    const double lam = E0 * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    const double mu = E0 / (2.0 * (1.0 + nu));
    const double m1[2][2] = {{2.0 / 6.0, 1.0 / 6.0}, {1.0 / 6.0, 2.0 / 6.0}};
    const double k1[2][2] = {{1.0, -1.0}, {-1.0, 1.0}};
    const double c1[2][2] = {{-0.5, -0.5}, {0.5, 0.5}};
    int off[8][3];
    for (int z = 0; z < 2; ++z)
        for (int y = 0; y < 2; ++y)
            for (int x = 0; x < 2; ++x) {
                const int a = gf::local_index(x, y, z);
                off[a][0] = x;
                off[a][1] = y;
                off[a][2] = z;
            }
    auto S = [&](int a, int b, int i, int j) {
        double v = 1.0;
        for (int d = 0; d < 3; ++d) {
            const int p = off[i][d], q = off[j][d];
            if (d == a && d == b) v *= k1[p][q];
            else if (d == a) v *= c1[p][q];
            else if (d == b) v *= c1[q][p];
            else v *= m1[p][q];
        }
        return v;
    };
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j)
            for (int al = 0; al < 3; ++al)
                for (int be = 0; be < 3; ++be) {
                    double v = lam * S(al, be, i, j) + mu * S(be, al, i, j);
                    if (al == be) v += mu * (S(0, 0, i, j) + S(1, 1, i, j) + S(2, 2, i, j));
                    K[(3 * i + al) * 24 + 3 * j + be] = v;
                }
}

}  // namespace

namespace {
int mlp_predict_host(gf_mlp* M, const double* feat, int n, int* cls);
int mlp_first_floors(gf_mlp* M, const double* feat, int n, double c, int nf, int* first);
}

struct gf_grid {
    int nx, ny, nz, L;
    double h, E0, nu;
    cudaStream_t stream;
    int device, sms;
    long long nodes, ndof, nel;
    std::vector<Level> lv;
    gf::K0Param<double> K0d;
    gf::ModalCoef Kmodal;             // K0 in the sum/difference basis (apply_modal_kernel)
    gf::ModalCoefF Kmodal32;          // the same in FP32 with K0's node blocks (modal_stencil_f32_kernel)
    bool modal_f32 = true;            // level-0 FP32 stencils in the modal basis (GF_MODAL_F32=0: node stencils)
    int4* modal_items = nullptr;      // work items of the modal FP32 fine level (tiles overlapping by one column)
    int modal_n = 0, modal_bx = 32, modal_by = 16;   // item count; CTA tile 32 x 16, 16 x 32 or 16 x 16 columns
    int4* modal64_items = nullptr;    // work items of the modal FP64 K*u (device; null: dense stencil)
    int modal64_n = 0, modal64_bx = 32, modal64_by = 16;
    bool half_sm = false;             // gf_set_sm_share: launch shapes that leave half of each SM free
    double* modal_side = nullptr;     // its side buffer: corner forces at the nodes on tile boundaries
    double* modal_es = nullptr;       // its elements' scaled coefficients E_e C, 9 x nel (modal_scale_kernel)
    bool coarse_ldl = true;           // coarsest inverse from the banded LDL^T factorisation (GF_COARSE_LDL=0: a sweep)
    bool sym_gj = true;               // else the blocked symmetric sweep (GF_SYM_GJ=0: the two-pivot form)
    double* ldl_ws = nullptr;         // its workspace: 1 / d (nc), X of the band rows (nc x LDL_C), Q (LDL_C^2)
    int geom = GF_GEOM_CANTILEVER;    // supports: the clamped face x = 0, or the bridge's (gf_set_geometry)
    gf::K0Param<float> K0f;
    gf::K0Pair K0p;                   // K0f with rows 3a, 3a+1 paired (node_stencil_f32x2_kernel)
    bool f32x2 = true;                // FP32 node stencil with paired FMAs (GF_F32X2=0: scalar FMAs)
    int ctpb = 128;                   // block size for levels too small to fill the SMs (0: as level 0)
    bool ck_fused = true;             // coarse-level Krylov solve in one CTA (GF_COARSE_FUSED=0: multi-launch)
    int coarse_kind = GF_COARSE_REDISCRETISED;   // gf_set_coarse_operator; applied by gf_set_floor
    double* galG = nullptr;           // G_c = T_c^T K0 T_c, 8 x 576 (Galerkin first coarse level)
    double* gal_s[2] = {nullptr, nullptr};   // FP64 scratch for the BF16-moduli chain
    gf::S3BFrag* B3 = nullptr;        // B fragments of M (K0 = s M) for stencil_tc32_kernel, device
    int stc_cz[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // > 0: level l's FP32 stencils on the tensor cores, cz layers per CTA
    double* rho64 = nullptr;
    __nv_bfloat16* rho16 = nullptr;
    double p = 3.0;
    bool has_density = false, has_floor = false;
    double rho_min = 0.0;
    double* Ainv = nullptr;
    int nc = 0;
    double* Agj = nullptr;            // second buffer of the double-buffered Gauss-Jordan
    int* cpos = nullptr;              // coarsest level: position of each DOF among the free ones (-1: fixed)
    int* cidx = nullptr;              // coarsest level: the free DOFs in order; ncf of them (+1 word: the count)
    int ncf = 0;
    int cband = 0;                    // coarsest level: bound on |p - q| over the operator's non-zeros (free DOFs)
    int* dflag = nullptr;
    // Krylov workspace
    int m_alloc = 0;
    long long ldk = 0;                // leading dimension of V, Z, Vd: ndof rounded up to 32 (256-byte rows)
    double *V = nullptr, *Z = nullptr, *partial = nullptr, *work = nullptr;
    int nbc[3][4] = {};               // grid of the FP64 Gram-Schmidt passes (dots, update+dots, update+norm) x NV 8/16/24/32
    double* ckx = nullptr;            // iterate of a probe true-residual check
    // fine-level adaptive correction: inner basis V (steps + 1), Z (steps), r, d, q, z in the
    // V-cycle's precision (fc_es bytes per entry), the inner solver's state and partial sums
    void *fcV = nullptr, *fcZ = nullptr, *fcR = nullptr, *fcD = nullptr, *fcQ = nullptr, *fcZT = nullptr;
    gf::FcState* fc = nullptr;
    double* fc_partial = nullptr;
    int fc_steps = 0, fc_es = 0, fc_nb = 0;
    int gkey_fine = -1;               // fine_steps the captured Arnoldi steps were built with
    int gkey_coarse = -1;             // coarse_steps the captured Arnoldi steps were built with
    int coarse_steps = 0;             // coarse-level inner FGMRES steps of the current solve (0: exact)
    double* ls_partial = nullptr;     // line search: per-block dot products
    double* ls_alpha = nullptr;       // line search: alpha of each level (device)
    int ls_nb = 0;
    double gkey_ls = -1.0;            // line-search ratio the captured Arnoldi steps were built with
    gf::LzState* lz = nullptr;        // conditioning diagnostic: Lanczos coefficients
    double* lzv = nullptr;            // its three vectors
    float2* Vd = nullptr;             // double-float copy of the basis (outer == 2)
    float2* pdd = nullptr;            // per-block partial pairs of the double-float passes
    unsigned int* ddticket = nullptr; // arrival counter of their last-block finish
    unsigned int* cgsticket = nullptr;   // the same for the FP64 Gram-Schmidt passes
    int md_alloc = 0, nbd = 0;        // nbd: largest grid of the double-float passes (partials rows)
    int nbd_k[3][3] = {};             // grid per pass (dots, update+dots, update+norm) and NV (8, 16, 32)
    gf::KState* st = nullptr;
    gf::KState* gst = nullptr;   // guard scratch
    double* hist = nullptr;
    int hist_cap = 0;
    int* host_status = nullptr;       // mapped pinned
    int* host_status_dev = nullptr;
    int nbr = 0;                      // blocks for reductions
    cudaEvent_t ev[3];
    gf_stats stats{};
    // CUDA graphs of the Arnoldi steps (one per j), captured on cap_stream
    cudaStream_t cur_stream = nullptr;   // where launch() enqueues (cap_stream while capturing)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t step_exec[gf::KRY_MMAX] = {};
    long long step_nodes[gf::KRY_MMAX] = {};
    int gkey_prec = -1, gkey_nu1 = -1, gkey_nu2 = -1;
    double gkey_omega = -1.0;
    bool use_graphs = true;
    int tpb[2] = {256, 256};          // node-stencil block size: [0] FP64, [1] FP32 (0 = smem-tiled kernel)
    bool skip_coarse_inverse = false; // batched set-up builds the coarsest inverse itself
    double dstat[3] = {0.0, 0.0, 0.0}; // fraction of rho_hat == 0, mean, std (at set_density)
    int vc_l0 = -1;                   // first level run by the cluster V-cycle kernel (-1: none)
    // split-integer operator: K0 = s_split * M with integer M (when it exists)
    bool has_split = false;
    double s_split = 0.0;
    gf::MParam Msplit;
    float2* Edf = nullptr;            // s_split * E_e (fine level) as float pairs
    gf::TcBFrag* Btc = nullptr;       // M as per-lane fp16 MMA B fragments (tensor-core split), device
    bool split_tc = true;             // element products on the tensor cores (see gf_create_grid)
    int gkey_outer = -1, gkey_smoother = -1;
    // Chebyshev smoothing: per precision (0 FP64, 1 FP32) and level, lambda_max and the
    // step coefficients {c1, c2}[CHEB_MAXDEG] on the device; valid until the next floor
    double* cheb = nullptr;           // [2][L][1 + 2*CHEB_MAXDEG] (lambda, then coefficients)
    double* cheb_ss = nullptr;        // power-method scratch scalar
    bool cheb_ready[2] = {false, false};
    // optimisation-loop scratch (allocated on first use)
    double *oc_rho = nullptr, *oc_dc = nullptr, *oc_dcx = nullptr, *oc_dvx = nullptr, *oc_ones = nullptr;
    gf::OCState* oc_st = nullptr;
};

namespace {
// Launch a kernel on the grid's stream, count it, and report launch errors.
template <typename... KArgs, typename... Args>
int launch_smem(gf_grid* g, dim3 grid, dim3 block, size_t smem, void (*kern)(KArgs...), Args... args)
{
    kern<<<grid, block, smem, g->cur_stream>>>(static_cast<KArgs>(args)...);
    g->stats.kernel_launches++;
    CK(cudaGetLastError());
    return GF_OK;
}

template <typename... KArgs, typename... Args>
int launch(gf_grid* g, dim3 grid, dim3 block, void (*kern)(KArgs...), Args... args)
{
    return launch_smem(g, grid, block, 0, kern, args...);
}
}  // namespace

#define LAUNCH(g, grid, block, kern, ...) RET(launch((g), dim3(grid), dim3(block), kern, __VA_ARGS__))
#define LAUNCH_SMEM(g, grid, block, smem, kern, ...) \
    RET(launch_smem((g), dim3(grid), dim3(block), (smem), kern, __VA_ARGS__))

namespace {

// Block size for a launch over `nodes` nodes: levels with fewer than two 256-thread
// blocks per SM take ctpb-thread blocks, so that every SM gets work (the results do not
// depend on the block size: one node per thread).
// Blocks of 256 threads for an elementwise pass over n entries: about four entries per
// thread (their loads in flight together), at least two blocks per SM.
int stream_blocks(const gf_grid* g, long long n)
{
    return (int)std::max<long long>(2LL * g->sms, (n + 1023) / 1024);
}

// Opt a kernel in to `bytes` of dynamic shared memory (above the default 48 KB), once.
template <auto KERN>
bool smem_opt_in(int bytes)
{
    static const bool ok =
        cudaFuncSetAttribute((const void*)KERN, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
    return ok;
}

// A modal kernel (modal.cuh) over n_items work items, with its dynamic shared memory.
template <typename T, int BX, int BY, auto KERN, typename... Args>
int launch_modal(gf_grid* g, int n_items, Args... args)
{
    constexpr int bytes = gf::modal_smem_bytes<T, BX, BY>();
    if (!smem_opt_in<KERN>(bytes)) return set_err(GF_ERR_CUDA, "shared memory of the modal kernel");
    return launch_smem(g, dim3(n_items), dim3(BX, BY), bytes, KERN, args...);
}

int level_tpb(const gf_grid* g, long long nodes, int base)
{
    return (g->ctpb > 0 && nodes < 512LL * g->sms) ? g->ctpb : base;
}

// grid and block of a node-per-thread launch over `nodes` nodes (256 threads, or ctpb)
dim3 lv_grid(const gf_grid* g, long long nodes) { return dim3(nblk(nodes, level_tpb(g, nodes, 256))); }
dim3 lv_block(const gf_grid* g, long long nodes) { return dim3(level_tpb(g, nodes, 256)); }

int check_grid(const gf_grid* g)
{
    if (!g) return set_err(GF_ERR_ARG, "null grid");
    return GF_OK;
}

int set_device(const gf_grid* g)
{
    CK(cudaSetDevice(g->device));
    return GF_OK;
}

// ------------------------------------------------------------------ stencils --
// FP32 shared-memory-tiled stencil on level l; b may be FP64 (level 0) and the
// output FP64 (the V-cycle's last sweep writes the FP64 result directly).
template <int MODE, typename BT, typename OT>
int tiled_f32(gf_grid* g, int l, const float* x, const BT* b, OT* out, const float* E, float omega, const int* halt)
{
    const Level& L = g->lv[l];
    if (g->stc_cz[l] > 0) {   // element products on the tensor cores (3xTF32)
        const int cz = g->stc_cz[l];
        const dim3 grid((L.nx + 1 + gf::S3_NX - 1) / gf::S3_NX, (L.ny + 1 + gf::S3_NY - 1) / gf::S3_NY,
                        (L.nz + 1 + cz - 1) / cz);
        LAUNCH_SMEM(g, grid, gf::S3_THREADS, sizeof(gf::S3Smem), (gf::stencil_tc32_kernel<MODE, BT, OT>), x, b, out,
                    E, L.dims(), g->Msplit, (const gf::S3BFrag*)g->B3, (float)g->s_split, omega, cz, halt);
        return GF_OK;
    }
    if (l == 0 && g->modal_f32 && g->modal_items && !L.fix && g->tpb[1] > 0) {   // the modal FP32 fine level
        if (g->modal_bx == 32)
            RET((launch_modal<float, 32, 16, gf::modal_stencil_f32_kernel<MODE, BT, OT, 32, 16>>(
                g, g->modal_n, x, b, out, E, L.dims(), g->Kmodal32, omega, (const int4*)g->modal_items, halt)));
        else if (g->modal_by == 32)
            RET((launch_modal<float, 16, 32, gf::modal_stencil_f32_kernel<MODE, BT, OT, 16, 32>>(
                g, g->modal_n, x, b, out, E, L.dims(), g->Kmodal32, omega, (const int4*)g->modal_items, halt)));
        else
            RET((launch_modal<float, 16, 16, gf::modal_stencil_f32_kernel<MODE, BT, OT, 16, 16>>(
                g, g->modal_n, x, b, out, E, L.dims(), g->Kmodal32, omega, (const int4*)g->modal_items, halt)));
        return GF_OK;
    }
    if (g->tpb[1] > 0 && g->f32x2) {   // the same, with paired FMAs
        const int tpb = level_tpb(g, L.nodes, g->tpb[1]);
        if (L.fix)   // supports other than the clamped face (bridge): per-node fixed components
            LAUNCH(g, nblk(L.nodes, tpb), tpb, (gf::node_stencil_f32x2_kernel<MODE, BT, OT, true>), x, b, out, E,
                   L.dims(), g->K0p, omega, halt);
        else
            LAUNCH(g, nblk(L.nodes, tpb), tpb, (gf::node_stencil_f32x2_kernel<MODE, BT, OT>), x, b, out, E, L.dims(),
                   g->K0p, omega, halt);
        return GF_OK;
    }
    if (g->tpb[1] > 0) {   // linear node-per-thread kernel with the autotuned block size
        const int tpb = level_tpb(g, L.nodes, g->tpb[1]);
        if (L.fix)
            LAUNCH(g, nblk(L.nodes, tpb), tpb, (gf::node_stencil_kernel<float, float, MODE, BT, OT, true>), x, b, out,
                   E, L.dims(), g->K0f, omega, halt);
        else
            LAUNCH(g, nblk(L.nodes, tpb), tpb, (gf::node_stencil_kernel<float, float, MODE, BT, OT>), x, b, out, E,
                   L.dims(), g->K0f, omega, halt);
        return GF_OK;
    }
    if (g->tpb[1] < 0) {   // 27-neighbour register-gather kernel
        const int tpb = -g->tpb[1];
        LAUNCH(g, nblk(L.nodes, tpb), tpb, (gf::node_stencil27_kernel<float, MODE, BT, OT>), x, b, out, E,
               L.dims(), g->K0f, omega, halt);
        return GF_OK;
    }
    const dim3 grid((L.nx + 1 + gf::TSX - 1) / gf::TSX, (L.ny + 1 + gf::TSY - 1) / gf::TSY,
                    (L.nz + 1 + gf::TSZ - 1) / gf::TSZ);
    LAUNCH(g, grid, dim3(gf::TSX, gf::TSY, gf::TSZ), (gf::tiled_stencil_f32_kernel<MODE, BT, OT>), x, b, out, E,
           L.dims(), g->K0f, omega, halt);
    return GF_OK;
}

template <typename T, typename ET, int MODE>
int stencil(gf_grid* g, int l, const T* x, const T* b, T* out, const ET* E, const gf::K0Param<T>& K0,
            T omega, const int* halt)
{
    const Level& L = g->lv[l];
    if constexpr (sizeof(T) == sizeof(float)) return tiled_f32<MODE, float, float>(g, l, x, b, out, E, omega, halt);
    const int tpb = g->tpb[sizeof(T) == sizeof(double) ? 0 : 1];
    if (L.fix)
        LAUNCH(g, nblk(L.nodes, tpb), tpb, (gf::node_stencil_kernel<T, ET, MODE, T, T, true>), x, b, out, E, L.dims(),
               K0, omega, halt);
    else
        LAUNCH(g, nblk(L.nodes, tpb), tpb, (gf::node_stencil_kernel<T, ET, MODE>), x, b, out, E, L.dims(), K0, omega,
               halt);
    return GF_OK;
}

template <typename T>
const gf::K0Param<T>& k0(const gf_grid* g);
template <>
const gf::K0Param<double>& k0<double>(const gf_grid* g) { return g->K0d; }
template <>
const gf::K0Param<float>& k0<float>(const gf_grid* g) { return g->K0f; }

template <typename T>
struct LvBuf;
template <>
struct LvBuf<double> {
    static double* b(Level& L) { return L.b64; }
    static double* x(Level& L) { return L.x64; }
    static double* t(Level& L) { return L.t64; }
    static double* r(Level& L) { return L.r64; }
    static double* q(Level& L) { return L.q64; }
    static const double* E(Level& L) { return L.E64; }
};
template <>
struct LvBuf<float> {
    static float* b(Level& L) { return L.b32; }
    static float* x(Level& L) { return L.x32; }
    static float* t(Level& L) { return L.t32; }
    static float* r(Level& L) { return L.r32; }
    static float* q(Level& L) { return L.q32; }
    static const float* E(Level& L) { return L.E32; }
};

template <typename T>
const T* gal_ke(const Level& L);
template <>
const double* gal_ke<double>(const Level& L) { return L.Ke64; }
template <>
const float* gal_ke<float>(const Level& L) { return L.Ke32; }

// Galerkin level operator (csrc/galerkin.cuh) on level l >= 1
template <typename T, int MODE>
int gal_level(gf_grid* g, int l, const T* x, const T* b, T* out, T omega, const int* halt)
{
    const Level& L = g->lv[l];
    LAUNCH(g, nblk(8 * L.nodes), 256, (gf::gal_node_kernel<T, MODE, T, T>), x, b, out, gal_ke<T>(L), L.dims(),
           omega, halt, (T*)nullptr, (const double*)nullptr);
    return GF_OK;
}

// Coarse-grid correction of level l: x += P xc, or (theta > 0) the line-searched,
// rejectable form x += alpha P xc (csrc/linesearch.cuh); c is free scratch of the level,
// r the level's residual before the correction.
template <typename T>
int coarse_correct(gf_grid* g, int l, T* x, const T* xc, T* c, const T* r, double theta, const int* halt);

template <typename T>
int coarsest_solve(gf_grid* g, const T* b, T* x, const int* halt);
template <typename TB, typename TX>
int free_gemv(gf_grid* g, const TB* b, TX* x, const int* halt);

// One V-cycle z = B v in precision T (Table solver-config: 2:1 trilinear transfer,
// damped node-block Jacobi smoothing, coarsest solve by the FP64 dense inverse).
template <typename T>
int vcycle_impl(gf_grid* g, const double* v, double* z, int nu1, int nu2, T omega, const int* halt, double ls = 0.0)
{
    using B = LvBuf<T>;
    const int L = g->L;
    const int NX0 = g->nx + 1;
    g->stats.vcycles++;
    if (L == 1) {
        double* bm = g->lv[0].b64;
        LAUNCH(g, 2 * g->sms, 256, (gf::masked_convert_kernel<double, double>), v, bm, g->ndof, NX0, halt, (const uint8_t*)g->lv[0].fix);
        if (g->coarse_ldl) return free_gemv<double, double>(g, (const double*)bm, z, halt);
        LAUNCH(g, nblk(32LL * g->nc), 256, (gf::dense_gemv_kernel<double, double>), g->Ainv, (const double*)bm, z,
               g->nc, halt);
        return GF_OK;
    }
    std::vector<T*> cur(L);
    // level-0 right-hand side
    const T* b0;
    if constexpr (sizeof(T) == sizeof(double)) {
        b0 = reinterpret_cast<const T*>(v);
    } else {
        LAUNCH(g, 2 * g->sms, 256, (gf::masked_convert_kernel<double, T>), v, B::b(g->lv[0]), g->ndof, NX0, halt, (const uint8_t*)g->lv[0].fix);
        b0 = B::b(g->lv[0]);
    }
    for (int l = 0; l < L - 1; ++l) {
        Level& lev = g->lv[l];
        const T* b = (l == 0) ? b0 : B::b(lev);
        T* x = B::x(lev);
        T* t = B::t(lev);
        const int tpb = g->tpb[sizeof(T) == sizeof(double) ? 0 : 1] > 0 ? g->tpb[sizeof(T) == sizeof(double) ? 0 : 1]
                                                                          : 256;
        if (l == 0)   // levels >= 1 got their first sweep with the restriction
            LAUNCH(g, nblk(lev.nodes, tpb), tpb, (gf::first_sweep_kernel<T, T, T>), b, x, B::E(lev), lev.dims(),
                   k0<T>(g), omega, halt);
        for (int s = 1; s < nu1; ++s) {
            RET((stencil<T, T, gf::ST_SWEEP>(g, l, x, b, t, B::E(lev), k0<T>(g), omega, halt)));
            std::swap(x, t);
        }
        cur[l] = x;
        RET((stencil<T, T, gf::ST_RESID>(g, l, x, b, B::r(lev), B::E(lev), k0<T>(g), omega, halt)));
        Level& c = g->lv[l + 1];
        if (l + 1 < L - 1)
            LAUNCH(g, lv_grid(g, c.nodes), lv_block(g, c.nodes), gf::restrict_first_sweep_kernel<T>,
                   (const T*)B::r(lev), B::b(c), B::x(c),
                   (const T*)B::E(c), c.dims(), k0<T>(g), omega, halt);
        else
            LAUNCH(g, lv_grid(g, c.nodes), lv_block(g, c.nodes), gf::restrict_kernel<T>,
                   B::r(lev), B::b(c), c.dims(), halt);
    }
    {
        Level& c = g->lv[L - 1];
        RET(coarsest_solve<T>(g, (const T*)B::b(c), B::x(c), halt));
        cur[L - 1] = B::x(c);
    }
    for (int l = L - 2; l >= 0; --l) {
        Level& lev = g->lv[l];
        const T* b = (l == 0) ? b0 : B::b(lev);
        T* x = cur[l];
        T* t = (x == B::x(lev)) ? B::t(lev) : B::x(lev);
        RET(coarse_correct<T>(g, l, x, cur[l + 1], t, B::r(lev), ls, halt));
        for (int s = 0; s < nu2; ++s) {
            T* out = t;
            const bool last = (l == 0 && s == nu2 - 1);
            if constexpr (sizeof(T) == sizeof(double)) {
                if (last) out = reinterpret_cast<T*>(z);
            }
            RET((stencil<T, T, gf::ST_SWEEP>(g, l, x, b, out, B::E(lev), k0<T>(g), omega, halt)));
            if (last && sizeof(T) == sizeof(double)) {
                x = out;
                break;
            }
            std::swap(x, t);
        }
        cur[l] = x;
    }
    if constexpr (sizeof(T) != sizeof(double))
        LAUNCH(g, 2 * g->sms, 256, (gf::masked_convert_kernel<T, double>), (const T*)cur[0], z, g->ndof, NX0, halt, (const uint8_t*)g->lv[0].fix);
    return GF_OK;
}

// The mixed V-cycle (FP32 stencils, linear or tiled per the grid's tuning): level 0's first
// sweep reads the FP64 input v and stores it rounded to FP32 (b32) for the level's other
// sweeps and residual (a conversion per entry instead of one per read: the conversions
// run on the FP64 pipe), and the last post-sweep writes the FP64 result z, so no
// separate conversion passes are needed.
int vcycle_mixed_tiled(gf_grid* g, const double* v, double* z, int nu1, int nu2, float omega, const int* halt,
                       double ls = 0.0)
{
    const int L = g->L;
    g->stats.vcycles++;
    std::vector<float*> cur(L);
    const int lc = g->coarse_steps > 0 ? 0 : g->vc_l0;   // levels >= lc run in one cluster launch
    const int Ldown = (lc > 0) ? lc : L - 1;
    for (int l = 0; l < Ldown; ++l) {
        Level& lev = g->lv[l];
        float* x = lev.x32;
        float* t = lev.t32;
        if (l == 0) {
            LAUNCH(g, nblk(lev.nodes), 256, (gf::first_sweep_store_kernel<float, float, double>), v, lev.b32, x,
                   (const float*)lev.E32, lev.dims(), g->K0f, omega, halt);
            for (int s = 1; s < nu1; ++s) {
                RET((tiled_f32<gf::ST_SWEEP, float, float>(g, l, x, lev.b32, t, lev.E32, omega, halt)));
                std::swap(x, t);
            }
            RET((tiled_f32<gf::ST_RESID, float, float>(g, l, x, lev.b32, lev.r32, lev.E32, omega, halt)));
        } else {   // first sweep done together with the restriction into this level
            for (int s = 1; s < nu1; ++s) {
                RET((tiled_f32<gf::ST_SWEEP, float, float>(g, l, x, lev.b32, t, lev.E32, omega, halt)));
                std::swap(x, t);
            }
            RET((tiled_f32<gf::ST_RESID, float, float>(g, l, x, lev.b32, lev.r32, lev.E32, omega, halt)));
        }
        cur[l] = x;
        Level& c = g->lv[l + 1];
        if (l + 1 < Ldown)
            LAUNCH(g, lv_grid(g, c.nodes), lv_block(g, c.nodes), gf::restrict_first_sweep_kernel<float>,
                   (const float*)lev.r32, c.b32, c.x32,
                   (const float*)c.E32, c.dims(), g->K0f, omega, halt);
        else
            LAUNCH(g, lv_grid(g, c.nodes), lv_block(g, c.nodes), gf::restrict_kernel<float>,
                   (const float*)lev.r32, c.b32, c.dims(), halt);
    }
    if (lc > 0) {
        gf::VcArgs va{};
        for (int l = lc; l < L; ++l) {
            Level& q = g->lv[l];
            va.lv[l] = gf::VcLevel{q.dims(), q.nodes, q.E32, q.b32, q.x32, q.t32, q.r32};
        }
        va.l0 = lc;
        va.L = L;
        va.nu1 = nu1;
        va.nu2 = nu2;
        va.nc = g->nc;
        va.omega = omega;
        va.Ainv = g->Ainv;
        va.halt = halt;
        LAUNCH(g, gf::VC_CLUSTER, gf::VC_THREADS, gf::coarse_vcycle_kernel, va, g->K0f);
        // the level-lc result sits in x32 or t32 by the parity of its smoothing swaps
        cur[lc] = (((nu1 - 1) + nu2) & 1) ? g->lv[lc].t32 : g->lv[lc].x32;
    } else {
        Level& c = g->lv[L - 1];
        RET(coarsest_solve<float>(g, (const float*)c.b32, c.x32, halt));
        cur[L - 1] = c.x32;
    }
    for (int l = ((lc > 0) ? lc : L - 1) - 1; l >= 0; --l) {
        Level& lev = g->lv[l];
        float* x = cur[l];
        float* t = (x == lev.x32) ? lev.t32 : lev.x32;
        RET(coarse_correct<float>(g, l, x, (const float*)cur[l + 1], t, lev.r32, ls, halt));
        for (int s = 0; s < nu2; ++s) {
            const bool last = (s == nu2 - 1);
            if (l == 0 && last) {
                RET((tiled_f32<gf::ST_SWEEP, float, double>(g, 0, x, lev.b32, z, lev.E32, omega, halt)));
            } else if (l == 0) {
                RET((tiled_f32<gf::ST_SWEEP, float, float>(g, 0, x, lev.b32, t, lev.E32, omega, halt)));
                std::swap(x, t);
            } else {
                RET((tiled_f32<gf::ST_SWEEP, float, float>(g, l, x, lev.b32, t, lev.E32, omega, halt)));
                std::swap(x, t);
            }
        }
        cur[l] = x;
    }
    return GF_OK;
}

int alloc(void** p, size_t bytes);
template <typename T>
int allocT(T** p, size_t n);

// Chebyshev slot of precision p (0 FP64, 1 FP32) and level l: [lambda, c1_0, c2_0, c1_1, ...]
double* cheb_slot(gf_grid* g, int p, int l) { return g->cheb + ((long long)p * g->L + l) * (1 + 2 * gf::CHEB_MAXDEG); }

// lambda_max of D_b^{-1} K on every smoothing level by the power method, and the
// Chebyshev coefficients; for the operator the V-cycle of precision prec smooths with
// (FP64 moduli, or the FP32 ones from the BF16 density). Runs outside graph capture.
template <typename T>
int cheb_setup_impl(gf_grid* g)
{
    using B = LvBuf<T>;
    const int p = sizeof(T) == sizeof(double) ? 0 : 1;
    for (int l = 0; l < g->L - 1; ++l) {
        Level& lev = g->lv[l];
        const long long n = 3 * lev.nodes;
        T* v = B::x(lev);
        T* w = B::t(lev);
        LAUNCH(g, nblk(n), 256, gf::cheb_ones_kernel<T>, v, n, lev.nx + 1);
        LAUNCH(g, 1, 1024, gf::cheb_sumsq_kernel<T>, (const T*)v, n, g->cheb_ss);
        LAUNCH(g, nblk(n), 256, gf::cheb_normalize_kernel<T>, (const T*)v, v, n, (const double*)g->cheb_ss);
        const bool gal = l > 0 && g->coarse_kind == GF_COARSE_GALERKIN;
        for (int it = 0; it < gf::CHEB_POWER_ITERS; ++it) {
            if (gal) {   // w = D^{-1} K v with the level's Galerkin operator (r as scratch)
                RET((gal_level<T, gf::ST_APPLY>(g, l, (const T*)v, (const T*)nullptr, B::r(lev), T(0), nullptr)));
                RET((gal_level<T, gf::GAL_FIRST>(g, l, (const T*)nullptr, (const T*)B::r(lev), w, T(1), nullptr)));
            } else {
                LAUNCH(g, nblk(lev.nodes), 256, (gf::dinvk_kernel<T, T>), (const T*)v, w, (const T*)B::E(lev),
                       lev.dims(), k0<T>(g));
            }
            LAUNCH(g, 1, 1024, gf::cheb_sumsq_kernel<T>, (const T*)w, n, g->cheb_ss);
            LAUNCH(g, nblk(n), 256, gf::cheb_normalize_kernel<T>, (const T*)w, v, n, (const double*)g->cheb_ss);
        }
        double* slot = cheb_slot(g, p, l);
        LAUNCH(g, 1, 32, gf::cheb_coef_kernel, (const double*)g->cheb_ss, slot, slot + 1);
    }
    return GF_OK;
}

int ensure_cheb(gf_grid* g, int prec)
{
    const int p = prec == GF_FP64 ? 0 : 1;
    if (g->cheb_ready[p]) return GF_OK;
    if (!g->cheb) {
        RET(allocT(&g->cheb, (size_t)2 * g->L * (1 + 2 * gf::CHEB_MAXDEG)));
        RET(allocT(&g->cheb_ss, 1));
    }
    if (p == 0) RET(cheb_setup_impl<double>(g));
    else RET(cheb_setup_impl<float>(g));
    g->cheb_ready[p] = true;
    return GF_OK;
}

// The V-cycle with Chebyshev smoothing (degree nu1 pre, nu2 post), otherwise as
// vcycle_impl: FP64 or FP32 levels (the FP32 form converts the FP64 right-hand side
// and result), restriction, coarsest GEMV, prolongation. The residual buffer of a
// level holds the Chebyshev direction d while the level smooths.
template <typename T>
int vcycle_cheb(gf_grid* g, const double* v, double* z, int nu1, int nu2, const int* halt)
{
    using B = LvBuf<T>;
    const int L = g->L, p = sizeof(T) == sizeof(double) ? 0 : 1;
    const int NX0 = g->nx + 1;
    g->stats.vcycles++;
    if (L == 1) return vcycle_impl<T>(g, v, z, nu1, nu2, T(0.6), halt);
    std::vector<T*> cur(L);
    const T* b0;
    if constexpr (sizeof(T) == sizeof(double)) {
        b0 = reinterpret_cast<const T*>(v);
    } else {
        LAUNCH(g, 2 * g->sms, 256, (gf::masked_convert_kernel<double, T>), v, B::b(g->lv[0]), g->ndof, NX0, halt, (const uint8_t*)g->lv[0].fix);
        b0 = B::b(g->lv[0]);
    }
    auto smooth = [&](int l, const T* b, T*& x, T*& t, int degree, bool from_zero) -> int {
        Level& lev = g->lv[l];
        const double* coef = cheb_slot(g, p, l) + 1;
        const bool gal = l > 0 && g->coarse_kind == GF_COARSE_GALERKIN;
        for (int k = 0; k < degree; ++k) {
            const T* xin = (from_zero && k == 0) ? (const T*)nullptr : (const T*)x;
            if (gal)
                LAUNCH(g, nblk(8 * lev.nodes), 256, (gf::gal_node_kernel<T, gf::GAL_CHEB, T, T>), xin, b, t,
                       gal_ke<T>(lev), lev.dims(), T(1), halt, B::r(lev), coef + 2 * k);
            else
                LAUNCH(g, nblk(lev.nodes), 256, (gf::cheb_step_kernel<T, T>), xin, b, t, B::r(lev),
                       (const T*)B::E(lev), lev.dims(), k0<T>(g), coef + 2 * k, halt);
            std::swap(x, t);
        }
        return GF_OK;
    };
    for (int l = 0; l < L - 1; ++l) {
        Level& lev = g->lv[l];
        const T* b = (l == 0) ? b0 : B::b(lev);
        T* x = B::t(lev);   // the first step writes B::x (x and t swap after every step)
        T* t = B::x(lev);
        RET(smooth(l, b, x, t, nu1, true));
        cur[l] = x;
        if (l > 0 && g->coarse_kind == GF_COARSE_GALERKIN)
            RET((gal_level<T, gf::ST_RESID>(g, l, (const T*)x, b, B::r(lev), T(0), halt)));
        else
            RET((stencil<T, T, gf::ST_RESID>(g, l, x, b, B::r(lev), B::E(lev), k0<T>(g), T(0), halt)));
        Level& c = g->lv[l + 1];
        LAUNCH(g, lv_grid(g, c.nodes), lv_block(g, c.nodes), gf::restrict_kernel<T>,
               B::r(lev), B::b(c), c.dims(), halt);
    }
    {
        Level& c = g->lv[L - 1];
        RET(coarsest_solve<T>(g, (const T*)B::b(c), B::x(c), halt));
        cur[L - 1] = B::x(c);
    }
    for (int l = L - 2; l >= 0; --l) {
        Level& lev = g->lv[l];
        const T* b = (l == 0) ? b0 : B::b(lev);
        T* x = cur[l];
        T* t = (x == B::x(lev)) ? B::t(lev) : B::x(lev);
        LAUNCH(g, lv_grid(g, lev.nodes), lv_block(g, lev.nodes), (gf::prolong_add_kernel<T, T>), x, cur[l + 1],
               lev.dims(), halt);
        RET(smooth(l, b, x, t, nu2, false));
        cur[l] = x;
    }
    if constexpr (sizeof(T) == sizeof(double))
        CK(cudaMemcpyAsync(z, cur[0], sizeof(double) * g->ndof, cudaMemcpyDeviceToDevice, g->cur_stream));
    else
        LAUNCH(g, 2 * g->sms, 256, (gf::masked_convert_kernel<T, double>), (const T*)cur[0], z, g->ndof, NX0, halt, (const uint8_t*)g->lv[0].fix);
    return GF_OK;
}

int vcycle_dispatch_plain(gf_grid* g, const double* v, double* z, int prec, int nu1, int nu2, double omega,
                          const int* halt, int smoother, double ls);
template <typename T>
int fine_correct(gf_grid* g, const double* v, double* z, int steps, const int* halt);

// The V-cycle on the Galerkin hierarchy: vcycle_impl's schedule, with every level
// l >= 1 smoothed, and its residual formed, by the assembled coarse operator
// (first sweep from x = 0, then nu1 - 1 sweeps, residual, restriction; prolongation,
// nu2 sweeps). Level 0 keeps the matrix-free stencils; the coarsest solve uses the
// dense inverse of the assembled Galerkin matrix.
template <typename T>
int vcycle_galerkin(gf_grid* g, const double* v, double* z, int nu1, int nu2, T omega, const int* halt,
                    double ls = 0.0)
{
    using B = LvBuf<T>;
    const int L = g->L;
    const int NX0 = g->nx + 1;
    g->stats.vcycles++;
    std::vector<T*> cur(L);
    const T* b0;
    if constexpr (sizeof(T) == sizeof(double)) {
        b0 = reinterpret_cast<const T*>(v);
    } else {
        LAUNCH(g, 2 * g->sms, 256, (gf::masked_convert_kernel<double, T>), v, B::b(g->lv[0]), g->ndof, NX0, halt, (const uint8_t*)g->lv[0].fix);
        b0 = B::b(g->lv[0]);
    }
    for (int l = 0; l < L - 1; ++l) {
        Level& lev = g->lv[l];
        const T* b = (l == 0) ? b0 : B::b(lev);
        T* x = B::x(lev);
        T* t = B::t(lev);
        if (l == 0) {
            const int tpb = g->tpb[sizeof(T) == sizeof(double) ? 0 : 1] > 0 ? g->tpb[sizeof(T) == sizeof(double) ? 0 : 1]
                                                                              : 256;
            LAUNCH(g, nblk(lev.nodes, tpb), tpb, (gf::first_sweep_kernel<T, T, T>), b, x, B::E(lev), lev.dims(),
                   k0<T>(g), omega, halt);
            for (int s = 1; s < nu1; ++s) {
                RET((stencil<T, T, gf::ST_SWEEP>(g, 0, x, b, t, B::E(lev), k0<T>(g), omega, halt)));
                std::swap(x, t);
            }
            RET((stencil<T, T, gf::ST_RESID>(g, 0, x, b, B::r(lev), B::E(lev), k0<T>(g), omega, halt)));
        } else {
            RET((gal_level<T, gf::GAL_FIRST>(g, l, (const T*)nullptr, b, x, omega, halt)));
            for (int s = 1; s < nu1; ++s) {
                RET((gal_level<T, gf::ST_SWEEP>(g, l, x, b, t, omega, halt)));
                std::swap(x, t);
            }
            RET((gal_level<T, gf::ST_RESID>(g, l, x, b, B::r(lev), omega, halt)));
        }
        cur[l] = x;
        Level& c = g->lv[l + 1];
        LAUNCH(g, lv_grid(g, c.nodes), lv_block(g, c.nodes), gf::restrict_kernel<T>,
               (const T*)B::r(lev), B::b(c), c.dims(), halt);
    }
    {
        Level& c = g->lv[L - 1];
        RET(coarsest_solve<T>(g, (const T*)B::b(c), B::x(c), halt));
        cur[L - 1] = B::x(c);
    }
    for (int l = L - 2; l >= 0; --l) {
        Level& lev = g->lv[l];
        const T* b = (l == 0) ? b0 : B::b(lev);
        T* x = cur[l];
        T* t = (x == B::x(lev)) ? B::t(lev) : B::x(lev);
        RET(coarse_correct<T>(g, l, x, cur[l + 1], t, B::r(lev), ls, halt));
        for (int s = 0; s < nu2; ++s) {
            T* out = t;
            const bool last = (l == 0 && s == nu2 - 1);
            if constexpr (sizeof(T) == sizeof(double)) {
                if (last) out = reinterpret_cast<T*>(z);
            }
            if (l == 0) RET((stencil<T, T, gf::ST_SWEEP>(g, 0, x, b, out, B::E(lev), k0<T>(g), omega, halt)));
            else RET((gal_level<T, gf::ST_SWEEP>(g, l, x, b, out, omega, halt)));
            if (last && sizeof(T) == sizeof(double)) {
                x = out;
                break;
            }
            std::swap(x, t);
        }
        cur[l] = x;
    }
    if constexpr (sizeof(T) != sizeof(double))
        LAUNCH(g, 2 * g->sms, 256, (gf::masked_convert_kernel<T, double>), (const T*)cur[0], z, g->ndof, NX0, halt, (const uint8_t*)g->lv[0].fix);
    return GF_OK;
}

// The preconditioner: one V-cycle, then (fine > 0) the fine-level adaptive correction.
int vcycle_dispatch(gf_grid* g, const double* v, double* z, int prec, int nu1, int nu2, double omega,
                    const int* halt, int smoother = 0, double ls = 0.0, int fine = 0)
{
    RET(vcycle_dispatch_plain(g, v, z, prec, nu1, nu2, omega, halt, smoother, ls));
    if (fine <= 0) return GF_OK;
    if (!g->fc || g->fc_steps < fine || g->fc_es != (prec == GF_MIXED ? (int)sizeof(float) : (int)sizeof(double)))
        return set_err(GF_ERR_STATE, "fine-level correction buffers not set up");
    if (prec == GF_MIXED) return fine_correct<float>(g, v, z, fine, halt);
    return fine_correct<double>(g, v, z, fine, halt);
}

int vcycle_dispatch_plain(gf_grid* g, const double* v, double* z, int prec, int nu1, int nu2, double omega,
                          const int* halt, int smoother, double ls)
{
    if (ls > 0.0 && (smoother == 1 || g->vc_l0 > 0 || g->L < 2 || !g->ls_alpha))
        return set_err(GF_ERR_ARG, "the line-searched coarse correction needs Jacobi smoothing, >= 2 levels and no "
                                   "cluster V-cycle");
    if (g->coarse_kind == GF_COARSE_GALERKIN && g->L > 1 && smoother == 0) {   // Chebyshev: vcycle_cheb
        if (prec == GF_MIXED) return vcycle_galerkin<float>(g, v, z, nu1, nu2, (float)omega, halt, ls);
        return vcycle_galerkin<double>(g, v, z, nu1, nu2, omega, halt, ls);
    }
    if (smoother == 1) {
        if (!g->cheb_ready[prec == GF_FP64 ? 0 : 1]) return set_err(GF_ERR_STATE, "Chebyshev bounds not set up");
        if (prec == GF_MIXED) return vcycle_cheb<float>(g, v, z, nu1, nu2, halt);
        return vcycle_cheb<double>(g, v, z, nu1, nu2, halt);
    }
    if (prec == GF_MIXED) {
        if (g->L > 1) return vcycle_mixed_tiled(g, v, z, nu1, nu2, (float)omega, halt, ls);
        return vcycle_impl<float>(g, v, z, nu1, nu2, (float)omega, halt, ls);
    }
    return vcycle_impl<double>(g, v, z, nu1, nu2, omega, halt, ls);
}

void drop_graphs(gf_grid* g);

// buffers of the fine-level adaptive correction for `steps` inner steps in the V-cycle
// precision of `prec` (outside any graph capture)
int ensure_fc(gf_grid* g, int steps, int prec)
{
    const int es = (prec == GF_MIXED) ? (int)sizeof(float) : (int)sizeof(double);
    if (g->fc && g->fc_steps >= steps && g->fc_es == es) return GF_OK;
    drop_graphs(g);
    void** bufs[6] = {&g->fcV, &g->fcZ, &g->fcR, &g->fcD, &g->fcQ, &g->fcZT};
    for (void** b : bufs) {
        cudaFree(*b);
        *b = nullptr;
    }
    const size_t n = (size_t)g->ndof;
    RET(allocT((unsigned char**)&g->fcV, (size_t)(steps + 1) * n * es));
    RET(allocT((unsigned char**)&g->fcZ, (size_t)steps * n * es));
    RET(allocT((unsigned char**)&g->fcR, n * es));
    RET(allocT((unsigned char**)&g->fcD, n * es));
    RET(allocT((unsigned char**)&g->fcQ, n * es));
    RET(allocT((unsigned char**)&g->fcZT, n * es));
    if (!g->fc) {
        RET(allocT(&g->fc, 1));
        CK(cudaMemset(g->fc, 0, sizeof(gf::FcState)));
        // 2 blocks per SM (8 per SM measured slower: 2.4 -> 3.6 ms per outer step at 96x48x48)
        g->fc_nb = (int)std::min<long long>(2LL * g->sms, std::max<long long>(1, (g->ndof + 1023) / 1024));
        RET(allocT(&g->fc_partial, (size_t)g->fc_nb * gf::FC_SLOTS));
    }
    g->fc_steps = steps;
    g->fc_es = es;
    return GF_OK;
}

// The fine-level correction's and the coarse-level solve's inner FGMRES buffers, and
// the coarse-level steps the V-cycles of this call use (outside any graph capture).
int set_coarse_steps(gf_grid* g, const gf_solve_opts* o)
{
    const int coarse = g->L > 1 ? o->coarse_steps : 0;
    const int steps = std::max(o->fine_steps, coarse);
    if (steps > 0) RET(ensure_fc(g, steps, o->prec));
    g->coarse_steps = coarse;
    return GF_OK;
}

// steps steps of an inner FGMRES(steps) from d = 0 on K_l d = r on level l, preconditioned
// by the level's 3x3 node-block Jacobi operator (first_sweep_kernel with omega = 1, or
// the Galerkin form), in precision T (finecorr.cuh); d = Z y unless the solve is skipped
// (r = 0 or halted), when d is left as it was. nb blocks for the reductions (<= fc_nb).
template <typename T>
int inner_fgmres(gf_grid* g, int l, const T* r, T* d, int steps, const int* halt, int nb)
{
    Level& lev = g->lv[l];
    const long long n = lev.ndof;
    const bool gal = l > 0 && g->coarse_kind == GF_COARSE_GALERKIN;
    T *V = (T*)g->fcV, *Z = (T*)g->fcZ;
    gf::FcState* st = g->fc;
    LAUNCH(g, nb, gf::FC_THREADS, gf::fc_start_kernel<T>, r, n, st, g->fc_partial, halt);
    LAUNCH(g, 2 * g->sms, 256, gf::fc_scale_kernel<T>, r, V, n, (const gf::FcState*)st);
    const int* stop = &st->stop;
    for (int j = 0; j < steps; ++j) {
        T* vj = V + (long long)j * n;
        T* zj = Z + (long long)j * n;
        T* w = V + (long long)(j + 1) * n;
        if (gal) {
            RET((gal_level<T, gf::GAL_FIRST>(g, l, (const T*)nullptr, (const T*)vj, zj, T(1), stop)));
            RET((gal_level<T, gf::ST_APPLY>(g, l, (const T*)zj, (const T*)nullptr, w, T(0), stop)));
        } else {
            LAUNCH(g, nblk(lev.nodes), 256, (gf::first_sweep_kernel<T, T, T>), (const T*)vj, zj, LvBuf<T>::E(lev),
                   lev.dims(), k0<T>(g), T(1), stop);
            RET((stencil<T, T, gf::ST_APPLY>(g, l, (const T*)zj, (const T*)nullptr, w, LvBuf<T>::E(lev), k0<T>(g),
                                             T(0), stop)));
        }
        LAUNCH(g, nb, gf::FC_THREADS, gf::fc_dots1_kernel<T>, (const T*)V, n, (const T*)w, n, j, st, g->fc_partial);
        LAUNCH(g, nb, gf::FC_THREADS, gf::fc_dots2_kernel<T>, (const T*)V, n, w, n, j, st, g->fc_partial);
        LAUNCH(g, nb, gf::FC_THREADS, gf::fc_norm_kernel<T>, (const T*)V, n, w, n, j, steps, st, g->fc_partial);
        if (j + 1 < steps) LAUNCH(g, 2 * g->sms, 256, gf::fc_vscale_kernel<T>, w, n, (const gf::FcState*)st);
    }
    LAUNCH(g, 1, 32, gf::fc_backsolve_kernel, st);
    LAUNCH(g, 2 * g->sms, 256, gf::fc_combine_kernel<T>, (const T*)Z, n, d, n, (const gf::FcState*)st);
    return GF_OK;
}

// The coarsest level's solve x = A_c^{-1} b: the dense FP64 inverse, or (coarse_steps > 0)
// x = A^-1 b on the coarsest level with the free-DOF inverse the LDL^T path leaves in Agj
// (free_gemv_kernel; eight rows per CTA).
template <typename TB, typename TX>
int free_gemv(gf_grid* g, const TB* b, TX* x, const int* halt)
{
    const int m = g->ncf;
    const size_t smem = sizeof(double) * (size_t)std::max(1, m);
    static const bool ok = cudaFuncSetAttribute((const void*)gf::free_gemv_kernel<TB, TX>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024) == cudaSuccess;
    if (!ok) return set_err(GF_ERR_CUDA, "shared memory of free_gemv_kernel");
    LAUNCH_SMEM(g, std::max(1, (m + 7) / 8), 256, smem, (gf::free_gemv_kernel<TB, TX>), (const double*)g->Agj, m,
                (const int*)g->cidx, b, x, g->nc, (const int*)g->cpos, halt);
    return GF_OK;
}

// Table solver-config's inner Krylov solve on the coarse level, from x = 0.
template <typename T>
int coarsest_solve(gf_grid* g, const T* b, T* x, const int* halt)
{
    if (g->coarse_steps > 0 && g->L > 1) {
        Level& c = g->lv[g->L - 1];
        CK(cudaMemsetAsync(x, 0, sizeof(T) * c.ndof, g->cur_stream));
        const size_t smem = sizeof(T) * (size_t)(2 * g->coarse_steps + 1) * (size_t)c.ndof;
        if (g->ck_fused && g->coarse_kind != GF_COARSE_GALERKIN && smem <= (size_t)gf::CK_SMEM_MAX) {
            // one CTA, basis in shared memory (csrc/coarse_krylov.cuh)
            LAUNCH_SMEM(g, 1, gf::CK_THREADS, smem, gf::coarse_fgmres_kernel<T>, b, x, (const T*)LvBuf<T>::E(c),
                        c.dims(), k0<T>(g), g->coarse_steps, halt);
            return GF_OK;
        }
        const int nb = (int)std::min<long long>(g->fc_nb, std::max<long long>(1, (c.ndof + 1023) / 1024));
        return inner_fgmres<T>(g, g->L - 1, b, x, g->coarse_steps, halt, nb);
    }
    if (g->coarse_ldl) return free_gemv<T, T>(g, b, x, halt);
    LAUNCH(g, nblk(32LL * g->nc), 256, (gf::dense_gemv_kernel<T, T>), (const double*)g->Ainv, b, x, g->nc, halt);
    return GF_OK;
}

// the fine-level adaptive correction of z = V-cycle(v), in precision T (finecorr.cuh)
template <typename T>
int fine_correct(gf_grid* g, const double* v, double* z, int steps, const int* halt)
{
    Level& lev = g->lv[0];
    const long long n = g->ndof;
    T *r = (T*)g->fcR, *d = (T*)g->fcD, *q = (T*)g->fcQ;
    gf::FcState* st = g->fc;
    const int nb = g->fc_nb;
    if constexpr (sizeof(T) == sizeof(double)) {   // r = v - K z
        RET((stencil<double, double, gf::ST_RESID>(g, 0, z, v, (double*)r, lev.E64, g->K0d, 0.0, halt)));
    } else {
        float* zt = (float*)g->fcZT;
        LAUNCH(g, 2 * g->sms, 256, (gf::masked_convert_kernel<double, float>), (const double*)z, zt, n, g->nx + 1,
               halt, (const uint8_t*)nullptr);
        RET((tiled_f32<gf::ST_RESID, double, float>(g, 0, zt, v, (float*)r, lev.E32, 0.0f, halt)));
    }
    RET(inner_fgmres<T>(g, 0, (const T*)r, d, steps, halt, nb));
    RET((stencil<T, T, gf::ST_APPLY>(g, 0, (const T*)d, (const T*)nullptr, q, LvBuf<T>::E(lev), k0<T>(g), T(0),
                                     &st->skip)));
    LAUNCH(g, nb, gf::FC_THREADS, gf::fc_accept_kernel<T>, (const T*)r, (const T*)q, n, st, g->fc_partial);
    LAUNCH(g, 2 * g->sms, 256, gf::fc_apply_kernel<T>, z, (const T*)d, n, (const gf::FcState*)st);
    return GF_OK;
}

// buffers of the line-searched coarse correction (outside any graph capture)
int ensure_ls(gf_grid* g)
{
    if (g->ls_alpha) return GF_OK;
    for (int l = 0; l < g->L - 1; ++l) {
        RET(allocT(&g->lv[l].q64, g->lv[l].ndof));
        RET(allocT(&g->lv[l].q32, g->lv[l].ndof));
    }
    g->ls_nb = (int)std::min<long long>(2LL * g->sms, std::max<long long>(1, (g->ndof + 1023) / 1024));
    RET(allocT(&g->ls_partial, (size_t)2 * g->ls_nb));
    RET(allocT(&g->ls_alpha, 8));
    return GF_OK;
}

template <typename T>
int coarse_correct(gf_grid* g, int l, T* x, const T* xc, T* c, const T* r, double theta, const int* halt)
{
    Level& lev = g->lv[l];
    const int tpb = level_tpb(g, lev.nodes, 256);
    if (!(theta > 0.0)) {
        LAUNCH(g, nblk(lev.nodes, tpb), tpb, (gf::prolong_add_kernel<T, T>), x, xc, lev.dims(), halt);
        return GF_OK;
    }
    CK(cudaMemsetAsync(c, 0, sizeof(T) * lev.ndof, g->cur_stream));
    LAUNCH(g, nblk(lev.nodes, tpb), tpb, (gf::prolong_add_kernel<T, T>), c, xc, lev.dims(), halt);
    if (l > 0 && g->coarse_kind == GF_COARSE_GALERKIN)   // q = K_l c with the level's Galerkin operator
        RET((gal_level<T, gf::ST_APPLY>(g, l, (const T*)c, (const T*)nullptr, LvBuf<T>::q(lev), T(0), halt)));
    else
        RET((stencil<T, T, gf::ST_APPLY>(g, l, (const T*)c, (const T*)nullptr, LvBuf<T>::q(lev), LvBuf<T>::E(lev),
                                         k0<T>(g), T(0), halt)));
    const int nb = (int)std::min<long long>(g->ls_nb, std::max<long long>(1, (lev.ndof + 1023) / 1024));
    LAUNCH(g, nb, gf::LS_THREADS, gf::ls_dots_kernel<T>, (const T*)c, r, (const T*)LvBuf<T>::q(lev), lev.ndof,
           g->ls_partial, halt);
    LAUNCH(g, 1, 32, gf::ls_finish_kernel, (const double*)g->ls_partial, nb, theta, g->ls_alpha + l, halt);
    LAUNCH(g, 2 * g->sms, 256, gf::ls_axpy_kernel<T>, x, (const T*)c, lev.ndof, (const double*)(g->ls_alpha + l), halt);
    return GF_OK;
}

int applyK64(gf_grid* g, const double* u, double* y, const int* halt)
{
    g->stats.apply_K_fp64++;
    if (g->modal64_items) {   // modal factorisation of K0 (default; GF_MODAL=0: dense node stencil)
        const bool mk = g->lv[0].fix != nullptr;   // per-node fixed components (bridge supports)
        const double* Es = g->modal_es;
        const int4* it = g->modal64_items;
        const gf::GridDims d = g->lv[0].dims();
        const int bx = g->modal64_bx, by = g->modal64_by;
        const gf::ModalSide sd = gf::modal_side(d, bx, by);
        double* side = g->modal_side;
#define GF_MODAL64(BXV, BYV)                                                                                      \
    (mk ? launch_modal<double, BXV, BYV, gf::apply_modal_kernel<BXV, BYV, true>>(g, g->modal64_n, u, y, Es, d, it, \
                                                                                  side, sd, halt)                 \
        : launch_modal<double, BXV, BYV, gf::apply_modal_kernel<BXV, BYV, false>>(g, g->modal64_n, u, y, Es, d, it, \
                                                                                   side, sd, halt))
        if (bx == 32)
            RET(GF_MODAL64(32, 16));
        else if (by == 32)
            RET(GF_MODAL64(16, 32));
        else
            RET(GF_MODAL64(16, 16));
#undef GF_MODAL64
        const long long ne = sd.entries(d);
        if (mk)
            LAUNCH(g, (unsigned)((ne + 255) / 256), 256, gf::modal_fixup_kernel<true>, (const double*)side, sd, y, d,
                   halt);
        else
            LAUNCH(g, (unsigned)((ne + 255) / 256), 256, gf::modal_fixup_kernel<false>, (const double*)side, sd, y, d,
                   halt);
        return GF_OK;
    }
    return stencil<double, double, gf::ST_APPLY>(g, 0, u, nullptr, y, g->lv[0].E64, g->K0d, 0.0, halt);
}

// grid of the tensor-core split kernel: 15 x 7 nodes x 8 layers per CTA
dim3 split_tc_grid(const gf_grid* g)
{
    return dim3((g->nx + 1 + gf::TC_NX - 1) / gf::TC_NX, (g->ny + 1 + gf::TC_NY - 1) / gf::TC_NY,
                (g->nz + 1 + gf::TC_CZ - 1) / gf::TC_CZ);
}

int applyKsplit(gf_grid* g, const double* u, double* y, const int* halt)
{
    g->stats.apply_K_fp64++;
    if (g->split_tc) {
        LAUNCH_SMEM(g, split_tc_grid(g), gf::TC_THREADS, sizeof(gf::TcSmem), gf::apply_split_tc_kernel<false>, u, y,
                    (float2*)nullptr, (const float2*)g->Edf, g->lv[0].dims(), (const gf::TcBFrag*)g->Btc, halt);
        return GF_OK;
    }
    const dim3 grid((g->nx + 1 + gf::SPX - 1) / gf::SPX, (g->ny + 1 + gf::SPY - 1) / gf::SPY,
                    (g->nz + 1 + gf::SPZ - 1) / gf::SPZ);
    LAUNCH(g, grid, dim3(gf::SPX, gf::SPY, gf::SPZ), gf::apply_split_kernel<false>, u, y, (float2*)nullptr,
           (const float2*)g->Edf, g->lv[0].dims(), g->Msplit, halt);
    return GF_OK;
}

// The same product written as double-float pairs (input of the double-float CGS2).
int applyKsplit_dd(gf_grid* g, const double* u, float2* yd, const int* halt)
{
    g->stats.apply_K_fp64++;
    if (g->split_tc) {
        LAUNCH_SMEM(g, split_tc_grid(g), gf::TC_THREADS, sizeof(gf::TcSmem), gf::apply_split_tc_kernel<true>, u,
                    (double*)nullptr, yd, (const float2*)g->Edf, g->lv[0].dims(), (const gf::TcBFrag*)g->Btc, halt);
        return GF_OK;
    }
    const dim3 grid((g->nx + 1 + gf::SPX - 1) / gf::SPX, (g->ny + 1 + gf::SPY - 1) / gf::SPY,
                    (g->nz + 1 + gf::SPZ - 1) / gf::SPZ);
    LAUNCH(g, grid, dim3(gf::SPX, gf::SPY, gf::SPZ), gf::apply_split_kernel<true>, u, (double*)nullptr, yd,
           (const float2*)g->Edf, g->lv[0].dims(), g->Msplit, halt);
    return GF_OK;
}

// The outer (Krylov) operator: native FP64, or the split-integer FP64-class one.
int applyOuter(gf_grid* g, const double* u, double* y, const int* halt, int outer)
{
    return outer ? applyKsplit(g, u, y, halt) : applyK64(g, u, y, halt);
}

// ------------------------------------------------------------------ set-up ----
int alloc(void** p, size_t bytes)
{
    CK(cudaMalloc(p, bytes));
    return GF_OK;
}

template <typename T>
int allocT(T** p, size_t n)
{
    return alloc(reinterpret_cast<void**>(p), n * sizeof(T));
}

// Galerkin element matrices of levels 1 .. L-1 (csrc/galerkin.cuh): Ke64 from the FP64
// moduli; Ke32 from the BF16-density moduli, that chain carried in FP64 scratch and
// rounded to FP32 per level (the mixed V-cycle's coarse operators).
int build_galerkin(gf_grid* g)
{
    const int L = g->L;
    if (L < 2) return GF_OK;
    if (!g->galG) {
        std::vector<double> G(8 * gf::GAL_KE);
        for (int c = 0; c < 8; ++c)
            for (int R = 0; R < 24; ++R)
                for (int S = 0; S < 24; ++S) {
                    const int b = R / 3, i = R % 3, bp = S / 3, j = S % 3;
                    double acc = 0.0;
                    for (int a = 0; a < 8; ++a)
                        for (int ap = 0; ap < 8; ++ap)
                            acc += gf::gal_weight(c, a, b) * g->K0d.k[(3 * a + i) * 24 + 3 * ap + j] *
                                   gf::gal_weight(c, ap, bp);
                    G[(c * 24 + R) * 24 + S] = acc;
                }
        RET(allocT(&g->galG, G.size()));
        CK(cudaMemcpy(g->galG, G.data(), G.size() * sizeof(double), cudaMemcpyHostToDevice));
        for (int l = 1; l < L; ++l) {
            Level& c = g->lv[l];
            RET(allocT(&c.Ke64, (size_t)c.nel * gf::GAL_KE));
            RET(allocT(&c.Ke32, (size_t)c.nel * gf::GAL_KE));
        }
        RET(allocT(&g->gal_s[0], (size_t)g->lv[1].nel * gf::GAL_KE));
        if (L > 2) RET(allocT(&g->gal_s[1], (size_t)g->lv[2].nel * gf::GAL_KE));
    }
    Level& c1 = g->lv[1];
    const long long n1 = c1.nel * gf::GAL_KE;
    LAUNCH(g, nblk(n1), 256, gf::gal_first_level_kernel<double>, (const double*)g->lv[0].E64,
           (const double*)g->galG, c1.Ke64, (float*)nullptr, c1.dims());
    LAUNCH(g, nblk(n1), 256, gf::gal_first_level_kernel<float>, (const float*)g->lv[0].E32, (const double*)g->galG,
           g->gal_s[0], c1.Ke32, c1.dims());
    for (int l = 2; l < L; ++l) {
        Level& c = g->lv[l];
        const long long nl = c.nel * gf::GAL_KE;
        LAUNCH(g, nblk(nl), 256, gf::gal_coarsen_kernel, (const double*)g->lv[l - 1].Ke64, c.Ke64, (float*)nullptr,
               c.dims());
        LAUNCH(g, nblk(nl), 256, gf::gal_coarsen_kernel, (const double*)g->gal_s[(l - 2) & 1], g->gal_s[(l - 1) & 1],
               c.Ke32, c.dims());
    }
    return GF_OK;
}

// The coarsest level's free-DOF map (cpos, cidx, ncf) for the current supports.
int build_coarse_map(gf_grid* g)
{
    const Level& c = g->lv[g->L - 1];
    gf::coarse_map_kernel<<<1, 32, 0, g->stream>>>(c.dims(), g->cpos, g->cidx, g->cidx + g->nc);
    CK(cudaGetLastError());
    int m = 0;
    CK(cudaMemcpyAsync(&m, g->cidx + g->nc, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    g->ncf = m;
    // nodes couple to the 27 nodes around them: in the compact order (coarse_axes) their
    // positions differ by at most 1 + N_a + N_a N_b, DOF positions by 3 of that + 2;
    // dropping the fixed DOFs only brings positions closer
    g->cband = gf::coarse_band(c.dims());
    return GF_OK;
}

// The coarsest inverse from the banded LDL^T factorisation (ldl.cuh): the free-DOF matrix
// assembled into Ainv (m x m), factored in place by blocks of LDL_C pivots, the inverse
// formed block by block from the last into Agj (m x m), then expanded into Ainv (n x n).
gf::LdlState ldl_state(gf_grid* g)
{
    gf::LdlState S;
    S.M = g->Ainv;
    S.Z = g->Agj;
    S.dinv = g->ldl_ws;
    S.Xs = S.dinv + g->nc;
    S.Qs = S.Xs + (long long)g->nc * gf::LDL_C;
    S.m = g->ncf;
    S.b = g->cband;
    return S;
}

// The free-DOF matrix of the coarsest level into M (the first step of either inverse).
int assemble_coarse_free(gf_grid* g, double* M)
{
    Level& c = g->lv[g->L - 1];
    const long long m = g->ncf;
    if (g->coarse_kind == GF_COARSE_GALERKIN && g->L > 1)
        LAUNCH(g, nblk(m * m), 256, gf::gal_assemble_kernel, (const double*)c.Ke64, M, c.dims(), (const int*)g->cidx,
               (int)m);
    else
        LAUNCH(g, nblk(m * m), 256, gf::coarse_assemble_kernel, c.E64, M, c.dims(), g->K0d, (const int*)g->cidx,
               (int)m);
    return GF_OK;
}

// Dynamic shared memory of the inverse's row and Y kernels (single and batched), once.
bool ldl_smem_opt_in()
{
    static const bool ok = [] {
        const int bytes = 200 * 1024;
        bool r = true;
        for (const void* k : {(const void*)gf::ldl_inv_rows_kernel, (const void*)gf::ldl_inv_diag_kernel,
                              (const void*)gf::ldl_inv_rows_batch_kernel, (const void*)gf::ldl_inv_diag_batch_kernel})
            r = r && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
        return r;
    }();
    return ok;
}

int build_coarse_inverse_ldl(gf_grid* g)
{
    const gf::LdlState S = ldl_state(g);
    const int m = S.m;
    RET(assemble_coarse_free(g, S.M));
    if (!ldl_smem_opt_in()) return set_err(GF_ERR_CUDA, "shared memory of the LDL^T inverse kernels");
    int j0, c, r1;
    for (int s = 0; gf::ldl_factor_step(m, S.b, s, j0, c, r1); ++s) {   // A = L D L^T
        LAUNCH(g, 1, 512, gf::ldl_diag_kernel, S, j0, c);
        if (j0 + c >= m) break;
        LAUNCH(g, gf::ldl_panel_ctas(j0 + c, r1), gf::LDL_WARPS * 32, gf::ldl_panel_kernel, S, j0, c, r1);
        LAUNCH(g, gf::ldl_update_ctas(j0 + c, r1), 256, gf::ldl_update_kernel, S, j0, c, r1);
    }
    int kend;
    for (int s = 0; gf::ldl_inverse_step(m, S.b, s, j0, c, kend); ++s) {   // Z = A^-1, last block first
        const int j1 = j0 + c;
        if (gf::ldl_rows_smem(kend - j1) > 200 * 1024)
            return set_err(GF_ERR_ARG, "coarsest band too wide for the LDL^T inverse");
        if (j1 < m)
            LAUNCH_SMEM(g, gf::ldl_rows_ctas(m, j1), gf::LDL_WARPS * 32, gf::ldl_rows_smem(kend - j1),
                        gf::ldl_inv_rows_kernel, S, j0, c, kend);
        LAUNCH_SMEM(g, c, gf::LDL_WARPS * 32, gf::ldl_diag_smem(kend - j1), gf::ldl_inv_diag_kernel, S, j0, c, kend);
        LAUNCH(g, gf::ldl_diag2_ctas(c), gf::LDL_WARPS * 32, gf::ldl_inv_diag2_kernel, S, j0, c);
    }
    const long long n = g->nc;
    LAUNCH(g, std::min<long long>(nblk(n * n), 4LL * g->sms), 256, gf::sym_expand_kernel, (const double*)S.Z, m,
           (const int*)g->cpos, g->Ainv, (int)n);
    return GF_OK;
}

int build_coarse_inverse(gf_grid* g)
{
    Level& c = g->lv[g->L - 1];
    const long long n = g->nc;
    gf::K0Param<double> K = g->K0d;   // the level's E64 already carries h
    if (g->coarse_ldl) return build_coarse_inverse_ldl(g);
    if (g->sym_gj) {
        // blocked symmetric sweep on the upper triangle of the operator restricted to the
        // free DOFs (m x m; the fixed ones only carry identity rows), ceil(m / SGJ_B)
        // double-buffered steps ending in Agj, then the expansion into Ainv (n x n)
        const long long m = g->ncf;
        const long long steps = (m + gf::SGJ_B - 1) / gf::SGJ_B;
        double* src = (steps & 1) ? g->Ainv : g->Agj;
        for (double* buf : {g->Ainv, g->Agj}) {   // both buffers start as A (the entries ahead of the band)
            if (g->coarse_kind == GF_COARSE_GALERKIN && g->L > 1)
                LAUNCH(g, nblk(m * m), 256, gf::gal_assemble_kernel, (const double*)c.Ke64, buf, c.dims(),
                       (const int*)g->cidx, (int)m);
            else
                LAUNCH(g, nblk(m * m), 256, gf::coarse_assemble_kernel, c.E64, buf, c.dims(), K, (const int*)g->cidx,
                       (int)m);
        }
        double* Pb = g->Agj + n * n;   // two P buffers past the matrix
        if (m > 0) LAUNCH(g, 1, 256, gf::sym_gj_first_kernel, (const double*)src, (int)m, Pb);
        for (long long k = 0; k < m; k += gf::SGJ_B) {
            double* dst = (src == g->Ainv) ? g->Agj : g->Ainv;
            const int s = (int)(k / gf::SGJ_B);
            const int tiles = (gf::sgj_active((int)m, (int)k, g->cband) + gf::SGJ_T - 1) / gf::SGJ_T;
            LAUNCH(g, 1 + tiles * (tiles + 1) / 2, dim3(16, 16), gf::sym_gj_kernel, (const double*)src, dst, (int)m,
                   (int)k, (const double*)(Pb + gf::SGJ_B * gf::SGJ_B * (s & 1)),
                   Pb + gf::SGJ_B * gf::SGJ_B * ((s + 1) & 1), tiles);
            src = dst;
        }
        LAUNCH(g, std::min<long long>(nblk(n * n), 4LL * g->sms), 256, gf::sym_expand_kernel, (const double*)g->Agj,
               (int)m, (const int*)g->cpos, g->Ainv, (int)n);
        return GF_OK;
    }
    // two-pivot Gauss-Jordan on all DOFs: ceil(n/2) double-buffered steps; start in the
    // buffer that makes the last one land in Ainv
    const long long steps = (n + 1) / 2;
    double* src = (steps & 1) ? g->Agj : g->Ainv;
    if (g->coarse_kind == GF_COARSE_GALERKIN && g->L > 1)
        LAUNCH(g, nblk(n * n), 256, gf::gal_assemble_kernel, (const double*)c.Ke64, src, c.dims(), (const int*)nullptr,
               0);
    else
        LAUNCH(g, nblk(n * n), 256, gf::coarse_assemble_kernel, c.E64, src, c.dims(), K, (const int*)nullptr, 0);
    LAUNCH(g, nblk(n * n), 256, gf::coarse_fix_kernel, src, c.dims());
    const unsigned tiles = (unsigned)((n + gf::GJ_T - 1) / gf::GJ_T);
    for (int k = 0; k < n; k += 2) {
        double* dst = (src == g->Ainv) ? g->Agj : g->Ainv;
        LAUNCH(g, dim3(tiles, tiles), dim3(gf::GJ_T, gf::GJ_R), gf::gj_step_kernel, (const double*)src, dst, (int)n, k);
        src = dst;
    }
    return GF_OK;
}

void drop_graphs(gf_grid* g)
{
    for (int j = 0; j < gf::KRY_MMAX; ++j) {
        if (g->step_exec[j]) cudaGraphExecDestroy(g->step_exec[j]);
        g->step_exec[j] = nullptr;
        g->step_nodes[j] = 0;
    }
}

int ensure_krylov(gf_grid* g, int m, int kmax, int outer)
{
    if (m > g->m_alloc || kmax + 1 > g->hist_cap || (outer == 2 && m > g->md_alloc)) drop_graphs(g);
    if (outer == 2 && m > g->md_alloc) {
        cudaFree(g->Vd);
        g->Vd = nullptr;
        g->md_alloc = 0;
        RET(allocT(&g->Vd, (size_t)(m + 1) * g->ldk));
        if (!g->pdd) {
            // each pass's grid is the blocks resident at once on this GPU (one round),
            // capped by the number of row tiles
            const long long tiles = (g->ndof + gf::DD_TILE - 1) / gf::DD_TILE;
            const void* kern[3][3] = {
                {(const void*)gf::ddgs_dots_kernel<8>, (const void*)gf::ddgs_dots_kernel<16>,
                 (const void*)gf::ddgs_dots_kernel<32>},
                {(const void*)gf::ddgs_update_dots_kernel<8>, (const void*)gf::ddgs_update_dots_kernel<16>,
                 (const void*)gf::ddgs_update_dots_kernel<32>},
                {(const void*)gf::ddgs_update_norm_kernel<8>, (const void*)gf::ddgs_update_norm_kernel<16>,
                 (const void*)gf::ddgs_update_norm_kernel<32>}};
            g->nbd = 1;
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q) {
                    int nb = 0;
                    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern[p][q], gf::DD_THREADS, 0) != cudaSuccess ||
                        nb <= 0)
                        nb = 2;
                    g->nbd_k[p][q] = (int)std::max<long long>(1, std::min<long long>((long long)nb * g->sms, tiles));
                    g->nbd = std::max(g->nbd, g->nbd_k[p][q]);
                }
            RET(allocT(&g->pdd, (size_t)g->nbd * (gf::KRY_NV + 1)));
            RET(allocT(&g->ddticket, 1));
            CK(cudaMemset(g->ddticket, 0, sizeof(unsigned int)));
        }
        g->md_alloc = m;
    }
    if (m > g->m_alloc) {
        cudaFree(g->V);
        cudaFree(g->Z);
        g->V = g->Z = nullptr;
        g->m_alloc = 0;
        RET(allocT(&g->V, (size_t)(m + 1) * g->ldk));
        RET(allocT(&g->Z, (size_t)m * g->ldk));
        g->m_alloc = m;
    }
    if (kmax + 1 > g->hist_cap) {
        cudaFree(g->hist);
        g->hist = nullptr;
        g->hist_cap = 0;
        RET(allocT(&g->hist, (size_t)kmax + 1));
        g->hist_cap = kmax + 1;
    }
    return GF_OK;
}

__global__ void init_state_kernel(gf::KState* st, int kmax, int m, double tol)
{
    st->k = 0;
    st->kmax = kmax;
    st->m = m;
    st->tol = tol;
    st->status = gf::KS_RUN;
    st->flag = 1;
    st->J = 0;
    st->j = 0;
    st->skip = 0;
}

struct HostState {
    int k, flag, status, J;
};

int read_state(gf_grid* g, HostState* hs)
{
    gf::KState* st = g->st;
    CK(cudaMemcpyAsync(&hs->k, &st->k, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(&hs->flag, &st->flag, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(&hs->status, &st->status, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return GF_OK;
}

// Register width of the Gram-Schmidt passes for nv basis vectors: the FP64 passes also
// have a 24-wide form (17..24 vectors loaded in one group, against a second group of 1..8
// in the 32-wide one); the double-float passes 8, 16 and 32.
int pick_nv(int nv, bool dd)
{
    return nv <= 8 ? 8 : (nv <= 16 ? 16 : (nv <= 24 && !dd ? 24 : 32));
}

template <int NV>
int cgs2_step(gf_grid* g, int j, double* w, int outer)
{
    const long long n = g->ndof, ld = g->ldk;
    const int nv = j + 1;
    if constexpr (NV != 24) if (outer == 2) {   // double-float passes on the FP32 pipe; w arrives as wd
        float2* wd = g->Vd + (long long)(j + 1) * ld;
        const int q = NV == 8 ? 0 : (NV == 16 ? 1 : 2);
        LAUNCH(g, g->nbd_k[0][q], gf::DD_THREADS, gf::ddgs_dots_kernel<NV>, (const float2*)g->Vd, ld, nv,
               (const float2*)wd, n, g->pdd, g->st, g->ddticket);
        LAUNCH(g, g->nbd_k[1][q], gf::DD_THREADS, gf::ddgs_update_dots_kernel<NV>, (const float2*)g->Vd, ld, nv, wd,
               n, g->pdd, g->st, g->ddticket);
        LAUNCH(g, g->nbd_k[2][q], gf::DD_THREADS, gf::ddgs_update_norm_kernel<NV>, (const float2*)g->Vd, ld, nv, wd,
               n, g->pdd, g->st, g->ddticket);
        LAUNCH(g, 1, 32, gf::arnoldi_tail_kernel, g->st, g->hist, j, NV, g->host_status_dev, 1e-14);
        return GF_OK;
    }
    const int q = NV == 8 ? 0 : (NV == 16 ? 1 : (NV == 24 ? 2 : 3));
    const int b0 = g->nbc[0][q], b1 = g->nbc[1][q], b2 = g->nbc[2][q];
    // each pass sums its block rows in its last block to arrive (fp64_finish): h1, h2, ||w||^2;
    // the last pass's last block then runs the Arnoldi tail
    LAUNCH(g, b0, gf::RED_THREADS, gf::cgs_dots_kernel<NV>, g->V, ld, nv, w, n, g->partial, g->st, g->st,
           g->cgsticket);
    if (g->half_sm)
        LAUNCH(g, b1, 128, (gf::cgs_update_dots_kernel<NV, 128>), g->V, ld, nv, w, n, g->partial, g->st, g->st,
               g->cgsticket);
    else
        LAUNCH(g, b1, gf::RED_THREADS, gf::cgs_update_dots_kernel<NV>, g->V, ld, nv, w, n, g->partial, g->st, g->st,
               g->cgsticket);
    LAUNCH(g, b2, gf::RED_THREADS, gf::cgs_update_norm_kernel<NV>, g->V, ld, nv, w, n, g->partial, g->st, g->st,
           g->cgsticket, g->hist, j, NV, (volatile int*)g->host_status_dev, 1e-14);   // + the Arnoldi tail
    return GF_OK;
}

// CGS2 for step j with j + 1 > KRY_NV basis vectors: the passes of cgs2_step run over
// slices of KRY_NV vectors. Pass 1 dots every slice against w (and ||w||^2 for the
// breakdown test into h1[KRY_MMAX + 1]); w -= V h1 slice by slice; the second dots into
// h2; w -= V h2 slice by slice, the last slice also forming ||w||^2. outer == 2 runs
// the double-float passes on Vd and wd, otherwise FP64 on V and w.
int cgs2_step_long(gf_grid* g, int j, double* w, int outer)
{
    constexpr int NS = gf::KRY_NV;
    const long long n = g->ndof, ld = g->ldk;
    const int nv = j + 1, slices = (nv + NS - 1) / NS;
    double* h1 = g->st->h1;   // device addresses of the state's slots
    double* h2 = g->st->h2;
    const gf::KState* cst = g->st;
    if (outer == 2) {
        float2* wd = g->Vd + (long long)(j + 1) * ld;
        for (int pass = 0; pass < 2; ++pass) {
            double* h = pass == 0 ? h1 : h2;
            for (int c = 0; c < slices; ++c) {
                const int off = c * NS, cnt = std::min(NS, nv - off);
                double* wwdst = (pass == 0 && c == 0) ? h1 + gf::KRY_MMAX + 1 : nullptr;
                LAUNCH(g, g->nbd_k[0][2], gf::DD_THREADS, gf::ddgs_slice_dots_kernel<NS>,
                       (const float2*)(g->Vd + off * ld), ld, cnt, (const float2*)wd, n, g->pdd, cst, g->ddticket,
                       h + off, wwdst);
            }
            for (int c = 0; c < slices; ++c) {
                const int off = c * NS, cnt = std::min(NS, nv - off);
                double* wwdst = (pass == 1 && c == slices - 1) ? &g->st->ww : nullptr;
                LAUNCH(g, g->nbd_k[2][2], gf::DD_THREADS, gf::ddgs_slice_update_kernel<NS>,
                       (const float2*)(g->Vd + off * ld), ld, cnt, wd, n, g->pdd, cst, g->ddticket,
                       (const double*)(h + off), wwdst);
            }
        }
        LAUNCH(g, 1, 32, gf::arnoldi_tail_kernel, g->st, g->hist, j, gf::KRY_MMAX + 1, g->host_status_dev, 1e-14);
        return GF_OK;
    }
    for (int pass = 0; pass < 2; ++pass) {
        double* h = pass == 0 ? h1 : h2;
        for (int c = 0; c < slices; ++c) {
            const int off = c * NS, cnt = std::min(NS, nv - off);
            LAUNCH(g, g->nbr, gf::RED_THREADS, gf::cgs_dots_kernel<NS>, (const double*)(g->V + off * ld), ld, cnt,
                   (const double*)w, n, g->partial, (const gf::KState*)g->st, (gf::KState*)nullptr,
                   (unsigned int*)nullptr);
            LAUNCH(g, 1, 32 * 32, gf::reduce_slice_kernel, (const double*)g->partial, g->nbr, NS + 1, 0, cnt, h + off,
                   (const gf::KState*)g->st);
            if (pass == 0 && c == 0)
                LAUNCH(g, 1, 32, gf::reduce_slice_kernel, (const double*)g->partial, g->nbr, NS + 1, NS, 1,
                       h1 + gf::KRY_MMAX + 1, (const gf::KState*)g->st);
        }
        for (int c = 0; c < slices; ++c) {
            const int off = c * NS, cnt = std::min(NS, nv - off);
            double* part = (pass == 1 && c == slices - 1) ? g->partial : nullptr;
            LAUNCH(g, g->nbr, gf::RED_THREADS, gf::cgs_slice_update_kernel<NS>, (const double*)(g->V + off * ld), ld,
                   cnt, w, n, (const double*)(h + off), part, (const gf::KState*)g->st);
        }
    }
    LAUNCH(g, 1, 32, gf::reduce_slice_kernel, (const double*)g->partial, g->nbr, 1, 0, 1, &g->st->ww,
           (const gf::KState*)g->st);
    LAUNCH(g, 1, 32, gf::arnoldi_tail_kernel, g->st, g->hist, j, gf::KRY_MMAX + 1, g->host_status_dev, 1e-14);
    return GF_OK;
}

int arnoldi_step(gf_grid* g, int j, const gf_solve_opts* o)
{
    const long long ld = g->ldk;
    double* vj = g->V + (long long)j * ld;
    double* zj = g->Z + (long long)j * ld;
    double* w = g->V + (long long)(j + 1) * ld;
    const int* halt = &g->st->status;
    RET(vcycle_dispatch(g, vj, zj, o->prec, o->nu1, o->nu2, o->omega, halt, o->smoother, o->ls_ratio,
                        o->fine_steps));
    if (o->outer == 2) RET(applyKsplit_dd(g, zj, g->Vd + (long long)(j + 1) * ld, halt));
    else RET(applyOuter(g, zj, w, halt, o->outer));
    if (j + 1 > gf::KRY_NV) RET(cgs2_step_long(g, j, w, o->outer));
    else switch (pick_nv(j + 1, o->outer == 2)) {
        case 8: RET(cgs2_step<8>(g, j, w, o->outer)); break;
        case 16: RET(cgs2_step<16>(g, j, w, o->outer)); break;
        case 24: RET(cgs2_step<24>(g, j, w, o->outer)); break;
        default: RET(cgs2_step<32>(g, j, w, o->outer)); break;
    }
    if (o->outer == 2)
        LAUNCH(g, 2 * g->sms, 256, gf::ddgs_scale_kernel, g->Vd + (long long)(j + 1) * ld, w, g->ndof, g->st);
    else
        LAUNCH(g, stream_blocks(g, g->ndof), 256, gf::scale_kernel, w, g->ndof, g->st, 1);
    return GF_OK;
}

// r = M f - K x into V_0, ||r||, ||Mf||, history[k], g = beta e1, V_0 /= beta.
int cycle_start(gf_grid* g, const double* f, const double* x, bool x_zero, bool first, int outer)
{
    double* v0 = g->V;
    const int* skip = &g->st->skip;
    if (!x_zero) RET(applyOuter(g, x, v0, skip, outer));
    LAUNCH(g, g->nbr, gf::RED_THREADS, gf::residual_norms_kernel, f, v0, v0, g->ndof, g->nx + 1, g->partial,
           x_zero ? 1 : 0, skip, (const uint8_t*)g->lv[0].fix);
    LAUNCH(g, 1, 64, gf::reduce_partials_kernel, g->partial, g->nbr, 2, 2, g->st, 0, 0);
    LAUNCH(g, 1, 32, gf::cycle_start_tail_kernel, g->st, g->hist, g->host_status_dev, first ? 1 : 0);
    if (outer == 2)
        LAUNCH(g, 2 * g->sms, 256, gf::ddgs_scale_fp64_kernel, v0, g->Vd, g->ndof, g->st);
    else
        LAUNCH(g, stream_blocks(g, g->ndof), 256, gf::scale_kernel, v0, g->ndof, g->st, 1);
    return GF_OK;
}

// Replay the captured graph of Arnoldi step j (capturing it on first use).
int run_step(gf_grid* g, int j, const gf_solve_opts* o)
{
    if (!g->use_graphs) return arnoldi_step(g, j, o);
    if (g->gkey_prec != o->prec || g->gkey_nu1 != o->nu1 || g->gkey_nu2 != o->nu2 || g->gkey_omega != o->omega ||
        g->gkey_outer != o->outer || g->gkey_smoother != o->smoother || g->gkey_ls != o->ls_ratio ||
        g->gkey_fine != o->fine_steps || g->gkey_coarse != o->coarse_steps) {
        drop_graphs(g);
        g->gkey_coarse = o->coarse_steps;
        g->gkey_ls = o->ls_ratio;
        g->gkey_fine = o->fine_steps;
        g->gkey_outer = o->outer;
        g->gkey_smoother = o->smoother;
        g->gkey_prec = o->prec;
        g->gkey_nu1 = o->nu1;
        g->gkey_nu2 = o->nu2;
        g->gkey_omega = o->omega;
    }
    if (!g->step_exec[j]) {
        const gf_stats before = g->stats;
        CK(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
        g->cur_stream = g->cap_stream;
        const int r = arnoldi_step(g, j, o);
        g->cur_stream = g->stream;
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(g->cap_stream, &graph);
        if (r != GF_OK) {
            if (graph) cudaGraphDestroy(graph);
            return r;
        }
        CK(e);
        const cudaError_t ei = cudaGraphInstantiate(&g->step_exec[j], graph, 0);
        cudaGraphDestroy(graph);
        CK(ei);
        g->step_nodes[j] = g->stats.kernel_launches - before.kernel_launches;
        g->stats = before;
    }
    CK(cudaGraphLaunch(g->step_exec[j], g->stream));
    g->stats.kernel_launches += g->step_nodes[j];
    g->stats.apply_K_fp64 += 1;
    g->stats.vcycles += 1;
    return GF_OK;
}

// Optional pause after `at` Arnoldi steps: the probe of Algorithm 1 read off the
// running solve. Because the solver is deterministic, the first `at` steps of the
// selected solve at rho0 are the probe's steps, bit for bit.
// Optional true-residual checks during the first `upto` steps (every `every` steps):
// the iterate of the step (cycle-start iterate plus Z y of the current triangular
// system) and its FP64 guard residual, beside the projected estimate of the step.
struct ProbeHook {
    int at = -1;
    const gf_policy* pol = nullptr;
    std::function<int(double, double, int*)> decide;   // -> first floor index (0 = rho0)
    bool decided = false, escalate = false;
    int first = 0, err = GF_OK;
    double r50 = 0.0, r100 = 0.0;
    int every = 0, upto = 0, n = 0;
    double ratio = 10.0;
    int ck[GF_MAX_TRUE_CHECKS];
    double est[GF_MAX_TRUE_CHECKS], eta[GF_MAX_TRUE_CHECKS];
    bool fired = false;
};

int guard_impl(gf_grid* g, const double* f, const double* u, double* eta);

int true_check(gf_grid* g, const double* f, const double* u, ProbeHook* hook, int k)
{
    if (!g->ckx) RET(allocT(&g->ckx, g->ndof));
    LAUNCH(g, 1, 1, gf::backsolve_kernel, g->st);   // y of the current J columns (recomputed at the cycle end)
    CK(cudaMemcpyAsync(g->ckx, u, sizeof(double) * g->ndof, cudaMemcpyDeviceToDevice, g->stream));
    LAUNCH(g, 2 * g->sms, 256, gf::update_x_kernel, g->ckx, g->Z, g->ldk, g->ndof, g->st);
    double eta = 0.0, est = 0.0;
    RET(guard_impl(g, f, g->ckx, &eta));
    CK(cudaMemcpy(&est, g->hist + k, sizeof(double), cudaMemcpyDeviceToHost));
    hook->ck[hook->n] = k;
    hook->est[hook->n] = est;
    hook->eta[hook->n] = eta;
    hook->n++;
    if (eta > hook->ratio * est) hook->fired = true;
    return GF_OK;
}

int solve_impl(gf_grid* g, const double* f, double* u, const gf_solve_opts* o, gf_solve_info* info,
               bool x_zero, double* host_hist, ProbeHook* hook = nullptr)
{
    const int m = o->restart;
    RET(ensure_krylov(g, m, o->kmax, o->outer));
    if (o->smoother == 1) RET(ensure_cheb(g, o->prec));
    if (o->ls_ratio > 0.0) RET(ensure_ls(g));
    RET(set_coarse_steps(g, o));
    const int NX0 = g->nx + 1;
    // fixed entries of u are written as 0
    LAUNCH(g, 2 * g->sms, 256, (gf::masked_convert_kernel<double, double>), u, u, g->ndof, NX0, nullptr, (const uint8_t*)g->lv[0].fix);
    LAUNCH(g, 1, 1, init_state_kernel, g->st, o->kmax, m, o->tol);
    *g->host_status = gf::KS_RUN;
    bool first = true, aborted = false;
    long long launched = 0;
    HostState hs{};
    for (;;) {
        RET(cycle_start(g, f, u, x_zero && first, first, o->outer));
        first = false;
        x_zero = false;
        CK(cudaStreamSynchronize(g->stream));
        if (*(volatile int*)g->host_status != gf::KS_RUN) break;
        for (int j = 0; j < m; ++j) {
            RET(run_step(g, j, o));
            ++launched;
            CK(cudaEventRecord(g->ev[j % 3], g->stream));
            if (hook && hook->every > 0 && launched % hook->every == 0 && launched <= hook->upto &&
                hook->n < GF_MAX_TRUE_CHECKS) {
                RET(read_state(g, &hs));
                if (hs.status == gf::KS_RUN) RET(true_check(g, f, u, hook, (int)launched));
            }
            if (hook && !hook->decided && launched == hook->at) {
                RET(read_state(g, &hs));
                if (hs.status == gf::KS_RUN) {
                    double h2[2];
                    const int ia = std::min(hook->pol->checkpoint_a, hs.k), ib = std::min(hook->pol->checkpoint_b, hs.k);
                    CK(cudaMemcpy(&h2[0], g->hist + ia, sizeof(double), cudaMemcpyDeviceToHost));
                    CK(cudaMemcpy(&h2[1], g->hist + ib, sizeof(double), cudaMemcpyDeviceToHost));
                    hook->decided = true;
                    hook->r50 = h2[0];
                    hook->r100 = h2[1];
                    RET(hook->decide(h2[0], h2[1], &hook->first));
                    hook->escalate = hook->first > 0;
                    if (hook->escalate) {
                        aborted = true;
                        break;
                    }
                }
            }
            if (j >= 1) {
                CK(cudaEventSynchronize(g->ev[(j - 1) % 3]));
                if (*(volatile int*)g->host_status != gf::KS_RUN) break;
            }
        }
        if (aborted) break;
        LAUNCH(g, 1, 1, gf::backsolve_kernel, g->st);
        LAUNCH(g, 2 * g->sms, 256, gf::update_x_kernel, u, g->Z, g->ldk, g->ndof, g->st);
        RET(read_state(g, &hs));
        if (hs.status != gf::KS_RUN) break;
    }
    RET(read_state(g, &hs));
    if (info) {
        info->iters = hs.k;
        info->flag = hs.flag;
        double est = 0.0;
        CK(cudaMemcpy(&est, g->hist + hs.k, sizeof(double), cudaMemcpyDeviceToHost));
        info->stop_estimate = est;
    }
    if (host_hist) CK(cudaMemcpy(host_hist, g->hist, sizeof(double) * (hs.k + 1), cudaMemcpyDeviceToHost));
    return GF_OK;
}

int validate_opts(const gf_solve_opts* o)
{
    if (!o) return set_err(GF_ERR_ARG, "null opts");
    if (o->restart < 1 || o->restart > gf::KRY_MMAX) return set_err(GF_ERR_ARG, "restart must be in [1, 300]");
    if (o->kmax < 0) return set_err(GF_ERR_ARG, "kmax < 0");
    if (!(o->tol >= 0.0)) return set_err(GF_ERR_ARG, "tol must be >= 0");
    if (o->prec != GF_FP64 && o->prec != GF_MIXED) return set_err(GF_ERR_ARG, "prec");
    if (o->nu1 < 1 || o->nu2 < 1 || o->nu1 > 16 || o->nu2 > 16) return set_err(GF_ERR_ARG, "nu1/nu2 in [1,16]");
    if (!(o->omega > 0.0 && o->omega < 2.0)) return set_err(GF_ERR_ARG, "omega in (0,2)");
    if (o->outer < 0 || o->outer > 2)
        return set_err(GF_ERR_ARG, "outer must be 0 (FP64), 1 (split K*u) or 2 (split K*u, double-float CGS2)");
    if (o->smoother != 0 && o->smoother != 1) return set_err(GF_ERR_ARG, "smoother must be 0 (Jacobi) or 1 (Chebyshev)");
    if (!(o->ls_ratio >= 0.0 && std::isfinite(o->ls_ratio))) return set_err(GF_ERR_ARG, "ls_ratio must be finite and >= 0");
    if (o->ls_ratio > 0.0 && o->smoother != 0) return set_err(GF_ERR_ARG, "ls_ratio > 0 needs smoother 0");
    if (o->fine_steps < 0 || o->fine_steps > gf::FC_MAX) return set_err(GF_ERR_ARG, "fine_steps in [0, 32]");
    if (o->coarse_steps < 0 || o->coarse_steps > gf::FC_MAX) return set_err(GF_ERR_ARG, "coarse_steps in [0, 32]");
    return GF_OK;
}

// The bridge geometry (per-node fixed components) runs the default solver: native FP64
// Krylov, node-block Jacobi smoothing, rediscretised coarse levels, no adaptive components.
int validate_geom(const gf_grid* g, const gf_solve_opts* o)
{
    if (g->geom == GF_GEOM_CANTILEVER) return GF_OK;
    if (o->outer != 0 || o->smoother != 0 || o->ls_ratio > 0.0 || o->fine_steps != 0 || o->coarse_steps != 0)
        return set_err(GF_ERR_ARG, "the bridge geometry takes outer 0, smoother 0 and no adaptive components");
    return GF_OK;
}

int guard_impl(gf_grid* g, const double* f, const double* u, double* eta)
{
    RET(applyK64(g, u, g->work, nullptr));
    LAUNCH(g, g->nbr, gf::RED_THREADS, gf::residual_norms_kernel, f, g->work, (double*)nullptr, g->ndof,
           g->nx + 1, g->partial, 0, (const int*)nullptr, (const uint8_t*)g->lv[0].fix);
    LAUNCH(g, 1, 64, gf::reduce_partials_kernel, g->partial, g->nbr, 2, 2, g->gst, 0, 0);
    double h[2];
    CK(cudaMemcpyAsync(h, g->gst->h1, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (!std::isfinite(h[0]) || !std::isfinite(h[1])) return set_err(GF_ERR_NONFINITE, "non-finite residual");
    if (h[1] == 0.0) return set_err(GF_ERR_ARG, "f is zero on the free DOFs");
    *eta = std::sqrt(h[0]) / std::sqrt(h[1]);
    return GF_OK;
}

int filter_radius_cells(double r_min) { return (int)std::ceil(r_min) - 1; }

int filter_impl(gf_grid* g, const double* x, double* out, double r_min, bool adjoint)
{
    const int R = filter_radius_cells(r_min);
    if (adjoint)
        LAUNCH(g, nblk(g->nel), 256, gf::hat_filter_kernel<true>, x, out, g->lv[0].dims(), r_min, R);
    else
        LAUNCH(g, nblk(g->nel), 256, gf::hat_filter_kernel<false>, x, out, g->lv[0].dims(), r_min, R);
    return GF_OK;
}

int ensure_oc(gf_grid* g)
{
    if (g->oc_rho) return GF_OK;
    RET(allocT(&g->oc_rho, g->nel));
    RET(allocT(&g->oc_dc, g->nel));
    RET(allocT(&g->oc_dcx, g->nel));
    RET(allocT(&g->oc_dvx, g->nel));
    RET(allocT(&g->oc_ones, g->nel));
    RET(allocT(&g->oc_st, 1));
    std::vector<double> ones((size_t)g->nel, 1.0);
    CK(cudaMemcpy(g->oc_ones, ones.data(), sizeof(double) * g->nel, cudaMemcpyHostToDevice));
    return GF_OK;
}

int oc_update_impl(gf_grid* g, const double* x, const double* dc, const double* dv, double volfrac, double move,
                   double* xnew)
{
    RET(ensure_oc(g));
    const long long n = g->nel;
    const int nb = (int)std::min<long long>(2LL * g->sms, std::max<long long>(1, (n + 1023) / 1024));
    const double tol = 1e-3;
    const int max_iters = 200;
    LAUNCH(g, 1, 1, gf::oc_init_kernel, g->oc_st);
    // every bisection iteration is two launches; iterations after the stop test early-exit
    for (int it = 0; it < max_iters; ++it) {
        LAUNCH(g, nb, 256, gf::oc_partial_kernel, x, dc, dv, n, move, tol, g->oc_st, g->partial);
        LAUNCH(g, 1, 32, gf::oc_bisect_kernel, (const double*)g->partial, nb, n, volfrac, tol, max_iters, g->oc_st);
        if ((it & 15) == 15) {
            int done = 0;
            CK(cudaMemcpyAsync(&done, &g->oc_st->done, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
            CK(cudaStreamSynchronize(g->stream));
            if (done) break;
        }
    }
    LAUNCH(g, nblk(n), 256, gf::oc_apply_kernel, x, dc, dv, xnew, n, move, (const gf::OCState*)g->oc_st);
    return GF_OK;
}

int dot_impl(gf_grid* g, const double* a, const double* b, long long n, double* out)
{
    const int nb = (int)std::min<long long>(2LL * g->sms, std::max<long long>(1, (n + 1023) / 1024));
    LAUNCH(g, nb, 256, gf::dot_partial_kernel, a, b, n, g->partial);
    std::vector<double> part((size_t)nb);
    CK(cudaMemcpyAsync(part.data(), g->partial, sizeof(double) * nb, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    double s = 0.0;
    for (int i = 0; i < nb; ++i) s += part[i];   // fixed order
    *out = s;
    return GF_OK;
}

// fp16 bit pattern of a small integer (|v| <= 2048, exact)
unsigned short half_bits_of_int(int v)
{
    if (v == 0) return 0;
    const unsigned short sg = v < 0 ? 0x8000 : 0;
    const int a = v < 0 ? -v : v;
    int e = 0;
    while ((a >> (e + 1)) != 0) ++e;                       // a in [2^e, 2^(e+1))
    const int mant = (a << (10 - e)) & 0x3FF;              // exact: a has <= 11 significant bits
    return (unsigned short)(sg | ((e + 15) << 10) | mant);
}

// M' (24x24, row/col q' = comp * 8 + a', a' = x + 2y + 4z) as the m16n8k16 B fragments
// of each lane: for output component t, K-step 0 holds columns comp 0 | comp 1, K-step
// 1 holds comp 2 | zero padding. Lane (g = lane/4, c = lane%4) holds rows k = 2c, 2c+1
// (and 2c+8, 2c+9) of column n = g.
// B fragments of stencil_tc32_kernel: lane (g, cq) of output tile t and K-step c holds
// M[(a' = g, t)][(a' = cq, c)] and M[(a' = g, t)][(a' = cq + 4, c)] (a' = x + 2y + 4z;
// K0 = s M, integers exact in TF32).
void build_s3_bfrag(const gf::MParam& M, gf::S3BFrag* B)
{
    auto li = [](int ap) { return gf::local_index(ap & 1, (ap >> 1) & 1, ap >> 2); };
    for (int lane = 0; lane < 32; ++lane) {
        const int g = lane >> 2, cq = lane & 3;
        for (int t = 0; t < 3; ++t)
            for (int c = 0; c < 3; ++c)
                for (int r = 0; r < 2; ++r)
                    B->w[(t * 3 + c) * 2 + r][lane] = M.m[(3 * li(g) + t) * 24 + 3 * li(cq + 4 * r) + c];
    }
}

// dynamic shared memory of every stencil_tc32_kernel instantiation the V-cycles launch
template <int MODE, typename BT, typename OT>
bool stc_smem_attr()
{
    return cudaFuncSetAttribute(gf::stencil_tc32_kernel<MODE, BT, OT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(gf::S3Smem)) == cudaSuccess;
}
bool stc_smem_attrs()
{
    return stc_smem_attr<gf::ST_APPLY, float, float>() && stc_smem_attr<gf::ST_RESID, float, float>() &&
           stc_smem_attr<gf::ST_SWEEP, float, float>() && stc_smem_attr<gf::ST_RESID, double, float>() &&
           stc_smem_attr<gf::ST_SWEEP, double, float>() && stc_smem_attr<gf::ST_SWEEP, double, double>() &&
           stc_smem_attr<gf::ST_SWEEP, float, double>();
}

// Node layers per CTA of stencil_tc32_kernel on a level: the fewest element layers per
// SM slot over whole waves (each CTA computes cz + 1 element layers for cz node layers).
int stc_layers(const Level& L, int slots)
{
    const long long txy = (long long)((L.nx + 1 + gf::S3_NX - 1) / gf::S3_NX) * ((L.ny + 1 + gf::S3_NY - 1) / gf::S3_NY);
    const int NZ = L.nz + 1;
    int best = 4;
    long long best_cost = -1;
    for (int cz = 4; cz <= 16; ++cz) {
        const long long ctas = txy * ((NZ + cz - 1) / cz);
        const long long cost = ((ctas + slots - 1) / slots) * (cz + 1);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = cz;
        }
    }
    return best;
}

void build_tc_bfrag(const gf::MParam& M, gf::TcBFrag* B)
{
    auto orig = [](int qp) {   // original DOF index 3 a + comp of q'
        const int comp = qp / 8, ap = qp % 8;
        return 3 * gf::local_index(ap & 1, (ap >> 1) & 1, ap >> 2) + comp;
    };
    auto mp = [&](int ip, int jp) -> unsigned int {
        if (ip >= 24 || jp >= 24) return 0u;
        return half_bits_of_int((int)M.m[orig(ip) * 24 + orig(jp)]);
    };
    for (int lane = 0; lane < 32; ++lane) {
        const int g = lane >> 2, c = lane & 3;
        for (int t = 0; t < 3; ++t) {
            const int ip = 8 * t + g;
            for (int ks = 0; ks < 2; ++ks)
                for (int r = 0; r < 2; ++r) {
                    const int j0 = 16 * ks + 8 * r + 2 * c;
                    B->w[4 * t + 2 * ks + r][lane] = mp(ip, j0) | (mp(ip, j0 + 1) << 16);
                }
        }
    }
}

}  // namespace

// ====================================================================== C ABI ====
extern "C" {

const char* gf_last_error(void) { return g_err.c_str(); }

}  // extern "C"
namespace {
int modal_autotune(gf_grid* g);
int modal_default_plan(gf_grid* g);
int cgs_grids(gf_grid* g, long long* partial_rows);
}
extern "C" {
int gf_create_grid(int nx, int ny, int nz, double h, double E0, double nu, int levels, void* stream,
                   gf_grid** out)
{
    if (!out) return set_err(GF_ERR_ARG, "null out");
    *out = nullptr;
    if (nx < 1 || ny < 2 || nz < 2 || (ny & 1) || (nz & 1)) return set_err(GF_ERR_ARG, "need nx>=1, even ny,nz >= 2");
    if (levels < 1 || levels > 8) return set_err(GF_ERR_ARG, "levels in [1,8]");
    const int div = 1 << (levels - 1);
    if (nx % div || ny % div || nz % div) return set_err(GF_ERR_ARG, "grid not divisible by 2^(levels-1)");
    if (!(h > 0) || !(E0 > 0) || !(nu > -1.0 && nu < 0.5)) return set_err(GF_ERR_ARG, "h, E0 > 0, nu in (-1,0.5)");
    const long long cn = 3LL * (nx / div + 1) * (ny / div + 1) * (nz / div + 1);
    if (cn > 8192) return set_err(GF_ERR_ARG, "coarsest level above 8192 DOFs: add levels");
    gf_grid* g = new gf_grid();
    g->nx = nx; g->ny = ny; g->nz = nz; g->L = levels;
    g->h = h; g->E0 = E0; g->nu = nu;
    g->stream = (cudaStream_t)stream;
    g->cur_stream = g->stream;
    auto fail = [&](int code) { gf_destroy_grid(g); return code; };
    if (cudaGetDevice(&g->device) != cudaSuccess) return fail(set_err(GF_ERR_CUDA, "cudaGetDevice"));
    if (cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess)
        return fail(set_err(GF_ERR_CUDA, "SM count"));
    g->nodes = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    if (g->nodes >= (1LL << 31)) return fail(set_err(GF_ERR_ARG, "grid of 2^31 nodes or more"));
    g->ndof = 3 * g->nodes;
    g->nel = (long long)nx * ny * nz;
    double K[576];
    build_k0(E0, nu, K);
    for (int q = 0; q < 576; ++q) {
        g->K0d.k[q] = K[q];
        g->K0f.k[q] = (float)K[q];
    }
    g->Kmodal = gf::modal_coef(E0, nu);
    for (int q = 0; q < 6; ++q) g->Kmodal32.diag[q] = (float)g->Kmodal.diag[q];
    for (int q = 0; q < 4; ++q) g->Kmodal32.cross[q] = (float)g->Kmodal.cross[q];
    for (int a = 0; a < 8; ++a) {
        const int r0 = 3 * a;
        g->Kmodal32.blk[a][0] = (float)K[(r0 + 0) * 24 + r0 + 0];
        g->Kmodal32.blk[a][1] = (float)K[(r0 + 1) * 24 + r0 + 1];
        g->Kmodal32.blk[a][2] = (float)K[(r0 + 2) * 24 + r0 + 2];
        g->Kmodal32.blk[a][3] = (float)K[(r0 + 0) * 24 + r0 + 1];
        g->Kmodal32.blk[a][4] = (float)K[(r0 + 0) * 24 + r0 + 2];
        g->Kmodal32.blk[a][5] = (float)K[(r0 + 1) * 24 + r0 + 2];
    }
    {
        const char* e = getenv("GF_MODAL_F32");
        g->modal_f32 = !(e && e[0] == '0');
    }
    {
        const char* e = getenv("GF_SYM_GJ");
        g->sym_gj = !(e && e[0] == '0');
        const char* l = getenv("GF_COARSE_LDL");
        g->coarse_ldl = !(l && l[0] == '0') && g->sym_gj;
    }
    {   // modal FP64 K*u (GF_MODAL=0: the dense node stencil)
        const char* e = getenv("GF_MODAL");
        if (!(e && e[0] == '0')) {
            const int rp = modal_default_plan(g);
            if (rp != GF_OK) return fail(rp);
            const gf::GridDims d0{nx, ny, nz, nullptr};   // the fine level (the levels come later)
            const long long side = std::max(std::max(gf::modal_side(d0, 32, 16).entries(d0),
                                                     gf::modal_side(d0, 16, 32).entries(d0)),
                                            gf::modal_side(d0, 16, 16).entries(d0));
            if (alloc((void**)&g->modal_es, sizeof(double) * 9 * (size_t)g->nel) != GF_OK ||
                alloc((void**)&g->modal_side, sizeof(double) * 12 * (size_t)side) != GF_OK)
                return fail(GF_ERR_OOM);
        }
    }
    for (int a = 0; a < 8; ++a)
        for (int bl = 0; bl < 8; ++bl)
            for (int c = 0; c < 3; ++c) {
                g->K0p.p[a][bl][c] = make_float2(g->K0f.k[(3 * a + 0) * 24 + 3 * bl + c], g->K0f.k[(3 * a + 1) * 24 + 3 * bl + c]);
                g->K0p.s[a][bl][c] = g->K0f.k[(3 * a + 2) * 24 + 3 * bl + c];
            }
    {   // paired FMAs in the FP32 node stencil (default; GF_F32X2=0 selects the scalar kernel):
        // 14.6 -> 12.5 us per fine-level launch at 96x48x48, 76.1 -> 67.9 us at 192x96x96
        // 128-thread blocks on levels below two 256-thread blocks per SM (GF_COARSE_TPB=0:
        // 256 as before, or 32/64): 96x48x48 V-cycle 191.6 -> 184-189 us, bit-identical
        const char* cf = getenv("GF_COARSE_FUSED");
        g->ck_fused = !(cf && cf[0] == '0');
        const char* ct = getenv("GF_COARSE_TPB");
        if (ct) g->ctpb = atoi(ct);
        if (g->ctpb != 0 && g->ctpb != 32 && g->ctpb != 64 && g->ctpb != 128) g->ctpb = 128;
        const char* e = getenv("GF_F32X2");
        g->f32x2 = !(e && e[0] == '0');
    }
    // K0 = s * M with integer M. The 24-term digit products stay exact in FP32 when
    // 24 |M| (2^12 - 1) < 2^24, i.e. |M| <= 170 (88 for nu = 0.3).
    for (int kk = 1; kk <= 170 && !g->has_split; ++kk) {
        const double sc = K[0] / kk;
        bool ok = true;
        for (int q = 0; q < 576 && ok; ++q) {
            const double mq = K[q] / sc, rq = std::nearbyint(mq);
            ok = std::fabs(mq - rq) <= 1e-9 * std::max(1.0, std::fabs(mq)) && std::fabs(rq) <= 170.0;
        }
        if (ok) {
            g->has_split = true;
            g->s_split = sc;
            for (int q = 0; q < 576; ++q) g->Msplit.m[q] = (float)std::nearbyint(K[q] / sc);
        }
    }
    if (g->has_split) {
        gf::TcBFrag hb;
        build_tc_bfrag(g->Msplit, &hb);
        if (int r0 = allocT(&g->Btc, 1)) return fail(r0);
        if (cudaMemcpy(g->Btc, &hb, sizeof(hb), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(set_err(GF_ERR_CUDA, "B fragments of the tensor-core split kernel"));
        // tensor cores when the grid gives every SM a CTA (fewer CTAs leave the kernel
        // latency-bound and the CUDA-core one is faster: 35 vs 13 us at 16x8x8, 8 CTAs);
        // GF_SPLIT_TC=1 / 0 forces either
        const dim3 tg = split_tc_grid(g);
        const long long ctas = (long long)tg.x * tg.y * tg.z;
        const char* e = getenv("GF_SPLIT_TC");
        g->split_tc = e ? (e[0] != '0') : (ctas >= g->sms);
        if (g->split_tc &&
            (cudaFuncSetAttribute(gf::apply_split_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sizeof(gf::TcSmem)) != cudaSuccess ||
             cudaFuncSetAttribute(gf::apply_split_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sizeof(gf::TcSmem)) != cudaSuccess))
            return fail(set_err(GF_ERR_CUDA, "shared-memory size of the tensor-core split kernel"));
    } else {
        g->split_tc = false;
    }
    if (cudaFuncSetAttribute(gf::coarse_fgmres_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             gf::CK_SMEM_MAX) != cudaSuccess ||
        cudaFuncSetAttribute(gf::coarse_fgmres_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             gf::CK_SMEM_MAX) != cudaSuccess)
        return fail(set_err(GF_ERR_CUDA, "shared-memory size of the coarse-level Krylov kernel"));
    for (int l = 0; l < levels; ++l) {
        Level L;
        L.nx = nx >> l; L.ny = ny >> l; L.nz = nz >> l;
        L.h = h * (double)(1 << l);
        L.nodes = (long long)(L.nx + 1) * (L.ny + 1) * (L.nz + 1);
        L.ndof = 3 * L.nodes;
        L.nel = (long long)L.nx * L.ny * L.nz;
        int r = GF_OK;
        if ((r = allocT(&L.E64, L.nel)) || (r = allocT(&L.E32, L.nel)) ||
            (r = allocT(&L.b64, L.ndof)) || (r = allocT(&L.x64, L.ndof)) || (r = allocT(&L.t64, L.ndof)) ||
            (r = allocT(&L.r64, L.ndof)) || (r = allocT(&L.b32, L.ndof)) || (r = allocT(&L.x32, L.ndof)) ||
            (r = allocT(&L.t32, L.ndof)) || (r = allocT(&L.r32, L.ndof))) {
            g->lv.push_back(L);
            return fail(r);
        }
        g->lv.push_back(L);
    }
    g->nc = (int)g->lv.back().ndof;
    // FP32 level stencils on the tensor cores (opt-in, GF_STENCIL_TC=1, when K0 has its
    // small-integer form): parity-tested, but slower than the CUDA-core kernel on B300
    // (17.0 vs 14.4 us at 96x48x48, 86 vs 74 us at 192x96x96; each element layer of a CTA
    // spends ~1.8k cycles on TF32 mma.sync and ~400 B of shared-memory traffic per element)
    const char* stc_env = getenv("GF_STENCIL_TC");
    if (g->has_split && stc_env && stc_env[0] != '0') {
        gf::S3BFrag hb;
        build_s3_bfrag(g->Msplit, &hb);
        int occ = 0;
        if (int r0 = allocT(&g->B3, 1)) return fail(r0);
        if (cudaMemcpy(g->B3, &hb, sizeof(hb), cudaMemcpyHostToDevice) != cudaSuccess || !stc_smem_attrs() ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gf::stencil_tc32_kernel<gf::ST_SWEEP, double, float>,
                                                          gf::S3_THREADS, sizeof(gf::S3Smem)) != cudaSuccess ||
            occ < 1)
            return fail(set_err(GF_ERR_CUDA, "set-up of the tensor-core stencil"));
        for (int l = 0; l < levels; ++l) g->stc_cz[l] = stc_layers(g->lv[l], occ * g->sms);
    }
    // Opt-in (GF_VC_CLUSTER=<max nodes>): the cluster kernel takes the levels from the
    // first one (>= 1) with at most that many nodes, when at least one smoothing level
    // lies above the coarsest. Off by default: in graph-replayed solves the per-level
    // launches cost ~2 us each, and 8 SMs run the stages no faster than that.
    if (const char* e = getenv("GF_VC_CLUSTER")) {
        const long long maxn = atoll(e);
        for (int l = 1; maxn > 0 && l < levels - 1; ++l)
            if (g->lv[l].nodes <= maxn) {
                g->vc_l0 = l;
                break;
            }
    }
    int r = GF_OK;
    g->nbr = (int)std::min<long long>(2LL * g->sms, std::max<long long>(1, (g->ndof + 1023) / 1024));
    g->ldk = (g->ndof + 31) / 32 * 32;
    // the FP64 Gram-Schmidt passes' partial rows (both launch shapes: gf_set_sm_share) share
    // g->partial with the other reductions
    long long partial_rows = (long long)g->nbr * 40;
    for (int h = 1; h >= 0; --h) {
        long long rows = 0;
        g->half_sm = h != 0;
        cgs_grids(g, &rows);
        partial_rows = std::max(partial_rows, rows);
    }
    if ((r = allocT(&g->Ainv, (size_t)g->nc * g->nc)) || (r = allocT(&g->Agj, (size_t)g->nc * g->nc + 2 * gf::SGJ_B * gf::SGJ_B)) ||
        (r = allocT(&g->ldl_ws, (size_t)g->nc * (1 + gf::LDL_C) + gf::LDL_C * gf::LDL_C)) ||
        (r = allocT(&g->cpos, (size_t)g->nc)) || (r = allocT(&g->cidx, (size_t)g->nc + 1)) ||
        (r = allocT(&g->dflag, 4)) || (r = allocT(&g->rho64, g->nel)) ||
        (r = allocT(&g->rho16, g->nel)) || (r = allocT(&g->work, g->ndof)) ||
        (r = allocT(&g->partial, (size_t)partial_rows)) || (r = allocT(&g->st, 1)) || (r = allocT(&g->cgsticket, 1)) || (r = allocT(&g->gst, 1)) ||
        (r = allocT(&g->Edf, g->nel)))
        return fail(r);
    if (cudaMemset(g->cgsticket, 0, sizeof(unsigned int)) != cudaSuccess)
        return fail(set_err(GF_ERR_CUDA, "Gram-Schmidt ticket"));
    if (cudaHostAlloc((void**)&g->host_status, sizeof(int), cudaHostAllocMapped) != cudaSuccess)
        return fail(set_err(GF_ERR_CUDA, "cudaHostAlloc"));
    if (cudaHostGetDevicePointer((void**)&g->host_status_dev, g->host_status, 0) != cudaSuccess)
        return fail(set_err(GF_ERR_CUDA, "cudaHostGetDevicePointer"));
    for (int i = 0; i < 3; ++i)
        if (cudaEventCreateWithFlags(&g->ev[i], cudaEventDisableTiming) != cudaSuccess)
            return fail(set_err(GF_ERR_CUDA, "event"));
    if (cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(set_err(GF_ERR_CUDA, "capture stream"));
    g->cur_stream = g->stream;
    {
        const char* e = getenv("GF_GRAPHS");
        g->use_graphs = !(e && e[0] == '0');
    }
    if ((r = build_coarse_map(g)) != GF_OK) return fail(r);
    if (g->modal64_items && !getenv("GF_MODAL_CHUNK") && !getenv("GF_MODAL_BX"))
        if ((r = modal_autotune(g)) != GF_OK) return fail(r);
    *out = g;
    return GF_OK;
}

}  // extern "C"
namespace {
// Launch plans of the modal kernels by modal_plan's cost model alone: the FP32 fine level's
// (tiles overlapping by one column) and the FP64 K*u's (tiles apart), each the cheaper of
// the two full-SM tile shapes, or the 16 x 16 shape when the grid shares its SMs
// (half_sm). GF_MODAL_CHUNK=<planes> forces runs of that many node planes per CTA and
// GF_MODAL_BX=32/16 the tile shape (tests). Replaces the items held before.
int modal_default_plan(gf_grid* g)
{
    int per_sm = 0;
    if (!smem_opt_in<gf::apply_modal_kernel<32, 16, false>>(gf::modal_smem_bytes<double, 32, 16>()) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gf::apply_modal_kernel<32, 16>, gf::MODAL_THREADS,
                                                      gf::modal_smem_bytes<double, 32, 16>()) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const char* ch = getenv("GF_MODAL_CHUNK");
    const char* bxs = getenv("GF_MODAL_BX");
    const int forced = ch ? std::max(0, atoi(ch)) : 0;
    for (int f32 = 1; f32 >= 0; --f32) {
        double c32 = 0, c16 = 0;
        std::vector<int4> i32 = gf::modal_plan(g->nx, g->ny, g->nz, 32, 16, g->sms * per_sm, forced, &c32, f32);
        std::vector<int4> i16 =
            gf::modal_plan(g->nx, g->ny, g->nz, 16, g->half_sm ? 16 : 32, g->sms * per_sm, forced, &c16, f32);
        const bool use32 = !g->half_sm && (bxs ? atoi(bxs) == 32 : c32 <= c16);
        const std::vector<int4>& items = use32 ? i32 : i16;
        int4** dst = f32 ? &g->modal_items : &g->modal64_items;
        cudaFree(*dst);
        *dst = nullptr;
        (f32 ? g->modal_bx : g->modal64_bx) = use32 ? 32 : 16;
        (f32 ? g->modal_by : g->modal64_by) = use32 ? 16 : (g->half_sm ? 16 : 32);
        (f32 ? g->modal_n : g->modal64_n) = (int)items.size();
        RET(alloc((void**)dst, sizeof(int4) * items.size()));
        CK(cudaMemcpy(*dst, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
    }
    return GF_OK;
}

// Grids of the FP64 Gram-Schmidt passes: the blocks resident at once (one round), capped
// by 256-row tiles; half_sm: half of them, and the update-and-dots pass in 128-thread
// blocks, so that each leaves about half of an SM's registers to other streams.
// *partial_rows: the partial-sum rows the passes need.
int cgs_grids(gf_grid* g, long long* partial_rows)
{
    const void* kc[3][4] = {
        {(const void*)gf::cgs_dots_kernel<8>, (const void*)gf::cgs_dots_kernel<16>,
         (const void*)gf::cgs_dots_kernel<24>, (const void*)gf::cgs_dots_kernel<32>},
        {(const void*)gf::cgs_update_dots_kernel<8>, (const void*)gf::cgs_update_dots_kernel<16>,
         (const void*)gf::cgs_update_dots_kernel<24>, (const void*)gf::cgs_update_dots_kernel<32>},
        {(const void*)gf::cgs_update_norm_kernel<8>, (const void*)gf::cgs_update_norm_kernel<16>,
         (const void*)gf::cgs_update_norm_kernel<24>, (const void*)gf::cgs_update_norm_kernel<32>}};
    const void* kh[4] = {(const void*)gf::cgs_update_dots_kernel<8, 128>, (const void*)gf::cgs_update_dots_kernel<16, 128>,
                         (const void*)gf::cgs_update_dots_kernel<24, 128>, (const void*)gf::cgs_update_dots_kernel<32, 128>};
    const int nvq[4] = {8, 16, 24, 32};
    const long long tiles = std::max<long long>(1, (g->ndof + gf::RED_THREADS - 1) / gf::RED_THREADS);
    long long rows = 0;
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 4; ++q) {
            const bool h128 = g->half_sm && p == 1;
            int nb = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, h128 ? kh[q] : kc[p][q], h128 ? 128 : gf::RED_THREADS,
                                                              0) != cudaSuccess ||
                nb <= 0)
                nb = 2;
            if (g->half_sm) nb = std::max(1, nb / 2);
            g->nbc[p][q] = (int)std::min<long long>((long long)nb * g->sms, tiles);
            const int stride = p == 0 ? nvq[q] + 1 : (p == 1 ? nvq[q] : 1);
            rows = std::max(rows, (long long)g->nbc[p][q] * stride);
        }
    *partial_rows = rows;
    return GF_OK;
}

// Time the modal kernels under a few launch plans -- the cheapest ones by modal_plan's
// cost model over both tile shapes and several run lengths -- and keep the fastest, for
// the FP64 K*u (tiles apart, with its tile-boundary fix-up) and the FP32 fine-level sweep
// (tiles overlapping by one column) apart.
// The plan changes which CTA computes what, never the arithmetic of a node, so neither
// result depends on it. Runs once per grid, on zeroed
// level-0 scratch, on the grid's stream.
int modal_autotune(gf_grid* g)
{
    int per_sm = 0;
    if (!smem_opt_in<gf::apply_modal_kernel<32, 16, false>>(gf::modal_smem_bytes<double, 32, 16>()) ||
        !smem_opt_in<gf::apply_modal_kernel<16, 32, false>>(gf::modal_smem_bytes<double, 16, 32>()) ||
        !smem_opt_in<gf::modal_stencil_f32_kernel<gf::ST_SWEEP, float, float, 32, 16>>(
            gf::modal_smem_bytes<float, 32, 16>()) ||
        !smem_opt_in<gf::modal_stencil_f32_kernel<gf::ST_SWEEP, float, float, 16, 32>>(
            gf::modal_smem_bytes<float, 16, 32>()) ||
        !smem_opt_in<gf::apply_modal_kernel<16, 16, false>>(gf::modal_smem_bytes<double, 16, 16>()) ||
        !smem_opt_in<gf::modal_stencil_f32_kernel<gf::ST_SWEEP, float, float, 16, 16>>(
            gf::modal_smem_bytes<float, 16, 16>()))
        return set_err(GF_ERR_CUDA, "shared memory of the modal kernels");
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gf::apply_modal_kernel<32, 16>, gf::MODAL_THREADS,
                                                      gf::modal_smem_bytes<double, 32, 16>()) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    struct Cand {
        int bx, by;
        double cost;
        std::vector<int4> items;
    };
    Level& f = g->lv[0];
    const gf::GridDims d = f.dims();
    const int NZ = g->nz + 1;
    if (cudaMemsetAsync(g->modal_es, 0, sizeof(double) * 9 * f.nel, g->stream) != cudaSuccess ||
        cudaMemsetAsync(f.x64, 0, sizeof(double) * f.ndof, g->stream) != cudaSuccess ||
        cudaMemsetAsync(f.x32, 0, sizeof(float) * f.ndof, g->stream) != cudaSuccess ||
        cudaMemsetAsync(f.b32, 0, sizeof(float) * f.ndof, g->stream) != cudaSuccess ||
        cudaMemsetAsync(f.E32, 0, sizeof(float) * f.nel, g->stream) != cudaSuccess)
        return set_err(GF_ERR_CUDA, "modal autotune set-up");
    for (int f32 = 0; f32 <= 1; ++f32) {
        if (f32 && !g->modal_f32) break;
        std::vector<Cand> cand;
        for (int bx : {32, 16})
            for (int L : {0, 2, 3, 4, 6, 8, 12, 16, 24, 33, 48, 64}) {
                if (L > NZ || (g->half_sm && bx == 32)) continue;
                const int by = g->half_sm ? 16 : gf::MODAL_THREADS / bx;
                Cand c{bx, by, 0.0, {}};
                c.items = gf::modal_plan(g->nx, g->ny, g->nz, bx, by, g->sms * per_sm, L, &c.cost, f32);
                cand.push_back(std::move(c));
            }
        std::stable_sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) { return a.cost < b.cost; });
        if (cand.size() > 6) cand.resize(6);
        size_t maxn = 0;
        for (const Cand& c : cand) maxn = std::max(maxn, c.items.size());
        int4* dev = nullptr;
        RET(alloc((void**)&dev, sizeof(int4) * maxn));
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        int rc = GF_OK;
        float best = 1e30f;
        int best_i = -1;
        auto run = [&](const Cand& c) {
            const unsigned n = (unsigned)c.items.size();
            const gf::ModalSide sd = gf::modal_side(d, c.bx, c.by);
            const long long ne = sd.entries(d);
            if (!f32) {
                if (c.bx == 32)
                    gf::apply_modal_kernel<32, 16><<<n, dim3(32, 16), gf::modal_smem_bytes<double, 32, 16>(),
                                                     g->stream>>>(f.x64, f.t64, g->modal_es, d, dev, g->modal_side,
                                                                  sd, nullptr);
                else if (c.by == 32)
                    gf::apply_modal_kernel<16, 32><<<n, dim3(16, 32), gf::modal_smem_bytes<double, 16, 32>(),
                                                     g->stream>>>(f.x64, f.t64, g->modal_es, d, dev, g->modal_side,
                                                                  sd, nullptr);
                else
                    gf::apply_modal_kernel<16, 16><<<n, dim3(16, 16), gf::modal_smem_bytes<double, 16, 16>(),
                                                     g->stream>>>(f.x64, f.t64, g->modal_es, d, dev, g->modal_side,
                                                                  sd, nullptr);
                gf::modal_fixup_kernel<false><<<(unsigned)((ne + 255) / 256), 256, 0, g->stream>>>(
                    g->modal_side, sd, f.t64, d, nullptr);
            } else if (c.bx == 32) {   // the FP32 sweep (tiles overlapping by one column; no fix-up)
                gf::modal_stencil_f32_kernel<gf::ST_SWEEP, float, float, 32, 16>
                    <<<n, dim3(32, 16), gf::modal_smem_bytes<float, 32, 16>(), g->stream>>>(
                        f.x32, (const float*)f.b32, f.t32, f.E32, d, g->Kmodal32, 0.6f, dev, nullptr);
            } else if (c.by == 32) {
                gf::modal_stencil_f32_kernel<gf::ST_SWEEP, float, float, 16, 32>
                    <<<n, dim3(16, 32), gf::modal_smem_bytes<float, 16, 32>(), g->stream>>>(
                        f.x32, (const float*)f.b32, f.t32, f.E32, d, g->Kmodal32, 0.6f, dev, nullptr);
            } else {
                gf::modal_stencil_f32_kernel<gf::ST_SWEEP, float, float, 16, 16>
                    <<<n, dim3(16, 16), gf::modal_smem_bytes<float, 16, 16>(), g->stream>>>(
                        f.x32, (const float*)f.b32, f.t32, f.E32, d, g->Kmodal32, 0.6f, dev, nullptr);
            }
        };
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
            rc = set_err(GF_ERR_CUDA, "modal autotune events");
        for (size_t i = 0; rc == GF_OK && i < cand.size(); ++i) {
            const Cand& c = cand[i];
            if (cudaMemcpyAsync(dev, c.items.data(), sizeof(int4) * c.items.size(), cudaMemcpyHostToDevice,
                                g->stream) != cudaSuccess) {
                rc = set_err(GF_ERR_CUDA, "modal autotune items");
                break;
            }
            run(c);
            cudaEventRecord(e0, g->stream);
            for (int r = 0; r < 3; ++r) run(c);
            cudaEventRecord(e1, g->stream);
            float ms = 0.0f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
                cudaGetLastError() != cudaSuccess) {
                rc = set_err(GF_ERR_CUDA, "modal autotune launch");
                break;
            }
            if (ms < best) {
                best = ms;
                best_i = (int)i;
            }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(dev);
        RET(rc);
        if (best_i >= 0) {
            const Cand& c = cand[best_i];
            int4** dst = f32 ? &g->modal_items : &g->modal64_items;
            cudaFree(*dst);
            *dst = nullptr;
            RET(alloc((void**)dst, sizeof(int4) * c.items.size()));
            CK(cudaMemcpy(*dst, c.items.data(), sizeof(int4) * c.items.size(), cudaMemcpyHostToDevice));
            (f32 ? g->modal_n : g->modal64_n) = (int)c.items.size();
            (f32 ? g->modal_bx : g->modal64_bx) = c.bx;
            (f32 ? g->modal_by : g->modal64_by) = c.by;
        }
    }
    return GF_OK;
}
}  // namespace
extern "C" {

int gf_destroy_grid(gf_grid* g)
{
    if (!g) return GF_OK;
    cudaSetDevice(g->device);
    cudaStreamSynchronize(g->stream);
    for (Level& L : g->lv) {
        cudaFree(L.E64); cudaFree(L.E32);
        cudaFree(L.b64); cudaFree(L.x64); cudaFree(L.t64); cudaFree(L.r64);
        cudaFree(L.b32); cudaFree(L.x32); cudaFree(L.t32); cudaFree(L.r32);
        cudaFree(L.q64); cudaFree(L.q32);
        cudaFree(L.Ke64); cudaFree(L.Ke32);
        cudaFree(L.fix);
    }
    cudaFree(g->galG); cudaFree(g->gal_s[0]); cudaFree(g->gal_s[1]);
    cudaFree(g->ls_partial); cudaFree(g->ls_alpha);
    cudaFree(g->fcV); cudaFree(g->fcZ); cudaFree(g->fcR); cudaFree(g->fcD); cudaFree(g->fcQ); cudaFree(g->fcZT);
    cudaFree(g->fc); cudaFree(g->fc_partial);
    cudaFree(g->Ainv); cudaFree(g->Agj); cudaFree(g->ldl_ws); cudaFree(g->cpos); cudaFree(g->cidx); cudaFree(g->dflag); cudaFree(g->cheb); cudaFree(g->cheb_ss);
    cudaFree(g->rho64); cudaFree(g->rho16); cudaFree(g->work); cudaFree(g->partial);
    cudaFree(g->st); cudaFree(g->gst); cudaFree(g->V); cudaFree(g->Vd); cudaFree(g->pdd); cudaFree(g->ddticket); cudaFree(g->cgsticket); cudaFree(g->Z); cudaFree(g->hist);
    cudaFree(g->ckx);
    cudaFree(g->lz);
    cudaFree(g->lzv);
    cudaFree(g->Edf);
    cudaFree(g->modal_items);
    cudaFree(g->modal64_items);
    cudaFree(g->modal_side);
    cudaFree(g->modal_es);
    cudaFree(g->B3);
    cudaFree(g->Btc);
    cudaFree(g->oc_rho); cudaFree(g->oc_dc); cudaFree(g->oc_dcx); cudaFree(g->oc_dvx); cudaFree(g->oc_ones);
    cudaFree(g->oc_st);
    if (g->host_status) cudaFreeHost(g->host_status);
    drop_graphs(g);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    for (int i = 0; i < 3; ++i)
        if (g->ev[i]) cudaEventDestroy(g->ev[i]);
    delete g;
    return GF_OK;
}

int gf_grid_sizes(const gf_grid* g, int* n_dof, int* n_elem, int* n_nodes, int* levels)
{
    RET(check_grid(g));
    if (n_dof) *n_dof = (int)g->ndof;
    if (n_elem) *n_elem = (int)g->nel;
    if (n_nodes) *n_nodes = (int)g->nodes;
    if (levels) *levels = g->L;
    return GF_OK;
}

int gf_set_density(gf_grid* g, const double* rho_hat, double p)
{
    RET(check_grid(g));
    if (!rho_hat) return set_err(GF_ERR_ARG, "null rho_hat");
    if (!(p >= 1.0 && p <= 16.0)) return set_err(GF_ERR_ARG, "p in [1,16]");
    RET(set_device(g));
    CK(cudaMemsetAsync(g->dflag, 0, sizeof(int), g->stream));
    LAUNCH(g, nblk(g->nel), 256, gf::density_check_kernel, rho_hat, g->rho16, g->rho64, g->nel, g->dflag);
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, g->dflag, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    g->has_floor = false;
    if (bad) {
        g->has_density = false;
        return set_err(GF_ERR_NONFINITE, "density has NaN/Inf or values outside [0,1]");
    }
    LAUNCH(g, g->nbr, 256, gf::density_stats_kernel, (const double*)g->rho64, g->nel, g->partial);
    std::vector<double> part((size_t)g->nbr * 3);
    CK(cudaMemcpyAsync(part.data(), g->partial, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    double z = 0.0, s1 = 0.0, s2 = 0.0;
    for (int b = 0; b < g->nbr; ++b) {
        z += part[3 * b];
        s1 += part[3 * b + 1];
        s2 += part[3 * b + 2];
    }
    const double n = (double)g->nel, mean = s1 / n;
    g->dstat[0] = z / n;
    g->dstat[1] = mean;
    g->dstat[2] = std::sqrt(std::max(0.0, s2 / n - mean * mean));
    g->p = p;
    g->has_density = true;
    return GF_OK;
}

int gf_set_floor(gf_grid* g, double rho_min)
{
    RET(check_grid(g));
    if (!g->has_density) return set_err(GF_ERR_STATE, "set_density first");
    if (!(rho_min > 0.0 && rho_min <= 1.0)) return set_err(GF_ERR_ARG, "rho_min in (0,1]");
    RET(set_device(g));
    const double p = g->p;
    const int p_int = (p == std::floor(p)) ? (int)p : 0;
    Level& f = g->lv[0];
    LAUNCH(g, nblk(g->nel), 256, gf::modulus_fp64_kernel, g->rho64, f.E64, g->nel, rho_min, p, p_int, f.h);
    if (g->modal_es)
        LAUNCH(g, nblk(g->nel), 256, gf::modal_scale_kernel, (const double*)f.E64, g->Kmodal, g->modal_es,
               (long long)g->nel);
    LAUNCH(g, nblk(g->nel), 256, gf::modulus_fp32_kernel, g->rho16, f.E32, g->nel, (float)rho_min, (float)p,
           p_int, (float)f.h);
    if (g->has_split) LAUNCH(g, nblk(g->nel), 256, gf::edf_kernel, (const double*)f.E64, g->s_split, g->Edf, g->nel);
    for (int l = 1; l < g->L; ++l) {
        Level& c = g->lv[l];
        LAUNCH(g, nblk(c.nel), 256, gf::coarsen_kernel<double>, g->lv[l - 1].E64, c.E64, c.dims());
        LAUNCH(g, nblk(c.nel), 256, gf::coarsen_kernel<float>, g->lv[l - 1].E32, c.E32, c.dims());
    }
    if (g->coarse_kind == GF_COARSE_GALERKIN) RET(build_galerkin(g));
    if (!g->skip_coarse_inverse) RET(build_coarse_inverse(g));
    g->rho_min = rho_min;
    g->has_floor = true;
    g->cheb_ready[0] = g->cheb_ready[1] = false;
    return GF_OK;
}

int gf_set_coarse_operator(gf_grid* g, int kind)
{
    RET(check_grid(g));
    if (kind != GF_COARSE_REDISCRETISED && kind != GF_COARSE_GALERKIN)
        return set_err(GF_ERR_ARG, "kind must be GF_COARSE_REDISCRETISED or GF_COARSE_GALERKIN");
    if (kind == g->coarse_kind) return GF_OK;
    if (g->geom != GF_GEOM_CANTILEVER) return set_err(GF_ERR_ARG, "the bridge geometry keeps rediscretised coarse levels");
    RET(set_device(g));
    drop_graphs(g);            // captured Arnoldi steps hold the other V-cycle
    g->coarse_kind = kind;
    g->has_floor = false;      // the next gf_set_floor builds the hierarchy
    return GF_OK;
}

int gf_set_sm_share(gf_grid* g, int share)
{
    RET(check_grid(g));
    if (share != 0 && share != 1) return set_err(GF_ERR_ARG, "share must be 0 or 1");
    if ((share != 0) == g->half_sm) return GF_OK;
    RET(set_device(g));
    drop_graphs(g);            // captured Arnoldi steps hold the other launch shapes
    g->has_floor = false;      // the modal autotune below runs on the level-0 buffers
    g->half_sm = share != 0;
    long long rows = 0;
    RET(cgs_grids(g, &rows));
    if (g->modal64_items) {
        RET(modal_default_plan(g));
        if (!getenv("GF_MODAL_CHUNK") && !getenv("GF_MODAL_BX")) RET(modal_autotune(g));
    }
    CK(cudaStreamSynchronize(g->stream));
    return GF_OK;
}

int gf_cantilever_load(gf_grid* g, double* f)
{
    RET(check_grid(g));
    if (!f) return set_err(GF_ERR_ARG, "null f");
    RET(set_device(g));
    LAUNCH(g, nblk(g->ndof), 256, gf::cantilever_load_kernel, f, g->lv[0].dims());
    return GF_OK;
}

int gf_set_geometry(gf_grid* g, int geometry)
{
    RET(check_grid(g));
    if (geometry != GF_GEOM_CANTILEVER && geometry != GF_GEOM_BRIDGE)
        return set_err(GF_ERR_ARG, "geometry must be GF_GEOM_CANTILEVER or GF_GEOM_BRIDGE");
    if (geometry == g->geom) return GF_OK;
    RET(set_device(g));
    if (geometry == GF_GEOM_BRIDGE) {
        if (g->nz % 2) return set_err(GF_ERR_ARG, "the bridge's mid-depth supports need even nz");
        if (g->coarse_kind != GF_COARSE_REDISCRETISED)
            return set_err(GF_ERR_ARG, "the bridge geometry keeps rediscretised coarse levels");
        for (int l = 0; l < g->L; ++l) {
            Level& c = g->lv[l];
            RET(allocT(&c.fix, (size_t)c.nodes));
            LAUNCH(g, nblk(c.nodes), 256, gf::bridge_fix_kernel, c.fix, gf::GridDims{c.nx, c.ny, c.nz}, l, g->nx, g->nz);
            g->stc_cz[l] = 0;   // the variants that read the clamped face from the index are off
        }
        g->vc_l0 = -1;
        if (g->tpb[1] <= 0) g->tpb[1] = 256;
    } else {
        for (Level& c : g->lv) {
            cudaFree(c.fix);
            c.fix = nullptr;
        }
    }
    RET(build_coarse_map(g));
    drop_graphs(g);
    g->geom = geometry;
    g->has_floor = false;   // gf_set_floor again: the coarsest inverse carries the supports
    return GF_OK;
}

int gf_bridge_load(gf_grid* g, double* f)
{
    RET(check_grid(g));
    if (!f) return set_err(GF_ERR_ARG, "null f");
    RET(set_device(g));
    LAUNCH(g, nblk(g->ndof), 256, gf::bridge_load_kernel, f, g->lv[0].dims(), g->h * g->h);
    return GF_OK;
}

int gf_free_mask(gf_grid* g, uint8_t* mask)
{
    RET(check_grid(g));
    if (!mask) return set_err(GF_ERR_ARG, "null mask");
    RET(set_device(g));
    LAUNCH(g, nblk(g->ndof), 256, gf::free_mask_kernel, mask, g->lv[0].dims());
    return GF_OK;
}

int gf_apply_K(gf_grid* g, const double* u, double* y)
{
    RET(check_grid(g));
    if (!u || !y || u == y) return set_err(GF_ERR_ARG, "u, y non-null and distinct");
    if (!g->has_floor) return set_err(GF_ERR_STATE, "set_floor first");
    RET(set_device(g));
    return applyK64(g, u, y, nullptr);
}

int gf_apply_K_split(gf_grid* g, const double* u, double* y)
{
    if (g && g->geom != GF_GEOM_CANTILEVER) return set_err(GF_ERR_ARG, "the split operator serves the cantilever only");
    RET(check_grid(g));
    if (!u || !y || u == y) return set_err(GF_ERR_ARG, "u, y non-null and distinct");
    if (!g->has_floor) return set_err(GF_ERR_STATE, "set_floor first");
    if (!g->has_split) return set_err(GF_ERR_ARG, "K0 has no small integer form for this Poisson ratio");
    RET(set_device(g));
    return applyKsplit(g, u, y, nullptr);
}

int gf_apply_K_f32(gf_grid* g, const float* u, float* y)
{
    RET(check_grid(g));
    if (!u || !y || u == y) return set_err(GF_ERR_ARG, "u, y non-null and distinct");
    if (!g->has_floor) return set_err(GF_ERR_STATE, "set_floor first");
    RET(set_device(g));
    return stencil<float, float, gf::ST_APPLY>(g, 0, u, nullptr, y, g->lv[0].E32, g->K0f, 0.0f, nullptr);
}

int gf_vcycle(gf_grid* g, const double* v, double* z, int prec, int nu1, int nu2, double omega)
{
    RET(check_grid(g));
    if (!v || !z || v == z) return set_err(GF_ERR_ARG, "v, z non-null and distinct");
    if (!g->has_floor) return set_err(GF_ERR_STATE, "set_floor first");
    if (prec != GF_FP64 && prec != GF_MIXED) return set_err(GF_ERR_ARG, "prec");
    if (nu1 < 1 || nu2 < 1 || nu1 > 16 || nu2 > 16 || !(omega > 0 && omega < 2)) return set_err(GF_ERR_ARG, "smoother");
    RET(set_device(g));
    g->coarse_steps = 0;
    return vcycle_dispatch(g, v, z, prec, nu1, nu2, omega, nullptr);
}

int gf_vcycle_ex(gf_grid* g, const double* v, double* z, const gf_solve_opts* o)
{
    RET(check_grid(g));
    RET(validate_opts(o));
    RET(validate_geom(g, o));
    if (!v || !z || v == z) return set_err(GF_ERR_ARG, "v, z non-null and distinct");
    if (!g->has_floor) return set_err(GF_ERR_STATE, "set_floor first");
    RET(set_device(g));
    if (o->smoother == 1) RET(ensure_cheb(g, o->prec));
    if (o->ls_ratio > 0.0) RET(ensure_ls(g));
    RET(set_coarse_steps(g, o));
    return vcycle_dispatch(g, v, z, o->prec, o->nu1, o->nu2, o->omega, nullptr, o->smoother, o->ls_ratio,
                           o->fine_steps);
}

int gf_chebyshev_lambda(gf_grid* g, int prec, double* lam, int n)
{
    RET(check_grid(g));
    if (!lam || n < g->L - 1) return set_err(GF_ERR_ARG, "lam needs levels - 1 entries");
    if (prec != GF_FP64 && prec != GF_MIXED) return set_err(GF_ERR_ARG, "prec");
    if (!g->has_floor) return set_err(GF_ERR_STATE, "set_floor first");
    RET(set_device(g));
    RET(ensure_cheb(g, prec));
    for (int l = 0; l < g->L - 1; ++l)
        CK(cudaMemcpyAsync(lam + l, cheb_slot(g, prec == GF_FP64 ? 0 : 1, l), sizeof(double), cudaMemcpyDeviceToHost,
                           g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return GF_OK;
}

int gf_solve(gf_grid* g, const double* f, double* u, const gf_solve_opts* opts, gf_solve_info* info)
{
    RET(check_grid(g));
    RET(validate_opts(opts));
    RET(validate_geom(g, opts));
    if (!f || !u || f == u) return set_err(GF_ERR_ARG, "f, u non-null and distinct");
    if (!g->has_floor) return set_err(GF_ERR_STATE, "set_floor first");
    RET(set_device(g));
    return solve_impl(g, f, u, opts, info, false, opts->history);
}

int gf_conditioning(gf_grid* g, const double* f, int iters, double* lambda_min, double* lambda_max,
                    double* eta_direct)
{
    if (g && g->geom != GF_GEOM_CANTILEVER) return set_err(GF_ERR_ARG, "the conditioning diagnostic serves the cantilever only");
    RET(check_grid(g));
    if (!lambda_min || !lambda_max || (eta_direct && !f)) return set_err(GF_ERR_ARG, "null pointer");
    if (g->L != 1) return set_err(GF_ERR_STATE, "gf_conditioning needs a one-level grid (levels = 1)");
    if (!g->has_floor) return set_err(GF_ERR_STATE, "set_floor first");
    if (iters < 2 || iters > gf::LZ_MAX) return set_err(GF_ERR_ARG, "iters in [2, 512]");
    RET(set_device(g));
    const long long n = g->ndof;
    if (!g->lz) RET(allocT(&g->lz, 1));
    if (!g->lzv) RET(allocT(&g->lzv, (size_t)3 * n));
    for (int pass = 0; pass < 2; ++pass) {   // 0: K (lambda_max), 1: K^{-1} (1 / lambda_min)
        double *v = g->lzv, *vp = g->lzv + n, *w = g->lzv + 2 * n;
        LAUNCH(g, 1, gf::LZ_THREADS, gf::lanczos_start_kernel, v, vp, n, g->nx + 1, g->lz);
        for (int j = 0; j < iters; ++j) {
            if (pass == 0)
                RET(applyK64(g, v, w, nullptr));
            else
                LAUNCH(g, nblk(32LL * n), 256, (gf::dense_gemv_kernel<double, double>), (const double*)g->Ainv,
                       (const double*)v, w, (int)n, (const int*)nullptr);
            LAUNCH(g, 1, gf::LZ_THREADS, gf::lanczos_step_kernel, w, (const double*)v, vp, n, j, g->lz);
            std::swap(v, vp);   // v_{j+1} was written over v_{j-1}
        }
        LAUNCH(g, 1, 32, gf::lanczos_tridiag_kernel, g->lz, iters);
        double hi = 0.0;
        CK(cudaMemcpyAsync(&hi, &g->lz->hi, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
        if (!(hi > 0.0) || !std::isfinite(hi)) return set_err(GF_ERR_NONFINITE, "Lanczos estimate not positive");
        if (pass == 0) *lambda_max = hi;
        else *lambda_min = 1.0 / hi;
    }
    if (eta_direct) {   // the direct solution u = K^{-1} f and its guard residual
        double* u = g->lzv;
        LAUNCH(g, nblk(32LL * n), 256, (gf::dense_gemv_kernel<double, double>), (const double*)g->Ainv, f, u, (int)n,
               (const int*)nullptr);
        RET(guard_impl(g, f, u, eta_direct));
    }
    return GF_OK;
}

int gf_conditioning_screen(double lambda_min, double lambda_max, double rho_min, double tau, double* rho_screen)
{
    if (!rho_screen || !(lambda_min > 0.0) || !(lambda_max >= lambda_min) || !(rho_min > 0.0) || !(tau > 0.0))
        return set_err(GF_ERR_ARG, "need 0 < lambda_min <= lambda_max, rho_min > 0, tau > 0");
    const double c = lambda_max / lambda_min * rho_min;   // kappa ~ c / rho_min
    *rho_screen = c * DBL_EPSILON / tau;
    return GF_OK;
}

int gf_true_residual(gf_grid* g, const double* f, const double* u, double* eta)
{
    RET(check_grid(g));
    if (!f || !u || !eta) return set_err(GF_ERR_ARG, "null pointer");
    if (!g->has_floor) return set_err(GF_ERR_STATE, "set_floor first");
    RET(set_device(g));
    return guard_impl(g, f, u, eta);
}

void gf_policy_defaults(gf_policy* pol)
{
    if (!pol) return;
    std::memset(pol, 0, sizeof(*pol));
    pol->rho0 = 1e-6;
    pol->ladder[0] = 1e-5;
    pol->ladder[1] = 1e-4;
    pol->ladder[2] = 1e-3;
    pol->n_ladder = 3;
    pol->tau = 1e-6;
    pol->kmax = 200;
    pol->probe_iters = 100;
    pol->r50_escalate = 1e-2;
    pol->r100_stall = 1e-4;
    pol->plateau_ratio = 0.6;
    pol->checkpoint_a = 50;
    pol->checkpoint_b = 100;
    pol->selector = GF_SEL_RULE;
    pol->first_index = 0;
    pol->fuse_probe = 1;
    pol->solve.restart = 30;
    pol->solve.kmax = 200;
    pol->solve.tol = 1e-6;
    pol->solve.prec = GF_FP64;
    pol->solve.nu1 = 2;
    pol->solve.nu2 = 2;
    pol->solve.omega = 0.6;
    pol->solve.history = nullptr;
    pol->solve.outer = 0;
    pol->mlp = nullptr;
    pol->mlp_confidence = 0.0;
    pol->true_check_every = 0;
    pol->true_check_ratio = 10.0;
}

int gf_trigger_rule(double r50, double r100, const gf_policy* pol)
{
    if (!pol) return set_err(GF_ERR_ARG, "null policy");
    return (r50 >= pol->r50_escalate) || (r100 >= pol->r100_stall && r100 / r50 >= pol->plateau_ratio) ? 1 : 0;
}

int gf_probe_features(const double* history, int k_stop, const gf_policy* pol, double* r50, double* r100)
{
    if (!history || !pol || !r50 || !r100 || k_stop < 0) return set_err(GF_ERR_ARG, "bad argument");
    *r50 = history[std::min(pol->checkpoint_a, k_stop)];
    *r100 = history[std::min(pol->checkpoint_b, k_stop)];
    return GF_OK;
}

// true-residual checks: GF_SEL_RULE (also GF_SEL_REUSE's fallback) on one grid
int validate_true_checks(const gf_policy* pol)
{
    if (pol->true_check_every < 0) return set_err(GF_ERR_ARG, "true_check_every < 0");
    if (pol->true_check_every == 0) return GF_OK;
    if (pol->selector != GF_SEL_RULE && pol->selector != GF_SEL_REUSE)
        return set_err(GF_ERR_ARG, "true_check_every needs GF_SEL_RULE or GF_SEL_REUSE");
    if (pol->probe_iters / pol->true_check_every > GF_MAX_TRUE_CHECKS)
        return set_err(GF_ERR_ARG, "probe_iters / true_check_every > GF_MAX_TRUE_CHECKS");
    if (!(pol->true_check_ratio > 0.0)) return set_err(GF_ERR_ARG, "true_check_ratio must be > 0");
    return GF_OK;
}

// GF_SEL_REUSE: the previous decision, then Algorithm 1 from scratch if the guard rejects it
int select_floor_reuse(gf_grid* g, const double* f, double* u, const gf_policy* pol, gf_select_info* info)
{
    const int nf = pol->n_ladder + 1;
    if (pol->first_index < 0 || pol->first_index >= nf) return set_err(GF_ERR_ARG, "first_index");
    if (pol->n_ladder > GF_MAX_LADDER - 1) return set_err(GF_ERR_ARG, "GF_SEL_REUSE: n_ladder <= GF_MAX_LADDER - 1");
    gf_solve_opts o = pol->solve;
    o.history = nullptr;
    o.tol = pol->tau;
    o.kmax = pol->kmax;
    RET(validate_opts(&o));
    RET(validate_geom(g, &o));
    RET(set_device(g));
    const double rm = pol->first_index == 0 ? pol->rho0 : pol->ladder[pol->first_index - 1];
    if (!(g->has_floor && g->rho_min == rm)) RET(gf_set_floor(g, rm));
    gf_solve_info si{};
    CK(cudaMemsetAsync(u, 0, sizeof(double) * g->ndof, g->stream));
    RET(solve_impl(g, f, u, &o, &si, true, nullptr));
    double eta = 0.0;
    RET(guard_impl(g, f, u, &eta));
    gf_attempt a{};
    a.rho_min = rm;
    a.iters = si.iters;
    a.flag = si.flag;
    a.stop_estimate = si.stop_estimate;
    a.eta = eta;
    a.accepted = eta <= pol->tau;
    if (a.accepted) {
        std::memset(info, 0, sizeof(*info));
        info->r50 = info->r100 = std::nan("");
        info->status = GF_ACCEPTED;
        info->floor_index = pol->first_index;
        info->rho_min = rm;
        info->eta = eta;
        info->escalated = pol->first_index > 0;
        info->n_attempts = 1;
        info->attempts[0] = a;
        return GF_OK;
    }
    gf_policy rule = *pol;
    rule.selector = GF_SEL_RULE;
    RET(gf_select_floor(g, f, u, &rule, info));
    for (int i = info->n_attempts; i > 0; --i) info->attempts[i] = info->attempts[i - 1];
    info->attempts[0] = a;
    info->n_attempts += 1;
    return GF_OK;
}

int gf_select_floor(gf_grid* g, const double* f, double* u, const gf_policy* pol, gf_select_info* info)
{
    RET(check_grid(g));
    if (!f || !u || !pol || !info || f == u) return set_err(GF_ERR_ARG, "null pointer");
    if (!g->has_density) return set_err(GF_ERR_STATE, "set_density first");
    if (pol->selector == GF_SEL_REUSE) {
        if (pol->n_ladder < 0) return set_err(GF_ERR_ARG, "n_ladder");
        if (!(pol->rho0 > 0) || pol->probe_iters < 0 || pol->kmax < 0) return set_err(GF_ERR_ARG, "policy");
        RET(validate_true_checks(pol));
        return select_floor_reuse(g, f, u, pol, info);
    }
    if (pol->n_ladder < 0 || pol->n_ladder > GF_MAX_LADDER) return set_err(GF_ERR_ARG, "n_ladder");
    if (!(pol->rho0 > 0) || pol->probe_iters < 0 || pol->kmax < 0) return set_err(GF_ERR_ARG, "policy");
    RET(validate_true_checks(pol));
    gf_solve_opts o = pol->solve;
    o.history = nullptr;
    o.tol = pol->tau;
    RET(validate_opts(&o));
    RET(validate_geom(g, &o));
    RET(set_device(g));
    std::memset(info, 0, sizeof(*info));
    info->r50 = info->r100 = std::nan("");
    info->floor_index = -1;
    info->rho_min = std::nan("");
    info->eta = std::nan("");
    double floors[GF_MAX_LADDER + 1];
    floors[0] = pol->rho0;
    for (int i = 0; i < pol->n_ladder; ++i) floors[i + 1] = pol->ladder[i];
    const int nf = pol->n_ladder + 1;
    int start = 0;
    if (pol->selector == GF_SEL_MLP && !pol->mlp) return set_err(GF_ERR_ARG, "GF_SEL_MLP needs a trained gf_mlp");
    ProbeHook hook;   // the fused probe's decision point and the probe's true-residual checks
    hook.every = pol->true_check_every;
    hook.upto = pol->probe_iters;
    hook.ratio = pol->true_check_ratio;
    auto decide = [&](double r50, double r100, int* first) -> int {
        if (pol->selector == GF_SEL_MLP) {
            double x[6];
            RET(gf_select_features(g, r50, r100, x));
            RET(mlp_first_floors(pol->mlp, x, 1, pol->mlp_confidence, nf, first));
        } else {   // Eq. (trigger), or the checkpointed detector
            *first = (gf_trigger_rule(r50, r100, pol) || hook.fired) ? 1 : 0;
        }
        return GF_OK;
    };
    auto record_checks = [&]() {
        info->n_true_checks = hook.n;
        for (int q = 0; q < hook.n; ++q) {
            info->true_check_k[q] = hook.ck[q];
            info->true_check_est[q] = hook.est[q];
            info->true_check_eta[q] = hook.eta[q];
        }
        info->true_check_fired = hook.fired ? 1 : 0;
    };
    if ((pol->selector == GF_SEL_RULE && pol->fuse_probe) || pol->selector == GF_SEL_MLP) {
        // Probe fused with the rho0 solve: run the rho0 solve with budget kmax and read
        // r50/r100 off its history after probe_iters steps (or at its stop).
        RET(gf_set_floor(g, pol->rho0));
        gf_solve_opts so = o;
        so.kmax = std::max(pol->kmax, pol->probe_iters);
        const bool cap = pol->probe_iters > pol->kmax;   // the probe may run past kmax
        gf_solve_opts so2 = o;
        so2.kmax = pol->kmax;
        hook.at = pol->probe_iters;
        hook.pol = pol;
        hook.decide = decide;
        std::vector<double> hist((size_t)so.kmax + 1);
        gf_solve_info si{};
        CK(cudaMemsetAsync(u, 0, sizeof(double) * g->ndof, g->stream));
        RET(solve_impl(g, f, u, cap ? &so : &so2, &si, true, hist.data(), &hook));
        if (hook.decided) {
            info->r50 = hook.r50;
            info->r100 = hook.r100;
            start = hook.first;
            info->probe_iters_run = pol->probe_iters;
        } else {
            info->probe_iters_run = std::min(si.iters, pol->probe_iters);
            RET(gf_probe_features(hist.data(), si.iters, pol, &info->r50, &info->r100));
            RET(decide(info->r50, info->r100, &start));
        }
        record_checks();
        info->escalated = start > 0;
        if (!info->escalated && !cap) {
            // the rho0 solve is the first candidate's selected solve
            double eta = 0.0;
            RET(guard_impl(g, f, u, &eta));
            gf_attempt& a = info->attempts[info->n_attempts++];
            a.rho_min = pol->rho0;
            a.iters = si.iters;
            a.flag = si.flag;
            a.stop_estimate = si.stop_estimate;
            a.eta = eta;
            a.accepted = eta <= pol->tau;
            if (a.accepted) {
                info->status = GF_ACCEPTED;
                info->floor_index = 0;
                info->rho_min = pol->rho0;
                info->eta = eta;
                return GF_OK;
            }
            start = 1;
        }
    } else if (pol->selector == GF_SEL_RULE) {
        RET(gf_set_floor(g, pol->rho0));
        std::vector<double> hist((size_t)pol->probe_iters + 1);
        gf_solve_opts po = o;
        po.kmax = pol->probe_iters;
        gf_solve_info pi{};
        CK(cudaMemsetAsync(u, 0, sizeof(double) * g->ndof, g->stream));
        RET(solve_impl(g, f, u, &po, &pi, true, hist.data(), &hook));   // hook.at < 0: checks only
        info->probe_iters_run = pi.iters;
        RET(gf_probe_features(hist.data(), pi.iters, pol, &info->r50, &info->r100));
        record_checks();
        info->escalated = gf_trigger_rule(info->r50, info->r100, pol) || hook.fired;
        start = info->escalated ? 1 : 0;
    } else if (pol->selector == GF_SEL_FULL) {
        start = 0;
    } else if (pol->selector == GF_SEL_GIVEN) {
        if (pol->first_index < 0 || pol->first_index >= nf) return set_err(GF_ERR_ARG, "first_index");
        start = pol->first_index;
        info->escalated = start > 0;
    } else {
        return set_err(GF_ERR_ARG, "selector");
    }
    info->status = GF_NO_ADMISSIBLE_FLOOR;
    for (int idx = start; idx < nf; ++idx) {
        if (idx == 0 && info->n_attempts > 0) continue;   // rho0 already attempted (fused probe)
        const double rm = floors[idx];
        if (!(g->has_floor && g->rho_min == rm)) RET(gf_set_floor(g, rm));
        o.kmax = pol->kmax;
        gf_solve_info si{};
        CK(cudaMemsetAsync(u, 0, sizeof(double) * g->ndof, g->stream));
        const bool rho0_full = (idx == 0 && pol->selector == GF_SEL_FULL);
        std::vector<double> h0(rho0_full ? (size_t)o.kmax + 1 : 0);
        RET(solve_impl(g, f, u, &o, &si, true, rho0_full ? h0.data() : nullptr));
        if (rho0_full)   // features of the rho0 attempt (what a probe would have recorded)
            RET(gf_probe_features(h0.data(), si.iters, pol, &info->r50, &info->r100));
        double eta = 0.0;
        RET(guard_impl(g, f, u, &eta));
        gf_attempt& a = info->attempts[info->n_attempts++];
        a.rho_min = rm;
        a.iters = si.iters;
        a.flag = si.flag;
        a.stop_estimate = si.stop_estimate;
        a.eta = eta;
        a.accepted = eta <= pol->tau;
        if (a.accepted) {
            info->status = GF_ACCEPTED;
            info->floor_index = idx;
            info->rho_min = rm;
            info->eta = eta;
            break;
        }
    }
    return GF_OK;
}

int gf_select_floor_many(int n, gf_grid* const* grids, const double* const* f, double* const* u,
                         const gf_policy* pol, gf_select_info* info)
{
    if (n < 0 || (n > 0 && (!grids || !f || !u || !pol || !info))) return set_err(GF_ERR_ARG, "null pointer / n < 0");
    for (int i = 0; i < n; ++i) {
        RET(check_grid(grids[i]));
        for (int k = 0; k < i; ++k)
            if (grids[k] == grids[i]) return set_err(GF_ERR_ARG, "the same grid twice");
    }
    std::vector<int> rc(n, GF_OK);
    std::vector<std::string> msg(n);
    std::vector<std::thread> workers;
    workers.reserve(n);
    for (int i = 0; i < n; ++i)
        workers.emplace_back([&, i] {
            rc[i] = gf_select_floor(grids[i], f[i], u[i], pol, &info[i]);
            if (rc[i] != GF_OK) msg[i] = g_err;   // the worker's thread-local message
        });
    for (std::thread& t : workers) t.join();
    for (int i = 0; i < n; ++i)
        if (rc[i] != GF_OK) return set_err(rc[i], "grid " + std::to_string(i) + ": " + msg[i]);
    return GF_OK;
}

int gf_sensitivity(gf_grid* g, const double* u, double* dc)
{
    RET(check_grid(g));
    if (!u || !dc) return set_err(GF_ERR_ARG, "null pointer");
    if (!g->has_floor) return set_err(GF_ERR_STATE, "set_floor first");
    RET(set_device(g));
    gf::K0Param<double> K = g->K0d;
    for (int q = 0; q < 576; ++q) K.k[q] *= g->h;
    const double p = g->p;
    const int pm1_int = (p == std::floor(p)) ? (int)p - 1 : -1;
    LAUNCH(g, nblk(g->nel), 256, gf::sensitivity_kernel, u, g->rho64, dc, g->lv[0].dims(), K,
           -p * (1.0 - g->rho_min), p - 1.0, pm1_int);
    return GF_OK;
}

int gf_filter(gf_grid* g, const double* x, double* xt, double r_min)
{
    RET(check_grid(g));
    if (!x || !xt || x == xt) return set_err(GF_ERR_ARG, "x, xt non-null and distinct");
    if (!(r_min > 1.0 && r_min <= 8.0)) return set_err(GF_ERR_ARG, "r_min in (1, 8]");
    RET(set_device(g));
    return filter_impl(g, x, xt, r_min, false);
}

int gf_filter_adjoint(gf_grid* g, const double* gs, double* out, double r_min)
{
    RET(check_grid(g));
    if (!gs || !out || gs == out) return set_err(GF_ERR_ARG, "inputs non-null and distinct");
    if (!(r_min > 1.0 && r_min <= 8.0)) return set_err(GF_ERR_ARG, "r_min in (1, 8]");
    RET(set_device(g));
    return filter_impl(g, gs, out, r_min, true);
}

int gf_oc_update(gf_grid* g, const double* x, const double* dc, const double* dv, double volfrac, double move,
                 double* xnew)
{
    RET(check_grid(g));
    if (!x || !dc || !dv || !xnew) return set_err(GF_ERR_ARG, "null pointer");
    if (!(volfrac > 0 && volfrac < 1) || !(move > 0 && move <= 1)) return set_err(GF_ERR_ARG, "volfrac/move");
    RET(set_device(g));
    return oc_update_impl(g, x, dc, dv, volfrac, move, xnew);
}

int gf_compliance(gf_grid* g, const double* f, const double* u, double* c)
{
    RET(check_grid(g));
    if (!f || !u || !c) return set_err(GF_ERR_ARG, "null pointer");
    RET(set_device(g));
    return dot_impl(g, f, u, g->ndof, c);
}

int gf_oc_iteration(gf_grid* g, double* x, const double* f, double* u, const gf_policy* pol, double p,
                    double volfrac, double r_min, double move, gf_select_info* info, double* compliance)
{
    RET(check_grid(g));
    if (!x || !f || !u || !pol || !info || !compliance) return set_err(GF_ERR_ARG, "null pointer");
    RET(set_device(g));
    RET(ensure_oc(g));
    RET(filter_impl(g, x, g->oc_rho, r_min, false));                 // physical density
    RET(gf_set_density(g, g->oc_rho, p));
    RET(gf_select_floor(g, f, u, pol, info));                          // guarded state solve
    *compliance = std::nan("");
    if (info->status != GF_ACCEPTED) return GF_OK;                     // design kept unchanged
    RET(dot_impl(g, f, u, g->ndof, compliance));
    RET(gf_sensitivity(g, u, g->oc_dc));
    RET(filter_impl(g, g->oc_dc, g->oc_dcx, r_min, true));
    RET(filter_impl(g, g->oc_ones, g->oc_dvx, r_min, true));
    RET(oc_update_impl(g, x, g->oc_dcx, g->oc_dvx, volfrac, move, g->oc_rho));
    CK(cudaMemcpyAsync(x, g->oc_rho, sizeof(double) * g->nel, cudaMemcpyDeviceToDevice, g->stream));
    return GF_OK;
}

int gf_select_features(const gf_grid* g, double r50, double r100, double* x)
{
    RET(check_grid(g));
    if (!x) return set_err(GF_ERR_ARG, "null x");
    if (!g->has_density) return set_err(GF_ERR_STATE, "set_density first");
    x[0] = std::log10(std::max(r50, 1e-30));
    x[1] = std::log10(std::max(r100, 1e-30));
    x[2] = r100 / r50;
    x[3] = g->dstat[0];
    x[4] = g->dstat[1];
    x[5] = g->dstat[2];
    return GF_OK;
}

int gf_set_stencil_blocks(gf_grid* g, int tpb64, int tpb32)
{
    if (g && g->geom != GF_GEOM_CANTILEVER && tpb32 <= 0)
        return set_err(GF_ERR_ARG, "the bridge geometry runs the node-per-thread FP32 stencils (tpb32 > 0)");
    RET(check_grid(g));
    const auto ok = [](int t, bool f32) {
        return t == 64 || t == 128 || t == 256 || (f32 && (t == 0 || t == -64 || t == -128 || t == -256));
    };
    if (!ok(tpb64, false) || !ok(tpb32, true))
        return set_err(GF_ERR_ARG, "block sizes: 64/128/256 (FP32 also 0 = tiled, -64/-128/-256 = 27-neighbour)");
    g->tpb[0] = tpb64;
    g->tpb[1] = tpb32;
    drop_graphs(g);
    return GF_OK;
}

int gf_get_stats(const gf_grid* g, gf_stats* s)
{
    RET(check_grid(g));
    if (!s) return set_err(GF_ERR_ARG, "null stats");
    *s = g->stats;
    return GF_OK;
}

int gf_reset_stats(gf_grid* g)
{
    RET(check_grid(g));
    g->stats = gf_stats{};
    return GF_OK;
}

}  // extern "C"

// ============================================================ no-allocation guard ====
// gf_true_residual_noalloc: the acceptance residual computed without any device
// allocation, for callers that may not call cudaMalloc at all. Examples: code that
// records its work into a CUDA graph or runs inside stream capture (allocation
// calls are illegal there), a host that hands the library a fixed, pre-reserved
// memory budget, or a real-time loop that must not touch the allocator. The
// scratch it needs (the modulus field, the operator product and the per-block
// partial sums) lives in the file-scope array below, which every GPU that loads
// this library reserves until the process exits.
namespace {

constexpr long long NOALLOC_MAX_DOF = 1LL << 20;            // largest grid: 1,048,576 DOFs
constexpr long long NOALLOC_MAX_ELEM = NOALLOC_MAX_DOF / 3;  // elements <= nodes = DOFs / 3
constexpr int NOALLOC_BLOCKS = 256;                          // partial-sum slots
constexpr long long NOALLOC_WORDS = NOALLOC_MAX_DOF + NOALLOC_MAX_ELEM + 2LL * NOALLOC_BLOCKS;

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_WORDS];

// Device address of g_noalloc_scratch per device. In host code the symbol's name is
// only a host-side stand-in, so the address is looked up with the device current.
constexpr int NOALLOC_MAX_DEVICES = 64;
double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
std::mutex g_noalloc_mu;

int noalloc_scratch(double** out)
{
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return set_err(GF_ERR_ARG, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return GF_OK;
}

// eta = sqrt(sum a) / sqrt(sum b) over the per-block partials, in fixed order.
__global__ void noalloc_eta_kernel(const double* __restrict__ partial, int nblocks, double* __restrict__ eta)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nblocks; ++i) {
        a += partial[2 * i + 0];
        b += partial[2 * i + 1];
    }
    *eta = (b > 0.0) ? sqrt(a) / sqrt(b) : nan("");
}

}  // namespace

namespace {
template <typename To, typename From>
int convert_array(const From* in, To* out, long long n, void* stream)
{
    if (n < 0) return set_err(GF_ERR_ARG, "n < 0");
    if (n == 0) return GF_OK;
    if (!in || !out) return set_err(GF_ERR_ARG, "null pointer");
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long blocks = std::min<long long>((n + 255) / 256, 8LL * sms);
    gf::convert_kernel<To, From><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(in, out, n);
    CK(cudaGetLastError());
    return GF_OK;
}
}  // namespace

extern "C" int gf_round_to_f32(const double* in, float* out, long long n, void* stream)
{
    return convert_array<float, double>(in, out, n, stream);
}

extern "C" int gf_widen_to_f64(const float* in, double* out, long long n, void* stream)
{
    return convert_array<double, float>(in, out, n, stream);
}

extern "C" int gf_true_residual_noalloc(int nx, int ny, int nz, double h, double E0, double nu,
                                        const double* rho_hat, double p, double rho_min, const double* f,
                                        const double* u, double* eta, void* stream)
{
    if (!rho_hat || !f || !u || !eta) return set_err(GF_ERR_ARG, "null pointer");
    if (nx < 1 || ny < 2 || nz < 2 || (ny & 1) || (nz & 1)) return set_err(GF_ERR_ARG, "need nx>=1, even ny,nz >= 2");
    if (!(h > 0) || !(E0 > 0) || !(nu > -1.0 && nu < 0.5)) return set_err(GF_ERR_ARG, "h, E0 > 0, nu in (-1,0.5)");
    if (!(p >= 1.0 && p <= 16.0)) return set_err(GF_ERR_ARG, "p in [1,16]");
    if (!(rho_min > 0.0 && rho_min <= 1.0)) return set_err(GF_ERR_ARG, "rho_min in (0,1]");
    const long long nodes = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    const long long ndof = 3 * nodes, nel = (long long)nx * ny * nz;
    if (ndof > NOALLOC_MAX_DOF)
        return set_err(GF_ERR_ARG, "grid has " + std::to_string(ndof) +
                                       " DOFs; gf_true_residual_noalloc handles at most 1048576");
    double* scratch = nullptr;
    RET(noalloc_scratch(&scratch));
    double* E = scratch;                              // nel words
    double* Ku = scratch + NOALLOC_MAX_ELEM;          // ndof words
    double* partial = Ku + NOALLOC_MAX_DOF;           // 2 * NOALLOC_BLOCKS words
    cudaStream_t s = (cudaStream_t)stream;
    double K[576];
    build_k0(E0, nu, K);
    gf::K0Param<double> K0;
    for (int q = 0; q < 576; ++q) K0.k[q] = K[q];
    const int p_int = (p == std::floor(p)) ? (int)p : 0;
    const gf::GridDims d{nx, ny, nz};
    const int nb = (int)std::min<long long>(NOALLOC_BLOCKS, std::max<long long>(1, (ndof + 1023) / 1024));
    // every word read below is written first in this call, so nothing is cleared
    gf::modulus_fp64_kernel<<<nblk(nel), 256, 0, s>>>(rho_hat, E, nel, rho_min, p, p_int, h);
    CK(cudaGetLastError());
    gf::node_stencil_kernel<double, double, gf::ST_APPLY, double, double><<<nblk(nodes), 256, 0, s>>>(
        u, (const double*)nullptr, Ku, E, d, K0, 0.0, (const int*)nullptr);
    CK(cudaGetLastError());
    gf::residual_norms_kernel<<<nb, gf::RED_THREADS, 0, s>>>(f, Ku, nullptr, ndof, nx + 1, partial, 0, nullptr, nullptr);
    CK(cudaGetLastError());
    noalloc_eta_kernel<<<1, 32, 0, s>>>(partial, nb, eta);
    CK(cudaGetLastError());
    return GF_OK;
}

#include "mlp.cuh"
#include "batch.cuh"
