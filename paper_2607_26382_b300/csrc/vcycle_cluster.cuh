// The coarse part of the FP32 V-cycle in one launch: a cluster of CTAs runs every
// level from l0 (a few thousand nodes or fewer) down to the coarsest solve and
// back up, with a hardware cluster barrier between the stages instead of one
// kernel launch per stage. Same per-node arithmetic as the level kernels
// (stencil_node, first_sweep_node, restrict_node, prolong_node), and the coarsest
// solve is the FP64 dense inverse applied one warp per row.
#pragma once
#include <cooperative_groups.h>

namespace gf {

constexpr int VC_CLUSTER = 8, VC_THREADS = 512, VC_MAXL = 8;

struct VcLevel {
    GridDims d;
    long long nodes;
    const float* E;
    float *b, *x, *t, *r;
};

struct VcArgs {
    VcLevel lv[VC_MAXL];
    int l0, L, nu1, nu2, nc;
    float omega;
    const double* Ainv;
    const int* halt;
};

__global__ void __cluster_dims__(VC_CLUSTER, 1, 1) __launch_bounds__(VC_THREADS)
coarse_vcycle_kernel(const __grid_constant__ VcArgs a, const __grid_constant__ K0Param<float> K0)
{
    namespace cg = cooperative_groups;
    if (a.halt != nullptr && *a.halt != 0) return;   // uniform over the cluster
    cg::cluster_group cl = cg::this_cluster();
    const long long tid = (long long)cl.block_rank() * VC_THREADS + threadIdx.x;
    const long long nthr = (long long)VC_CLUSTER * VC_THREADS;
    // a level's iterate after its down-sweeps sits in x or t by the parity of the
    // nu1 - 1 buffer swaps, after its up-sweeps by the parity of nu1 - 1 + nu2
    const bool down_odd = ((a.nu1 - 1) & 1) != 0, up_odd = ((a.nu1 - 1 + a.nu2) & 1) != 0;
    for (int l = a.l0; l < a.L - 1; ++l) {
        const VcLevel& v = a.lv[l];
        for (long long n = tid; n < v.nodes; n += nthr) first_sweep_node<float, float, float>(n, v.b, v.x, v.E, v.d, K0, a.omega);
        cl.sync();
        float *x = v.x, *t = v.t;
        for (int s = 1; s < a.nu1; ++s) {
            for (long long n = tid; n < v.nodes; n += nthr)
                stencil_node<float, float, ST_SWEEP, float, float>(n, x, v.b, t, v.E, v.d, K0, a.omega);
            cl.sync();
            float* q = x;
            x = t;
            t = q;
        }
        for (long long n = tid; n < v.nodes; n += nthr)
            stencil_node<float, float, ST_RESID, float, float>(n, x, v.b, v.r, v.E, v.d, K0, a.omega);
        cl.sync();
        const VcLevel& c = a.lv[l + 1];
        for (long long n = tid; n < c.nodes; n += nthr) restrict_node<float>(n, v.r, c.b, c.d);
        cl.sync();
    }
    {   // coarsest: x = Ainv b, FP64 accumulation, one warp per row
        const VcLevel& c = a.lv[a.L - 1];
        const int lane = threadIdx.x & 31;
        const long long warp = tid >> 5, nwarps = nthr >> 5;
        for (long long row = warp; row < a.nc; row += nwarps) {
            const double* Ar = a.Ainv + row * a.nc;
            double s = 0.0;
            for (int col = lane; col < a.nc; col += 32) s = fma(Ar[col], (double)c.b[col], s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) c.x[row] = (float)s;
        }
        cl.sync();
    }
    for (int l = a.L - 2; l >= a.l0; --l) {
        const VcLevel& v = a.lv[l];
        float *x = down_odd ? v.t : v.x, *t = down_odd ? v.x : v.t;
        const VcLevel& c = a.lv[l + 1];
        const float* xc = (l + 1 == a.L - 1) ? c.x : (up_odd ? c.t : c.x);
        for (long long n = tid; n < v.nodes; n += nthr) prolong_node<float, float>(n, x, xc, v.d);
        cl.sync();
        for (int s = 0; s < a.nu2; ++s) {
            for (long long n = tid; n < v.nodes; n += nthr)
                stencil_node<float, float, ST_SWEEP, float, float>(n, x, v.b, t, v.E, v.d, K0, a.omega);
            cl.sync();
            float* q = x;
            x = t;
            t = q;
        }
    }
}

}  // namespace gf
