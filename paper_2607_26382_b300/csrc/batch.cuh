// Batched frozen states (included at the end of gf_lib.cu; same translation unit).
//
// Many independent states of uneven size run Algorithm 1 together. Each FGMRES
// step j for the whole batch is ONE CUDA graph: the per-state chains (V-cycle, FP64
// K*z, CGS2, Givens tail) are captured on forked streams inside a single capture,
// so the GPU runs them concurrently. A per-state skip flag makes the chains of
// states that have finished (or sit out a phase) exit at once, so the same graphs
// serve every phase of the policy. The per-state decisions (probe features, rule,
// guard, next floor) are the single-state ones, applied state by state. The
// coarsest inverses of all states are built with Gauss-Jordan pivots in lockstep.
// Node-stencil block sizes are chosen per grid shape by timing (autotuner).
#pragma once

namespace gf {

struct BatchTables {
    KState** st;       // per state
    double** hist;
    double** A;        // coarsest dense matrices (the inverses, in the end)
    double** W;        // their second Gauss-Jordan buffers
    int* n;            // coarsest sizes
    int* m;            // coarsest free-DOF counts (the symmetric sweep's size)
    int** pos;         // coarsest free-DOF positions (gf_grid::cpos)
    int* band;         // coarsest operator bands (gf_grid::cband)
    LdlState* ldl;     // the states' LDL^T inverse buffers (ldl_state)
};

__global__ void batch_mark_kernel(KState** st, const int* __restrict__ active, int B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B || active[i]) return;
    st[i]->skip = 1;
    st[i]->status = KS_STOP;
}

// After a cycle end: a state that is no longer running sits out the next cycles,
// so its (already applied) update is not repeated.
__global__ void batch_retire_kernel(KState** st, int B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    if (!st[i]->skip && st[i]->status != KS_RUN) st[i]->skip = 1;
}

// out[4i..4i+3] = status, k, history[min(a,k)], history[min(b,k)]
__global__ void batch_gather_kernel(KState* const* st, double* const* hist, int B, int a, int b,
                                    double* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    const int k = st[i]->k;
    out[4 * i + 0] = (double)st[i]->status;
    out[4 * i + 1] = (double)k;
    out[4 * i + 2] = hist[i][a < k ? a : k];
    out[4 * i + 3] = hist[i][b < k ? b : k];
}

__global__ void batch_abort_kernel(KState** st, const int* __restrict__ abort_flags, int B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B || !abort_flags[i]) return;
    st[i]->status = KS_STOP;
    st[i]->flag = 3;
    st[i]->skip = 1;
}

// Gauss-Jordan step s (pivots 2s, 2s+1) on every state's matrix at once
// (blockIdx.z = state, tiles of GJ_T). State i runs ceil(n_i/2) steps; it starts in
// W_i when that count is odd, so its last step always writes A_i.
__global__ void __launch_bounds__(GJ_T * GJ_R)
batch_gj_step_kernel(BatchTables t, const int* __restrict__ active, int s)
{
    const int i = blockIdx.z;
    if (!active[i]) return;
    const int n = t.n[i], k = 2 * s;
    const int p0 = blockIdx.y * GJ_T, q0 = blockIdx.x * GJ_T;
    if (k >= n || p0 >= n || q0 >= n) return;   // uniform over the block
    const int steps = (n + 1) / 2;
    const bool from_w = ((steps & 1) ^ (s & 1)) != 0;
    gj_tile(from_w ? t.W[i] : t.A[i], from_w ? t.A[i] : t.W[i], n, k, p0, q0);
}

// The blocked symmetric sweep (sym_gj_kernel) on every state's free-DOF matrix at once:
// step s takes pivots SGJ_B*s .. SGJ_B*s + SGJ_B - 1. State i runs ceil(m_i/SGJ_B) steps
// and starts in A_i when that count is odd, so its last step writes the upper triangle
// (m_i x m_i) into W_i, as for one grid. The P buffers of state i sit past its full
// second matrix buffer, W_i + n_i^2. Grid: (1 + tiles (tiles + 1) / 2, 1, B), tiles the
// largest of the states' active tile counts at this step (sgj_active); block 0 forms the
// next P, the others one upper tile (states skip the tiles past their own bound).
__device__ __forceinline__ bool batch_sym_from_w(int m, int s)
{
    return (((m + SGJ_B - 1) / SGJ_B + s) & 1) == 0;
}

__global__ void __launch_bounds__(256)
batch_sym_gj_kernel(BatchTables t, const int* __restrict__ active, int s, int tiles)
{
    const int i = blockIdx.z;
    if (!active[i]) return;
    const int m = t.m[i], k = SGJ_B * s;
    if (k >= m) return;
    const bool from_w = batch_sym_from_w(m, s);
    const double* Min = from_w ? t.W[i] : t.A[i];
    double* Pb = t.W[i] + (long long)t.n[i] * t.n[i];
    if (blockIdx.x == 0) {   // the next pivot block's P, as sym_gj_kernel
        sym_gj_next_p(Min, m, k, Pb + SGJ_B * SGJ_B * (s & 1), Pb + SGJ_B * SGJ_B * ((s + 1) & 1));
        return;
    }
    int tp, tq;   // upper tiles of the leading tiles x tiles, as sym_gj_kernel
    sgj_upper_tile((int)blockIdx.x - 1, tiles, tp, tq);
    if (tq * SGJ_T >= sgj_active(m, k, t.band[i])) return;   // uniform over the block (tp <= tq)
    sym_gj_tile(Min, from_w ? t.A[i] : t.W[i], m, k, tp, tq, Pb + SGJ_B * SGJ_B * (s & 1));
}

// P of every active state's first pivot block (from the start buffer of its sweep).
__global__ void __launch_bounds__(256) batch_sym_gj_first_kernel(BatchTables t, const int* __restrict__ active)
{
    const int i = blockIdx.x;
    if (!active[i]) return;
    const int m = t.m[i];
    if (m == 0) return;
    const double* M = batch_sym_from_w(m, 0) ? t.W[i] : t.A[i];
    __shared__ double S[SGJ_B][SGJ_B];
    const int tid = threadIdx.x, bb = min(SGJ_B, m);
    const int bi = tid / SGJ_B, bj = tid % SGJ_B;
    if (tid < SGJ_B * SGJ_B && bi < bb && bj < bb) S[bi][bj] = M[(long long)min(bi, bj) * m + max(bi, bj)];
    __syncthreads();
    sgj_invert_block(S, bb, tid);
    if (tid < SGJ_B * SGJ_B) t.W[i][(long long)t.n[i] * t.n[i] + tid] = (bi < bb && bj < bb) ? S[bi][bj] : 0.0;
}

// The active states' full inverses A_i from their free-DOF sweeps in W_i (sym_expand).
__global__ void batch_sym_expand_kernel(BatchTables t, const int* __restrict__ active)
{
    const int i = blockIdx.y;
    if (!active[i]) return;
    sym_expand(t.W[i], t.m[i], t.pos[i], t.A[i], t.n[i], (long long)blockIdx.x * blockDim.x + threadIdx.x,
               (long long)gridDim.x * blockDim.x);
}

}  // namespace gf

struct gf_batch {
    int B = 0, L = 0, device = 0, sms = 0;
    cudaStream_t stream = nullptr;
    std::vector<gf_grid*> g;
    std::vector<double*> f, u;
    std::vector<cudaStream_t> cap;
    cudaStream_t capS = nullptr;
    cudaEvent_t evFork = nullptr;
    std::vector<cudaEvent_t> evJoin;
    cudaEvent_t ev[3] = {};
    // graphs over all states
    cudaGraphExec_t step[gf::KRY_MMAX] = {};
    cudaGraphExec_t start[2] = {};
    cudaGraphExec_t end = nullptr;
    long long nodes_step[gf::KRY_MMAX] = {}, nodes_start[2] = {}, nodes_end = 0;
    int key_prec = -1, key_nu1 = -1, key_nu2 = -1, key_m = -1, key_outer = -1, key_smoother = -1;
    double key_omega = -1.0;
    void* key_ptrs = nullptr;   // V of state 0 when captured (realloc invalidates)
    // device tables
    gf::BatchTables tab{};
    int* d_active = nullptr;
    int* d_abort = nullptr;
    double* gather_host = nullptr;   // mapped, 4 * B
    double* gather_dev = nullptr;
    int nc_max = 0;
    long long launches = 0;
};

namespace {

void batch_drop_graphs(gf_batch* b)
{
    for (int j = 0; j < gf::KRY_MMAX; ++j) {
        if (b->step[j]) cudaGraphExecDestroy(b->step[j]);
        b->step[j] = nullptr;
    }
    for (int q = 0; q < 2; ++q) {
        if (b->start[q]) cudaGraphExecDestroy(b->start[q]);
        b->start[q] = nullptr;
    }
    if (b->end) cudaGraphExecDestroy(b->end);
    b->end = nullptr;
}

// Capture per_state(i) for every state on its own forked stream into one graph.
template <class F>
int batch_capture(gf_batch* b, F per_state, cudaGraphExec_t* out, long long* nodes)
{
    std::vector<gf_stats> saved(b->B);
    long long count = 0;
    CK(cudaStreamBeginCapture(b->capS, cudaStreamCaptureModeThreadLocal));
    int rc = GF_OK;
    cudaError_t e = cudaEventRecord(b->evFork, b->capS);
    for (int i = 0; i < b->B && rc == GF_OK && e == cudaSuccess; ++i) {
        gf_grid* g = b->g[i];
        e = cudaStreamWaitEvent(b->cap[i], b->evFork, 0);
        if (e != cudaSuccess) break;
        saved[i] = g->stats;
        g->cur_stream = b->cap[i];
        rc = per_state(i);
        g->cur_stream = g->stream;
        count += g->stats.kernel_launches - saved[i].kernel_launches;
        g->stats = saved[i];
        if (rc == GF_OK) e = cudaEventRecord(b->evJoin[i], b->cap[i]);
        if (e == cudaSuccess && rc == GF_OK) e = cudaStreamWaitEvent(b->capS, b->evJoin[i], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->capS, &graph);
    if (rc != GF_OK || e != cudaSuccess || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (rc != GF_OK) return rc;
        return set_err(GF_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e != cudaSuccess ? e : ee));
    }
    const cudaError_t ei = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    CK(ei);
    *nodes = count;
    return GF_OK;
}

int batch_launch(gf_batch* b, cudaGraphExec_t ex, long long nodes)
{
    CK(cudaGraphLaunch(ex, b->stream));
    b->launches += nodes;
    return GF_OK;
}

int batch_graphs(gf_batch* b, const gf_solve_opts* o)
{
    const int m = o->restart;
    uintptr_t key = 0;
    for (gf_grid* g : b->g)
        key = key * 1000003u ^ (uintptr_t)g->V ^ ((uintptr_t)g->Z << 1) ^ ((uintptr_t)g->hist << 2);
    void* ptr0 = (void*)key;
    if (b->key_prec != o->prec || b->key_nu1 != o->nu1 || b->key_nu2 != o->nu2 || b->key_omega != o->omega ||
        b->key_m != m || b->key_ptrs != ptr0 || b->key_outer != o->outer || b->key_smoother != o->smoother) {
        batch_drop_graphs(b);
        b->key_outer = o->outer;
        b->key_smoother = o->smoother;
        b->key_prec = o->prec;
        b->key_nu1 = o->nu1;
        b->key_nu2 = o->nu2;
        b->key_omega = o->omega;
        b->key_m = m;
        b->key_ptrs = ptr0;
    }
    for (int first = 0; first < 2; ++first)
        if (!b->start[first])
            RET(batch_capture(b, [&](int i) { return cycle_start(b->g[i], b->f[i], b->u[i], first == 1, first == 1, o->outer); },
                              &b->start[first], &b->nodes_start[first]));
    for (int j = 0; j < m; ++j)
        if (!b->step[j])
            RET(batch_capture(b, [&](int i) { return arnoldi_step(b->g[i], j, o); }, &b->step[j], &b->nodes_step[j]));
    if (!b->end)
        RET(batch_capture(b,
                          [&](int i) {
                              gf_grid* g = b->g[i];
                              LAUNCH(g, 1, 1, gf::backsolve_kernel, g->st);
                              LAUNCH(g, 2 * g->sms, 256, gf::update_x_kernel, b->u[i], (const double*)g->Z, g->ldk,
                                     g->ndof, (const gf::KState*)g->st);
                              return GF_OK;
                          },
                          &b->end, &b->nodes_end));
    return GF_OK;
}

int batch_tables(gf_batch* b)
{
    std::vector<gf::KState*> st(b->B);
    std::vector<double*> hist(b->B);
    for (int i = 0; i < b->B; ++i) {
        st[i] = b->g[i]->st;
        hist[i] = b->g[i]->hist;
    }
    CK(cudaMemcpy(b->tab.st, st.data(), sizeof(void*) * b->B, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->tab.hist, hist.data(), sizeof(void*) * b->B, cudaMemcpyHostToDevice));
    return GF_OK;
}

struct BatchOut {
    int k = 0, flag = 0, status = 0, first = 0;
    double r50 = 0.0, r100 = 0.0, stop_estimate = 0.0;
    bool decided = false, escalated = false;
    std::vector<double> hist;
};

// First floor for the listed states from their r50/r100: Eq. (trigger), or the MLP
// on all rows at once.
int batch_decide(gf_batch* b, const gf_policy* pol, const std::vector<int>& rows, std::vector<BatchOut>& out)
{
    if (rows.empty()) return GF_OK;
    const int nf = pol->n_ladder + 1;
    if (pol->selector == GF_SEL_MLP) {
        std::vector<double> feat(rows.size() * 6);
        for (size_t r = 0; r < rows.size(); ++r)
            RET(gf_select_features(b->g[rows[r]], out[rows[r]].r50, out[rows[r]].r100, &feat[6 * r]));
        std::vector<int> cls(rows.size());
        for (size_t r0 = 0; r0 < rows.size(); r0 += 4096) {
            const int n = (int)std::min<size_t>(4096, rows.size() - r0);
            RET(mlp_first_floors(pol->mlp, &feat[6 * r0], n, pol->mlp_confidence, nf, &cls[r0]));
        }
        for (size_t r = 0; r < rows.size(); ++r) out[rows[r]].first = cls[r];
    } else {
        for (int i : rows) out[i].first = gf_trigger_rule(out[i].r50, out[i].r100, pol) ? 1 : 0;
    }
    for (int i : rows) out[i].escalated = out[i].first > 0;
    return GF_OK;
}

// One lockstep FGMRES solve of the active states from u = 0. probe_at > 0: at that
// step, states still running get their r50/r100 read and the rule applied;
// escalated states are stopped (their iterate is discarded).
int batch_solve(gf_batch* b, const gf_solve_opts* o, const std::vector<int>& active, int probe_at,
                const gf_policy* pol, std::vector<BatchOut>& out)
{
    const int B = b->B, m = o->restart;
    for (int i = 0; i < B; ++i) {
        RET(ensure_krylov(b->g[i], m, std::max(o->kmax, probe_at), o->outer));
        if (o->smoother == 1 && active[i]) RET(ensure_cheb(b->g[i], o->prec));
    }
    RET(batch_tables(b));
    RET(batch_graphs(b, o));
    CK(cudaMemcpyAsync(b->d_active, active.data(), sizeof(int) * B, cudaMemcpyHostToDevice, b->stream));
    for (int i = 0; i < B; ++i) {
        gf_grid* g = b->g[i];
        if (!active[i]) continue;
        CK(cudaMemsetAsync(b->u[i], 0, sizeof(double) * g->ndof, b->stream));
        LAUNCH(g, 1, 1, init_state_kernel, g->st, o->kmax, m, o->tol);
        *g->host_status = gf::KS_RUN;
    }
    LAUNCH(b->g[0], (B + 127) / 128, 128, gf::batch_mark_kernel, b->tab.st, (const int*)b->d_active, B);
    CK(cudaStreamSynchronize(b->stream));
    std::vector<int> aborted(B, 0), decided(B, 0);
    out.assign(B, BatchOut());
    auto any_running = [&]() {
        for (int i = 0; i < B; ++i)
            if (active[i] && !aborted[i] && *(volatile int*)b->g[i]->host_status == gf::KS_RUN) return true;
        return false;
    };
    long long launched = 0;
    bool first = true;
    for (int cycle = 0;; ++cycle) {
        RET(batch_launch(b, b->start[first ? 1 : 0], b->nodes_start[first ? 1 : 0]));
        first = false;
        CK(cudaStreamSynchronize(b->stream));
        if (!any_running()) break;
        for (int j = 0; j < m; ++j) {
            RET(batch_launch(b, b->step[j], b->nodes_step[j]));
            ++launched;
            CK(cudaEventRecord(b->ev[j % 3], b->stream));
            if (probe_at > 0 && launched == probe_at) {
                LAUNCH(b->g[0], (B + 127) / 128, 128, gf::batch_gather_kernel, (gf::KState* const*)b->tab.st,
                       (double* const*)b->tab.hist, B, pol->checkpoint_a, pol->checkpoint_b, b->gather_dev);
                CK(cudaStreamSynchronize(b->stream));
                std::vector<int> ab(B, 0), rows;
                bool any_ab = false;
                for (int i = 0; i < B; ++i) {
                    if (!active[i] || (int)b->gather_host[4 * i] != gf::KS_RUN) continue;
                    decided[i] = 1;
                    out[i].decided = true;
                    out[i].r50 = b->gather_host[4 * i + 2];
                    out[i].r100 = b->gather_host[4 * i + 3];
                    rows.push_back(i);
                }
                RET(batch_decide(b, pol, rows, out));
                for (int i : rows) {
                    if (out[i].escalated) {
                        ab[i] = aborted[i] = 1;
                        any_ab = true;
                    }
                }
                if (any_ab) {
                    CK(cudaMemcpyAsync(b->d_abort, ab.data(), sizeof(int) * B, cudaMemcpyHostToDevice, b->stream));
                    LAUNCH(b->g[0], (B + 127) / 128, 128, gf::batch_abort_kernel, b->tab.st, (const int*)b->d_abort, B);
                }
            }
            if (j >= 1) {
                CK(cudaEventSynchronize(b->ev[(j - 1) % 3]));
                if (!any_running()) break;
            }
        }
        RET(batch_launch(b, b->end, b->nodes_end));
        LAUNCH(b->g[0], (B + 127) / 128, 128, gf::batch_retire_kernel, b->tab.st, B);
        LAUNCH(b->g[0], (B + 127) / 128, 128, gf::batch_gather_kernel, (gf::KState* const*)b->tab.st,
               (double* const*)b->tab.hist, B, 0, 0, b->gather_dev);
        CK(cudaStreamSynchronize(b->stream));
        bool run = false;
        for (int i = 0; i < B; ++i)
            if (active[i] && !aborted[i] && (int)b->gather_host[4 * i] == gf::KS_RUN) run = true;
        if (!run) break;
    }
    for (int i = 0; i < B; ++i) {
        if (!active[i]) continue;
        gf_grid* g = b->g[i];
        HostState hs{};
        RET(read_state(g, &hs));
        out[i].k = hs.k;
        out[i].flag = hs.flag;
        out[i].status = hs.status;
        out[i].hist.resize((size_t)hs.k + 1);
        CK(cudaMemcpy(out[i].hist.data(), g->hist, sizeof(double) * (hs.k + 1), cudaMemcpyDeviceToHost));
        out[i].stop_estimate = out[i].hist[hs.k];
    }
    return GF_OK;
}

// Set the floor of the active states: moduli and hierarchy per state, then the
// coarsest inverses: each state's banded LDL^T inverse (the default, as one grid's), or
// the sweeps with lockstep pivots over the batch.
int batch_set_floor(gf_batch* b, const std::vector<int>& active, const std::vector<double>& rho_min)
{
    const int B = b->B;
    if (b->g[0]->coarse_ldl) {   // the banded LDL^T inverse, every state's steps in one launch
        int steps = 0;
        for (int i = 0; i < B; ++i) {
            if (!active[i]) continue;
            gf_grid* g = b->g[i];
            g->skip_coarse_inverse = true;
            const int rc = gf_set_floor(g, rho_min[i]);
            g->skip_coarse_inverse = false;
            if (rc != GF_OK) return rc;
            RET(assemble_coarse_free(g, g->Ainv));
            steps = std::max(steps, (g->ncf + gf::LDL_C - 1) / gf::LDL_C);
        }
        CK(cudaMemcpyAsync(b->d_active, active.data(), sizeof(int) * B, cudaMemcpyHostToDevice, b->stream));
        if (!ldl_smem_opt_in()) return set_err(GF_ERR_CUDA, "shared memory of the LDL^T inverse kernels");
        auto launch = [&](auto kern, int ctas, int threads, size_t smem, int s) -> int {
            if (ctas <= 0) return GF_OK;
            kern<<<dim3((unsigned)ctas, 1, (unsigned)B), threads, smem, b->stream>>>(
                (const gf::LdlState*)b->tab.ldl, (const int*)b->d_active, s);
            b->launches += 1;
            CK(cudaGetLastError());
            return GF_OK;
        };
        for (int s = 0; s < steps; ++s) {   // A = L D L^T, block s of every state
            int panel = 0, upd = 0;
            for (int i = 0; i < B; ++i) {
                int j0, c, r1;
                if (!active[i] || !gf::ldl_factor_step(b->g[i]->ncf, b->g[i]->cband, s, j0, c, r1)) continue;
                if (j0 + c >= b->g[i]->ncf) continue;
                panel = std::max(panel, gf::ldl_panel_ctas(j0 + c, r1));
                upd = std::max(upd, gf::ldl_update_ctas(j0 + c, r1));
            }
            RET(launch(gf::ldl_diag_batch_kernel, 1, 512, 0, s));
            RET(launch(gf::ldl_panel_batch_kernel, panel, gf::LDL_WARPS * 32, 0, s));
            RET(launch(gf::ldl_update_batch_kernel, upd, 256, 0, s));
        }
        for (int s = 0; s < steps; ++s) {   // Z = A^-1, last blocks first
            int rows = 0, cmax = 0;
            size_t rsm = 0, dsm = 0;
            for (int i = 0; i < B; ++i) {
                int j0, c, kend;
                const int m = b->g[i]->ncf;
                if (!active[i] || !gf::ldl_inverse_step(m, b->g[i]->cband, s, j0, c, kend)) continue;
                cmax = std::max(cmax, c);
                dsm = std::max(dsm, gf::ldl_diag_smem(kend - j0 - c));
                if (j0 + c < m) {
                    rows = std::max(rows, gf::ldl_rows_ctas(m, j0 + c));
                    rsm = std::max(rsm, gf::ldl_rows_smem(kend - j0 - c));
                }
            }
            if (rsm > 200 * 1024) return set_err(GF_ERR_ARG, "coarsest band too wide for the LDL^T inverse");
            RET(launch(gf::ldl_inv_rows_batch_kernel, rows, gf::LDL_WARPS * 32, rsm, s));
            RET(launch(gf::ldl_inv_diag_batch_kernel, cmax, gf::LDL_WARPS * 32, dsm, s));
            RET(launch(gf::ldl_inv_diag2_batch_kernel, gf::ldl_diag2_ctas(cmax), gf::LDL_WARPS * 32, 0, s));
        }
        gf::batch_sym_expand_kernel<<<dim3((unsigned)std::max(1, b->sms), B), 256, 0, b->stream>>>(b->tab, b->d_active);
        b->launches += 1;
        CK(cudaGetLastError());
        return GF_OK;
    }
    for (int i = 0; i < B; ++i) {
        if (!active[i]) continue;
        gf_grid* g = b->g[i];
        g->skip_coarse_inverse = true;
        const int rc = gf_set_floor(g, rho_min[i]);
        g->skip_coarse_inverse = false;
        if (rc != GF_OK) return rc;
        Level& c = g->lv[g->L - 1];
        const bool gal = g->coarse_kind == GF_COARSE_GALERKIN && g->L > 1;   // as build_coarse_inverse of one grid
        if (g->sym_gj) {   // the free-DOF matrix, in both buffers (as build_coarse_inverse of one grid)
            const long long m = g->ncf;
            for (double* buf : {g->Ainv, g->Agj}) {
                if (gal)
                    LAUNCH(g, nblk(m * m), 256, gf::gal_assemble_kernel, (const double*)c.Ke64, buf, c.dims(),
                           (const int*)g->cidx, (int)m);
                else
                    LAUNCH(g, nblk(m * m), 256, gf::coarse_assemble_kernel, (const double*)c.E64, buf, c.dims(),
                           g->K0d, (const int*)g->cidx, (int)m);
            }
            continue;
        }
        const long long n = g->nc;
        double* start = (((n + 1) / 2) & 1) ? g->Agj : g->Ainv;   // see batch_gj_step_kernel
        if (gal)
            LAUNCH(g, nblk(n * n), 256, gf::gal_assemble_kernel, (const double*)c.Ke64, start, c.dims(),
                   (const int*)nullptr, 0);
        else
            LAUNCH(g, nblk(n * n), 256, gf::coarse_assemble_kernel, (const double*)c.E64, start, c.dims(), g->K0d,
                   (const int*)nullptr, 0);
        LAUNCH(g, nblk(n * n), 256, gf::coarse_fix_kernel, start, c.dims());
    }
    CK(cudaMemcpyAsync(b->d_active, active.data(), sizeof(int) * B, cudaMemcpyHostToDevice, b->stream));
    int nmax = 0;
    for (int i = 0; i < B; ++i)
        if (active[i]) nmax = std::max(nmax, b->g[i]->nc);
    if (b->g[0]->sym_gj) {   // the single grid's algorithm, so that states stay bit-identical to it
        int mmax = 0;
        for (int i = 0; i < B; ++i)
            if (active[i]) mmax = std::max(mmax, b->g[i]->ncf);
        gf::batch_sym_gj_first_kernel<<<B, 256, 0, b->stream>>>(b->tab, b->d_active);
        b->launches += 1;
        CK(cudaGetLastError());
        for (int s = 0; gf::SGJ_B * s < mmax; ++s) {
            int ts = 1;   // the largest active tile count of the states still sweeping
            for (int i = 0; i < B; ++i)
                if (active[i] && gf::SGJ_B * s < b->g[i]->ncf)
                    ts = std::max(ts, (gf::sgj_active(b->g[i]->ncf, gf::SGJ_B * s, b->g[i]->cband) + gf::SGJ_T - 1) /
                                          gf::SGJ_T);
            gf::batch_sym_gj_kernel<<<dim3(1 + ts * (ts + 1) / 2, 1, B), dim3(16, 16), 0, b->stream>>>(
                b->tab, b->d_active, s, ts);
            b->launches += 1;
            CK(cudaGetLastError());
        }
        gf::batch_sym_expand_kernel<<<dim3((unsigned)std::max(1, b->sms), B), 256, 0, b->stream>>>(b->tab, b->d_active);
        b->launches += 1;
        CK(cudaGetLastError());
        return GF_OK;
    }
    const unsigned tiles = (unsigned)((nmax + gf::GJ_T - 1) / gf::GJ_T);
    for (int s = 0; 2 * s < nmax; ++s) {
        gf::batch_gj_step_kernel<<<dim3(tiles, tiles, B), dim3(gf::GJ_T, gf::GJ_R), 0, b->stream>>>(b->tab, b->d_active, s);
        b->launches += 1;
        CK(cudaGetLastError());
    }
    return GF_OK;
}

// Time the FP64 stencil at block sizes 64/128/256 and the FP32 one at 64/128/256,
// as the shared-memory-tiled kernel (0) and as the 27-neighbour gather kernel
// (-64/-128/-256), keeping the fastest of each.
int autotune_grid(gf_grid* g)
{
    if (!g->has_floor) return set_err(GF_ERR_STATE, "set_floor before autotuning");
    const int cand[7] = {64, 128, 256, 0, -64, -128, -256};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float* xf = reinterpret_cast<float*>(g->work);
    for (int prec = 0; prec < 2; ++prec) {
        float best = 1e30f;
        int pick = prec == 0 ? 256 : 0;
        for (int c : cand) {
            if (prec == 0 && c <= 0) continue;   // the tiled and 27-neighbour variants are FP32 only
            g->tpb[prec] = c;
            for (int rep = 0; rep < 4; ++rep) {
                if (rep == 1) CK(cudaEventRecord(e0, g->stream));
                if (prec == 0)
                    RET((stencil<double, double, gf::ST_APPLY>(g, 0, g->lv[0].x64, nullptr, g->lv[0].t64,
                                                                g->lv[0].E64, g->K0d, 0.0, nullptr)));
                else
                    RET((stencil<float, float, gf::ST_APPLY>(g, 0, g->lv[0].x32, nullptr, xf, g->lv[0].E32,
                                                              g->K0f, 0.0f, nullptr)));
            }
            CK(cudaEventRecord(e1, g->stream));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                pick = c;
            }
        }
        g->tpb[prec] = pick;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return GF_OK;
}

}  // namespace

extern "C" {

int gf_create_batch(int n_states, const int* dims, int levels, double h, double E0, double nu, void* stream,
                    gf_batch** out)
{
    if (!out || !dims || n_states < 1 || n_states > 4096) return set_err(GF_ERR_ARG, "n_states in [1,4096]");
    *out = nullptr;
    gf_batch* b = new gf_batch();
    b->B = n_states;
    b->L = levels;
    b->stream = (cudaStream_t)stream;
    auto fail = [&](int code) { gf_destroy_batch(b); return code; };
    if (cudaGetDevice(&b->device) != cudaSuccess) return fail(set_err(GF_ERR_CUDA, "cudaGetDevice"));
    for (int i = 0; i < n_states; ++i) {
        gf_grid* g = nullptr;
        const int rc = gf_create_grid(dims[3 * i], dims[3 * i + 1], dims[3 * i + 2], h, E0, nu, levels, stream, &g);
        if (rc != GF_OK) return fail(rc);
        b->g.push_back(g);
        double *f = nullptr, *u = nullptr;
        if (cudaMalloc(&f, sizeof(double) * g->ndof) != cudaSuccess ||
            cudaMalloc(&u, sizeof(double) * g->ndof) != cudaSuccess) {
            cudaFree(f);
            return fail(set_err(GF_ERR_OOM, "batch vectors"));
        }
        b->f.push_back(f);
        b->u.push_back(u);
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return fail(set_err(GF_ERR_CUDA, "stream"));
        b->cap.push_back(s);
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(set_err(GF_ERR_CUDA, "event"));
        b->evJoin.push_back(e);
        b->nc_max = std::max(b->nc_max, g->nc);
    }
    b->sms = b->g[0]->sms;
    if (cudaStreamCreateWithFlags(&b->capS, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->evFork, cudaEventDisableTiming) != cudaSuccess)
        return fail(set_err(GF_ERR_CUDA, "stream/event"));
    for (int q = 0; q < 3; ++q)
        if (cudaEventCreateWithFlags(&b->ev[q], cudaEventDisableTiming) != cudaSuccess)
            return fail(set_err(GF_ERR_CUDA, "event"));
    const size_t P = sizeof(void*) * n_states;
    if (cudaMalloc(&b->tab.st, P) != cudaSuccess || cudaMalloc(&b->tab.hist, P) != cudaSuccess ||
        cudaMalloc(&b->tab.A, P) != cudaSuccess || cudaMalloc(&b->tab.W, P) != cudaSuccess || cudaMalloc(&b->tab.n, sizeof(int) * n_states) != cudaSuccess ||
        cudaMalloc(&b->tab.m, sizeof(int) * n_states) != cudaSuccess || cudaMalloc(&b->tab.pos, P) != cudaSuccess ||
        cudaMalloc(&b->tab.band, sizeof(int) * n_states) != cudaSuccess ||
        cudaMalloc(&b->tab.ldl, sizeof(gf::LdlState) * n_states) != cudaSuccess ||
        cudaMalloc(&b->d_active, sizeof(int) * n_states) != cudaSuccess ||
        cudaMalloc(&b->d_abort, sizeof(int) * n_states) != cudaSuccess)
        return fail(set_err(GF_ERR_OOM, "batch tables"));
    if (cudaHostAlloc((void**)&b->gather_host, sizeof(double) * 4 * n_states, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&b->gather_dev, b->gather_host, 0) != cudaSuccess)
        return fail(set_err(GF_ERR_CUDA, "mapped gather"));
    std::vector<double*> A(n_states), W(n_states);
    std::vector<int*> pos(n_states);
    std::vector<int> n(n_states), m(n_states), band(n_states);
    std::vector<gf::LdlState> ldl(n_states);
    for (int i = 0; i < n_states; ++i) {
        ldl[i] = ldl_state(b->g[i]);
        A[i] = b->g[i]->Ainv;
        W[i] = b->g[i]->Agj;
        n[i] = b->g[i]->nc;
        m[i] = b->g[i]->ncf;
        band[i] = b->g[i]->cband;
        pos[i] = b->g[i]->cpos;
    }
    if (cudaMemcpy(b->tab.A, A.data(), P, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->tab.W, W.data(), P, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->tab.n, n.data(), sizeof(int) * n_states, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->tab.m, m.data(), sizeof(int) * n_states, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->tab.pos, pos.data(), P, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->tab.band, band.data(), sizeof(int) * n_states, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->tab.ldl, ldl.data(), sizeof(gf::LdlState) * n_states, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(set_err(GF_ERR_CUDA, "tables"));
    *out = b;
    return GF_OK;
}

int gf_destroy_batch(gf_batch* b)
{
    if (!b) return GF_OK;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop_graphs(b);
    for (gf_grid* g : b->g) gf_destroy_grid(g);
    for (double* p : b->f) cudaFree(p);
    for (double* p : b->u) cudaFree(p);
    for (cudaStream_t s : b->cap) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->evJoin) cudaEventDestroy(e);
    for (int q = 0; q < 3; ++q)
        if (b->ev[q]) cudaEventDestroy(b->ev[q]);
    if (b->evFork) cudaEventDestroy(b->evFork);
    if (b->capS) cudaStreamDestroy(b->capS);
    cudaFree(b->tab.st); cudaFree(b->tab.hist); cudaFree(b->tab.A); cudaFree(b->tab.W);
    cudaFree(b->tab.n); cudaFree(b->tab.m); cudaFree(b->tab.pos); cudaFree(b->tab.band); cudaFree(b->tab.ldl);
    cudaFree(b->d_active); cudaFree(b->d_abort);
    if (b->gather_host) cudaFreeHost(b->gather_host);
    delete b;
    return GF_OK;
}

int gf_batch_grid(gf_batch* b, int i, gf_grid** g)
{
    if (!b || !g || i < 0 || i >= b->B) return set_err(GF_ERR_ARG, "state index");
    *g = b->g[i];
    return GF_OK;
}

int gf_batch_set_state(gf_batch* b, int i, const double* rho_hat, double p, const double* f)
{
    if (!b || i < 0 || i >= b->B || !rho_hat || !f) return set_err(GF_ERR_ARG, "state index / null pointer");
    gf_grid* g = b->g[i];
    RET(set_device(g));
    RET(gf_set_density(g, rho_hat, p));
    CK(cudaMemcpyAsync(b->f[i], f, sizeof(double) * g->ndof, cudaMemcpyDeviceToDevice, b->stream));
    return GF_OK;
}

int gf_batch_solution(gf_batch* b, int i, double* u)
{
    if (!b || i < 0 || i >= b->B || !u) return set_err(GF_ERR_ARG, "state index / null pointer");
    CK(cudaMemcpyAsync(u, b->u[i], sizeof(double) * b->g[i]->ndof, cudaMemcpyDeviceToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return GF_OK;
}

int gf_batch_set_coarse_operator(gf_batch* b, int kind)
{
    if (!b) return set_err(GF_ERR_ARG, "null batch");
    for (gf_grid* g : b->g) RET(gf_set_coarse_operator(g, kind));
    batch_drop_graphs(b);   // the captured step graphs hold the other V-cycle
    b->key_prec = -1;
    return GF_OK;
}

int gf_batch_set_sm_share(gf_batch* b, int share)
{
    if (!b) return set_err(GF_ERR_ARG, "null batch");
    for (gf_grid* g : b->g) RET(gf_set_sm_share(g, share));
    batch_drop_graphs(b);   // the captured step graphs hold the other launch shapes
    b->key_prec = -1;
    return GF_OK;
}

int gf_batch_autotune(gf_batch* b, int* tpb_out)
{
    if (!b) return set_err(GF_ERR_ARG, "null batch");
    // one timing per distinct grid shape; states of the same shape share the pick
    std::vector<int> done(b->B, 0);
    for (int i = 0; i < b->B; ++i) {
        if (done[i]) continue;
        gf_grid* g = b->g[i];
        const bool had_density = g->has_density, had_floor = g->has_floor;
        const double old_floor = g->rho_min;
        if (!had_density) {
            // time on a placeholder field (all voids); the state is reset afterwards
            CK(cudaMemsetAsync(g->rho64, 0, sizeof(double) * g->nel, g->stream));
            CK(cudaMemsetAsync(g->rho16, 0, sizeof(__nv_bfloat16) * g->nel, g->stream));
            g->has_density = true;
        }
        if (!g->has_floor) RET(gf_set_floor(g, 1e-3));
        RET(autotune_grid(g));
        if (!had_density) {
            g->has_density = false;
            g->has_floor = false;
        } else if (!had_floor) {
            g->has_floor = false;
        } else {
            g->rho_min = old_floor;
        }
        for (int q = i; q < b->B; ++q)
            if (b->g[q]->nx == g->nx && b->g[q]->ny == g->ny && b->g[q]->nz == g->nz) {
                b->g[q]->tpb[0] = g->tpb[0];
                b->g[q]->tpb[1] = g->tpb[1];
                done[q] = 1;
            }
    }
    batch_drop_graphs(b);
    for (gf_grid* g : b->g) drop_graphs(g);
    if (tpb_out)
        for (int i = 0; i < b->B; ++i) {
            tpb_out[2 * i] = b->g[i]->tpb[0];
            tpb_out[2 * i + 1] = b->g[i]->tpb[1];
        }
    return GF_OK;
}

int gf_batch_select_floor(gf_batch* b, const gf_policy* pol, gf_select_info* infos)
{
    if (!b || !pol || !infos) return set_err(GF_ERR_ARG, "null pointer");
    if (pol->n_ladder < 0 || pol->n_ladder > GF_MAX_LADDER) return set_err(GF_ERR_ARG, "n_ladder");
    gf_solve_opts o = pol->solve;
    o.history = nullptr;
    o.tol = pol->tau;
    o.kmax = pol->kmax;
    for (gf_grid* gi : b->g)
        if (gi->geom != GF_GEOM_CANTILEVER) return set_err(GF_ERR_ARG, "the batch serves the cantilever only");
    RET(validate_opts(&o));
    if ((pol->selector == GF_SEL_RULE || pol->selector == GF_SEL_MLP) && pol->probe_iters > pol->kmax)
        return set_err(GF_ERR_ARG, "batched policy needs probe_iters <= kmax");
    if (pol->selector == GF_SEL_REUSE) return set_err(GF_ERR_ARG, "GF_SEL_REUSE is single-grid only");
    if (pol->true_check_every != 0) return set_err(GF_ERR_ARG, "true_check_every is single-grid only");
    if (pol->solve.ls_ratio != 0.0) return set_err(GF_ERR_ARG, "ls_ratio is single-grid only");
    if (pol->solve.fine_steps != 0) return set_err(GF_ERR_ARG, "fine_steps is single-grid only");
    if (pol->solve.coarse_steps != 0) return set_err(GF_ERR_ARG, "coarse_steps is single-grid only");
    const int B = b->B;
    for (int i = 0; i < B; ++i)
        if (!b->g[i]->has_density) return set_err(GF_ERR_STATE, "state " + std::to_string(i) + " has no density");
    CK(cudaSetDevice(b->device));
    double floors[GF_MAX_LADDER + 1];
    floors[0] = pol->rho0;
    for (int q = 0; q < pol->n_ladder; ++q) floors[q + 1] = pol->ladder[q];
    const int nf = pol->n_ladder + 1;
    std::vector<int> next(B, 0), done(B, 0);
    for (int i = 0; i < B; ++i) {
        std::memset(&infos[i], 0, sizeof(gf_select_info));
        infos[i].status = GF_NO_ADMISSIBLE_FLOOR;
        infos[i].floor_index = -1;
        infos[i].r50 = infos[i].r100 = infos[i].rho_min = infos[i].eta = std::nan("");
    }
    const bool rule = pol->selector == GF_SEL_RULE || pol->selector == GF_SEL_MLP;
    if (pol->selector == GF_SEL_MLP && !pol->mlp) return set_err(GF_ERR_ARG, "GF_SEL_MLP needs a trained gf_mlp");
    if (pol->selector == GF_SEL_GIVEN) {
        if (pol->first_index < 0 || pol->first_index >= nf) return set_err(GF_ERR_ARG, "first_index");
        for (int i = 0; i < B; ++i) {
            next[i] = pol->first_index;
            infos[i].escalated = pol->first_index > 0;
        }
    }
    for (int phase = 0;; ++phase) {
        std::vector<int> active(B, 0);
        std::vector<double> rm(B, 0.0);
        bool any = false;
        for (int i = 0; i < B; ++i)
            if (!done[i] && next[i] < nf) {
                active[i] = 1;
                rm[i] = floors[next[i]];
                any = true;
            }
        if (!any) break;
        RET(batch_set_floor(b, active, rm));
        const bool probe_phase = rule && phase == 0;
        gf_solve_opts so = o;
        if (probe_phase) so.kmax = std::max(o.kmax, pol->probe_iters);
        std::vector<BatchOut> res;
        RET(batch_solve(b, &so, active, probe_phase ? pol->probe_iters : 0, pol, res));
        for (int i = 0; i < B; ++i) {
            if (!active[i]) continue;
            gf_select_info& inf = infos[i];
            if (probe_phase) {
                if (res[i].decided) {
                    inf.probe_iters_run = pol->probe_iters;
                } else {
                    inf.probe_iters_run = std::min(res[i].k, pol->probe_iters);
                    RET(gf_probe_features(res[i].hist.data(), res[i].k, pol, &res[i].r50, &res[i].r100));
                    RET(batch_decide(b, pol, std::vector<int>{i}, res));
                }
                inf.r50 = res[i].r50;
                inf.r100 = res[i].r100;
                inf.escalated = res[i].escalated;
                if (inf.escalated) {
                    next[i] = res[i].first;
                    continue;
                }
            }
            if (phase == 0 && pol->selector == GF_SEL_FULL && next[i] == 0)   // rho0 attempt's features
                RET(gf_probe_features(res[i].hist.data(), res[i].k, pol, &inf.r50, &inf.r100));
            // guard on the selected solve
            double eta = 0.0;
            gf_grid* g = b->g[i];
            RET(guard_impl(g, b->f[i], b->u[i], &eta));
            gf_attempt& a = inf.attempts[inf.n_attempts++];
            a.rho_min = rm[i];
            a.iters = res[i].k;
            a.flag = res[i].flag;
            a.stop_estimate = res[i].stop_estimate;
            a.eta = eta;
            a.accepted = eta <= pol->tau;
            if (a.accepted) {
                inf.status = GF_ACCEPTED;
                inf.floor_index = next[i];
                inf.rho_min = rm[i];
                inf.eta = eta;
                done[i] = 1;
            } else {
                next[i] += 1;
            }
        }
    }
    return GF_OK;
}

int gf_batch_stats(const gf_batch* b, long long* kernel_launches)
{
    if (!b || !kernel_launches) return set_err(GF_ERR_ARG, "null pointer");
    long long s = b->launches;
    for (gf_grid* g : b->g) s += g->stats.kernel_launches;
    *kernel_launches = s;
    return GF_OK;
}

}  // extern "C"
