/*
 * gf.h -- C ABI of the B300 guarded floor-selection state solver.
 *
 * The operation (arXiv 2607.26382): for a frozen density field rho_hat on a
 * structured nx*ny*nz grid of cubic 8-node hexahedra, solve the linear-elastic
 * state equation K(rho_min) u = f (Eq. frozen_operator, with the floor scaling
 * E_e = rho_min + (1 - rho_min) rho_hat_e^p of Eq. floor_scaling) by
 * right-preconditioned restarted FGMRES with a matrix-free geometric-multigrid
 * V-cycle (Table solver-config), accept a solution only if the recomputed FP64
 * true residual ||f - K u|| / ||f|| <= tau (Eq. relative_residual, Table
 * residual-semantics), and choose the floor with the probe -> ladder -> guard
 * policy of Algorithm 1 with the rule of Eq. (trigger).
 *
 * Conventions shared by every call
 *  - Node n(i,j,k) = i + (nx+1)*(j + (ny+1)*k); DOF 3n+c (x,y,z interleaved);
 *    element e = ex + nx*(ey + ny*ez). Vectors of length n_dof, element arrays of
 *    length n_elem.
 *  - Cantilever support: every DOF of the nodes on the x = 0 face is fixed. The
 *    operator acts on free DOFs; fixed entries of inputs are ignored and fixed
 *    entries of outputs are written as 0.
 *  - Unless a pointer is documented as "host", it is a DEVICE pointer on the
 *    device that was current at gf_create_grid, owned by the caller, and must
 *    stay valid until the call's work on the grid's stream has completed.
 *  - Every call is enqueued on the stream given to gf_create_grid. Calls that
 *    return a host value (gf_true_residual, gf_solve, gf_select_floor) block
 *    until that value is known. A grid is not thread-safe.
 *  - Every call returns GF_OK (0) or a negative GF_ERR_* code and never throws;
 *    gf_last_error() gives a message for the calling thread. Solver outcomes
 *    (not converged, no admissible floor) are NOT errors: they are reported in
 *    the info structs.
 */
#ifndef GF_H
#define GF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define GF_OK              0
#define GF_ERR_ARG        -1   /* bad argument (size, null pointer, unsupported grid) */
#define GF_ERR_OOM        -2   /* device allocation failed */
#define GF_ERR_CUDA       -3   /* a CUDA runtime call failed */
#define GF_ERR_NONFINITE  -4   /* NaN/Inf (or out-of-range density) in an input */
#define GF_ERR_TIMEOUT    -5   /* a bounded device wait gave up */
#define GF_ERR_STATE      -6   /* call order: density or floor not set yet */

/* precision of the V-cycle (Krylov vectors, outer K*u and guard are always FP64) */
#define GF_FP64   0   /* FP64 everywhere */
#define GF_MIXED  1   /* FP32 smoothers / transfers / level K*u with BF16-stored densities;
                         coarsest solve FP64 */

/* FGMRES stop flags (gf_solve_info.flag) */
#define GF_FLAG_CONVERGED  0   /* recorded residual (projected or cycle-start true) <= tol */
#define GF_FLAG_MAX_ITERS  1   /* budget kmax reached */
#define GF_FLAG_BREAKDOWN  2   /* h_{j+1,j} ~ 0 without convergence */

/* policy outcome (gf_select_info.status), Algorithm 1 */
#define GF_ACCEPTED            0
#define GF_NO_ADMISSIBLE_FLOOR 1

/* first-floor selectors */
#define GF_SEL_RULE   0   /* probe at rho0, Eq. (trigger) picks (rho0, ladder) or ladder */
#define GF_SEL_FULL   1   /* no probe: try rho0 then every ladder floor in order */
#define GF_SEL_GIVEN  2   /* no probe: start at first_index of (rho0, ladder...) */
#define GF_SEL_MLP    3   /* probe at rho0 (fused), a trained gf_mlp picks the first floor */
#define GF_SEL_REUSE  4   /* optimisation loop (the cost reduction the Discussion, "When is the
                             guarded policy worth its cost?", names and
                             leaves untested): attempt floor first_index -- the previous
                             iteration's decision -- with no probe; if the guard rejects it, run
                             GF_SEL_RULE from scratch (the rejected attempt is attempts[0]).
                             Requires n_ladder <= GF_MAX_LADDER-1; single grid only. */

#define GF_MAX_LADDER 8
#define GF_MAX_TRUE_CHECKS 16   /* true-residual checks recorded per probe */

typedef struct gf_grid gf_grid;
typedef struct gf_mlp gf_mlp;

typedef struct {
    int    restart;    /* FGMRES restart length m, in [1, 300]. Past 32 basis vectors the CGS2 passes
                          run over slices of 32 vectors. */
    int    kmax;       /* iteration budget (Arnoldi steps over all cycles) */
    double tol;        /* stop when the recorded relative residual <= tol */
    int    prec;       /* GF_FP64 or GF_MIXED */
    int    nu1, nu2;   /* pre/post node-block Jacobi sweeps (>= 1) */
    double omega;      /* Jacobi damping */
    double* history;   /* host, optional: receives history[0..iters] (length >= kmax+1) */
    int    outer;      /* outer (Krylov) arithmetic: 0 = native FP64 K*u and CGS2; 1 = split-integer
                          FP64-class K*u (gf_apply_K_split), native FP64 CGS2; 2 = split-integer
                          K*u and CGS2 in double-float arithmetic (FP32 instructions, ~48-bit
                          basis vectors; h, rotations and least squares stay FP64). Other values:
                          GF_ERR_ARG. The guard is always native FP64. */
    int    smoother;   /* V-cycle smoother: 0 = damped node-block Jacobi (nu sweeps, omega);
                          1 = Chebyshev semi-iteration of degree nu1 / nu2 on D_b^{-1} K over
                          [lambda_max/30, 1.1 lambda_max] (the Chebyshev smoother Table
                          solver-config names; degree and interval are this library's readings),
                          lambda_max of each level from 15 power iterations from ones on the
                          free DOFs, computed on first use after each gf_set_floor. */
    double ls_ratio;   /* 0 = plain coarse correction x += P x_c. theta > 0: the line-searched,
                          rejectable coarse correction of Table solver-config's adaptive preconditioner
                          on every level: with c = P x_c, r the level's residual before the correction
                          and q = K c, alpha = (c.r)/(c.q) (the energy-optimal step, computed from r),
                          kept (x += alpha c) iff alpha >= theta (this library's reading of the
                          acceptance ratio). Needs smoother 0 and >= 2 levels; single grid only. The
                          preconditioner is then iterate-dependent, which FGMRES allows. Errors:
                          GF_ERR_ARG for a negative or non-finite value. */
    int    fine_steps; /* 0 = off. k in [1, 32]: the fine-level adaptive correction of Table
                          solver-config after every V-cycle: k steps of an inner FGMRES(k) from d = 0
                          on K d = r (r = v - K z, z the V-cycle's output), preconditioned by the 3x3
                          node-block Jacobi operator, in the V-cycle's precision; z += d only if the
                          recomputed ||r - K d|| < ||r||. All on the device (inside the captured
                          steps). Single grid only. Other values: GF_ERR_ARG. */
    int    coarse_steps; /* 0 = off: the coarsest level is solved exactly (dense FP64 inverse).
                          k in [1, 32]: the coarse-level solve of Table solver-config instead, k
                          steps of an inner FGMRES(k) from 0 on the coarsest level's operator,
                          preconditioned by its 3x3 node-block Jacobi operator, in the V-cycle's
                          precision (on the device, inside the captured steps). Needs >= 2 levels;
                          the cluster V-cycle is not used with it. Single grid only. Other values:
                          GF_ERR_ARG. */
} gf_solve_opts;

typedef struct {
    int    iters;          /* Arnoldi steps taken */
    int    flag;           /* GF_FLAG_* */
    double stop_estimate;  /* last recorded history value */
} gf_solve_info;

typedef struct {
    double rho0;                       /* original floor */
    double ladder[GF_MAX_LADDER];      /* escalation ladder, increasing */
    int    n_ladder;
    double tau;                        /* acceptance tolerance on the true residual */
    int    kmax;                       /* budget of each selected solve */
    int    probe_iters;                /* probe budget (100 in the paper) */
    double r50_escalate;               /* Eq. (trigger): 1e-2 */
    double r100_stall;                 /* 1e-4 */
    double plateau_ratio;              /* 0.6 */
    int    checkpoint_a, checkpoint_b; /* 50, 100 */
    int    selector;                   /* GF_SEL_* */
    int    first_index;                /* for GF_SEL_GIVEN */
    int    fuse_probe;                 /* 1: read the probe features off the running solve at
                                          rho0 (bit-identical to a separate probe followed by an
                                          independent solve, because the solver is deterministic);
                                          0: run the probe and the rho0 solve separately */
    gf_solve_opts solve;               /* restart, prec, smoother (kmax/tol/history ignored) */
    gf_mlp* mlp;                       /* GF_SEL_MLP: trained selector (else ignored) */
    double mlp_confidence;             /* GF_SEL_MLP: 0 = start at the most probable floor; c in
                                          (0,1] = start at the highest floor k with
                                          P(first admissible floor >= k) >= c (k = 0 always
                                          qualifies), so the selector skips a floor only
                                          when confident that it fails */
    int    true_check_every;           /* GF_SEL_RULE (and GF_SEL_REUSE's fallback): 0 = off; c > 0 =
                                          true-residual checks during the probe, the checkpointed
                                          variant Sec. 4.1.1 leaves untested. After every probe step
                                          k with k % c == 0 that does not end the solve, the iterate
                                          is formed as at a cycle end and its FP64 guard residual
                                          eta_k recomputed beside the projected estimate history[k].
                                          probe_iters / c <= GF_MAX_TRUE_CHECKS. The solve itself is
                                          unchanged. */
    double true_check_ratio;           /* detector (this library's reading): fires when some
                                          eta_k > ratio * history[k]; a firing detector escalates
                                          like Eq. (trigger). Default 10. */
} gf_policy;

typedef struct {
    double rho_min;
    int    iters;
    int    flag;
    double stop_estimate;
    double eta;        /* recomputed FP64 true residual */
    int    accepted;
} gf_attempt;

typedef struct {
    int    status;          /* GF_ACCEPTED or GF_NO_ADMISSIBLE_FLOOR */
    int    floor_index;     /* index into (rho0, ladder...), -1 if none */
    double rho_min;
    double eta;
    double r50, r100;       /* probe features (NaN when no probe ran) */
    int    escalated;
    int    probe_iters_run;
    int    n_attempts;
    gf_attempt attempts[GF_MAX_LADDER + 1];
    int    n_true_checks;                        /* probe true-residual checks taken */
    int    true_check_k[GF_MAX_TRUE_CHECKS];     /* their steps */
    double true_check_est[GF_MAX_TRUE_CHECKS];   /* projected estimate history[k] */
    double true_check_eta[GF_MAX_TRUE_CHECKS];   /* recomputed FP64 guard residual of the step's iterate */
    int    true_check_fired;                     /* the detector escalated (1) or not (0) */
} gf_select_info;

typedef struct {
    long long kernel_launches;   /* kernels this library launched on the grid */
    long long apply_K_fp64;      /* fine-level FP64 operator applications */
    long long vcycles;           /* preconditioner applications */
} gf_stats;

/* ---- lifetime ---------------------------------------------------------------- */

/* Create a grid of nx*ny*nz cubic elements of edge h, Young's modulus E0 (solid),
 * Poisson ratio nu, and a `levels`-level hierarchy (level l has (nx,ny,nz)/2^l
 * elements of edge h*2^l). Requires nx, ny, nz divisible by 2^(levels-1), ny and
 * nz even, 1 <= levels <= 8, and the coarsest level at most 8192 DOFs. `stream` is
 * a cudaStream_t (NULL = legacy default stream). Allocates all level workspace.
 * Sec. 3.1 (Discretization), Table solver-config. */
int gf_create_grid(int nx, int ny, int nz, double h, double E0, double nu, int levels,
                   void* stream, gf_grid** out);
int gf_destroy_grid(gf_grid* g);

/* Sizes: any pointer may be NULL. */
int gf_grid_sizes(const gf_grid* g, int* n_dof, int* n_elem, int* n_nodes, int* levels);

/* ---- state ------------------------------------------------------------------- */

/* Store the floor-independent density rho_hat (n_elem doubles in [0,1], device)
 * and the SIMP exponent p; keeps an FP64 and a BF16 copy. GF_ERR_NONFINITE if an
 * entry is NaN/Inf or outside [0,1]. Invalidates the floor. Sec. 3.2. */
int gf_set_density(gf_grid* g, const double* rho_hat, double p);

/* Set the floor: E_e = rho_min + (1 - rho_min) rho_hat_e^p (Eq. floor_scaling, E0
 * scales it), coarse moduli = mean of the 8 children, and the FP64 inverse of the
 * coarsest operator (from the banded LDL^T factorisation of the SPD operator restricted
 * to the free DOFs, block by block; identity rows on fixed DOFs). 0 < rho_min <= 1. */
int gf_set_floor(gf_grid* g, double rho_min);

/* Coarse-level operators of the V-cycle, used from the next gf_set_floor on:
 * GF_COARSE_REDISCRETISED (default): every coarse level applies K0(h_l) with the mean of
 *   the 8 child moduli, matrix-free.
 * GF_COARSE_GALERKIN: K_{l+1} = P^T K_l P with the 2:1 trilinear prolongation P (Table
 *   solver-config), held as one dense 24x24 matrix per coarse element and summed from
 *   the 8 children's matrices; node-block Jacobi smoothing on it and the dense inverse of
 *   the assembled coarsest level. FP64 matrices from the FP64 moduli, and FP32 ones (the
 *   mixed V-cycle) from the BF16-density moduli. Jacobi and Chebyshev smoothing (its
 *   lambda_max from the assembled operators), the line-searched coarse correction and
 *   the coarse-level Krylov solve all apply the assembled operators; the batch keeps the
 *   default.
 * Switching clears the floor (gf_set_floor again before solving) and the captured steps.
 * Memory: 576 * (8 + 4) bytes per coarse element, plus FP64 scratch for two levels.
 * Errors: GF_ERR_ARG for an unknown kind. */
#define GF_COARSE_REDISCRETISED 0
#define GF_COARSE_GALERKIN      1
int gf_set_coarse_operator(gf_grid* g, int kind);

/* Launch shapes for a grid whose solves share the GPU with other grids' solves (streams
 * running at once, e.g. gf_select_floor_many). share = 0 (default): every kernel is sized
 * to fill the SMs, the fastest shapes for one solve alone. share = 1: the FP64 modal K*u
 * and the FP32 fine-level operator run 16x16-column tiles planned for one CTA per SM, and
 * the FP64 Gram-Schmidt passes half of their resident blocks (the update-and-dots pass in
 * 128-thread blocks), so each takes about half of an SM's registers and another grid's
 * kernel can run beside it: on B300 the FP64 kernels issue from a small fraction of the
 * SM's instruction slots and the FP32 V-cycle from the rest. Results do not depend on it
 * (the operator is bit-identical under every launch plan; the Gram-Schmidt sums change
 * their block partition, within rounding). Re-plans and re-times the modal kernels on the
 * level-0 buffers, so switching clears the floor (gf_set_floor again before solving) and
 * the captured steps; call it before gf_set_density's first solve, off any capture.
 * Errors: GF_ERR_ARG for share outside {0, 1}. */
int gf_set_sm_share(gf_grid* g, int share);

/* out[q] = in[q] rounded to binary32 (round to nearest, ties to even; subnormal results,
 * overflow to infinity, NaN kept quiet), and out[q] = in[q] widened exactly to binary64,
 * for q < n: the conversions the mixed V-cycle applies to its FP64 input and its FP32
 * result (Sec. 3.3, the mixed-precision preconditioner), computed in integer arithmetic
 * so that they stay off the FP64 pipe, bit for bit the IEEE 754 conversions. `in` and
 * `out` are device arrays of n elements that do not overlap; enqueued on `stream` (a
 * cudaStream_t, NULL = legacy default) of the current device, no synchronisation.
 * n = 0 does nothing. Errors: GF_ERR_ARG for n < 0 or a null pointer with n > 0,
 * GF_ERR_CUDA if the launch fails. */
int gf_round_to_f32(const double* in, float* out, long long n, void* stream);
int gf_widen_to_f64(const float* in, double* out, long long n, void* stream);

/* f = unit point load in -z at the node (nx, ny/2, nz/2) (n_dof doubles, device);
 * the cantilever of Table geometries. */
int gf_cantilever_load(gf_grid* g, double* f);

/* Supports of the grid (Table geometries), used from the next gf_set_floor on:
 * GF_GEOM_CANTILEVER (default): every DOF of the nodes on the face x = 0 fixed.
 * GF_GEOM_BRIDGE: every DOF fixed at the nodes (0, 0, k) and y and z fixed (a roller, free
 *   in x) at (nx, 0, k), for k in {0, nz/2, nz}: the bridge's supports at the two faces and
 *   the mid-plane of the depth, y up. Needs even nz. Coarse levels take the supports by
 *   injection: coarse node (I, J, K) fixes the components fine node (2^l I, 2^l J, 2^l K)
 *   fixes, so a mid-depth support leaves the levels where nz / 2^l is odd. Every operator,
 *   smoother, transfer and the coarsest inverse then read and write fixed components as 0
 *   from a per-node bit mask held per level (n_nodes bytes each).
 *   The bridge runs the default solver only: native FP64 Krylov (outer 0), node-block
 *   Jacobi smoothing, rediscretised coarse levels, no adaptive components; other options,
 *   gf_apply_K_split, gf_conditioning, Galerkin coarse operators and the batch return
 *   GF_ERR_ARG. Switching clears the floor and the captured steps.
 * Errors: GF_ERR_ARG for an unknown geometry or odd nz; GF_ERR_OOM. */
#define GF_GEOM_CANTILEVER 0
#define GF_GEOM_BRIDGE     1
int gf_set_geometry(gf_grid* g, int geometry);

/* f = the bridge's load (Table geometries): a unit pressure on the top face y = ny h,
 * pointing down (-y), as consistent nodal forces, -h^2/4 from each top face around a node
 * (the bilinear face integral of a uniform pressure; total -Lx Lz); 0 on the grid's fixed
 * DOFs. n_dof doubles, device. */
int gf_bridge_load(gf_grid* g, double* f);

/* mask[d] = 1 if DOF d is free, 0 if fixed (n_dof bytes, device). */
int gf_free_mask(gf_grid* g, uint8_t* mask);

/* ---- operator and preconditioner -------------------------------------------- */

/* y = K(rho_min) u on free DOFs, FP64 (Eq. frozen_operator), matrix-free. u, y:
 * n_dof doubles, must not alias. */
int gf_apply_K(gf_grid* g, const double* u, double* y);

/* The same FP64 operator evaluated without FP64 multiply-adds: K0 = s*M with an
 * integer matrix M (exists for nu = 0.3 and other Poisson ratios with a small
 * integer form; GF_ERR_ARG otherwise). Each node tile writes its u values on a
 * common exponent with 48 bits, cuts them into four 12-bit digits, forms M times
 * each digit slice exactly in FP32, recombines the slices and applies s*E_e in
 * double-float arithmetic. Error ~2^-44 of the tile's largest |u| times |M| (a few
 * bits above FP64 rounding). u, y: n_dof doubles, distinct. */
int gf_apply_K_split(gf_grid* g, const double* u, double* y);

/* Same operator in FP32 with the moduli computed from the BF16 density copy (the
 * V-cycle's fine-level operator in GF_MIXED). u, y: n_dof floats. */
int gf_apply_K_f32(gf_grid* g, const float* u, float* y);

/* z = B v: one V-cycle (nu1 pre / nu2 post node-block Jacobi sweeps with damping
 * omega, restriction = transpose of trilinear prolongation, FP64 coarsest solve)
 * in precision `prec`. v, z: n_dof doubles; fixed entries of v are ignored. */
int gf_vcycle(gf_grid* g, const double* v, double* z, int prec, int nu1, int nu2, double omega);
/* The V-cycle with the V-cycle options of a solve-options struct: prec, nu1, nu2, omega, smoother;
 * the other fields are ignored. Same buffers and errors as gf_vcycle. With smoother = 1
 * the first call after gf_set_floor computes the levels' lambda_max (enqueue it
 * outside any stream capture). */
int gf_vcycle_ex(gf_grid* g, const double* v, double* z, const gf_solve_opts* opts);
/* The Chebyshev smoother's lambda_max(D_b^{-1} K) estimate of levels 0 .. levels-2 for
 * the V-cycle of precision prec (GF_FP64 on the FP64 moduli, GF_MIXED on the FP32 ones
 * from the BF16 density) into lam (host, n >= levels-1 entries); computes them if
 * needed. Blocks. GF_ERR_STATE before gf_set_floor. */
int gf_chebyshev_lambda(gf_grid* g, int prec, double* lam, int n);

/* ---- solve, guard, policy ----------------------------------------------------- */

/* Right-preconditioned restarted FGMRES(m) with classical Gram-Schmidt plus one
 * re-orthogonalisation and Givens rotations, preconditioned by gf_vcycle. u holds
 * the initial guess on entry (fixed entries ignored) and the solution on exit.
 * History entry k is the cycle-start true residual at a cycle start and the
 * Givens-projected estimate otherwise (Table residual-semantics). */
int gf_solve(gf_grid* g, const double* f, double* u, const gf_solve_opts* opts,
             gf_solve_info* info);

/* *eta (host) = ||M(f - K u)||_2 / ||M f||_2 in FP64: the acceptance guard, one
 * operator application (Eq. relative_residual, Table residual-semantics). */
int gf_true_residual(gf_grid* g, const double* f, const double* u, double* eta);

/* Algorithm 1: probe at rho0 for probe_iters, candidate list from Eq. (trigger)
 * (or the selector), an independent solve from u = 0 at each candidate floor,
 * accept the first with eta <= tau. On GF_ACCEPTED u holds the accepted solution
 * and the grid's floor is the accepted floor; otherwise u holds the last attempt. */
int gf_select_floor(gf_grid* g, const double* f, double* u, const gf_policy* pol,
                    gf_select_info* info);

/* Algorithm 1 on n frozen states at once, one grid each: one host thread per grid runs
 * gf_select_floor(grids[i], f[i], u[i], pol, &info[i]) (host arrays of n device
 * pointers; info a host array of n). Grids created on distinct streams run concurrently
 * on the device, each state's work in order on its own stream, so one state's
 * latency-bound phases (coarse V-cycle levels, small reductions, the early launches of
 * the coarsest inverse) fill the SMs another state's leaves idle. The grids must be
 * distinct (GF_ERR_ARG otherwise) and each must have its density set. Returns GF_OK, or
 * the lowest-index failing grid's status with its message in gf_last_error; the other
 * grids' results are still written. Blocks until every grid is done. */
int gf_select_floor_many(int n, gf_grid* const* grids, const double* const* f, double* const* u,
                         const gf_policy* pol, gf_select_info* info);

/* ---- floor-conditioning diagnostic (Sec. 4.1.3) ------------------------------ */

/* Extreme eigenvalues of the free-DOF operator K(rho_min) of Eq. (frozen_operator) on a
 * one-level grid (levels == 1, at most 8192 DOFs: gf_set_floor then holds K's dense
 * FP64 inverse, built from its LDL^T factorisation). *lambda_max: `iters` Lanczos steps on K
 * (matrix-free FP64 operator); *lambda_min: 1 / the largest eigenvalue after `iters`
 * Lanczos steps on the dense inverse. Both start from the all-ones vector on the free
 * DOFs, re-orthogonalise against the two previous vectors, and take the extreme
 * eigenvalue of the tridiagonal matrix by bisection; they are lower/upper estimates
 * that converge from inside the spectrum. eta_direct (optional, needs f, device):
 * the FP64 guard residual of the direct solution u = K^{-1} f -- the attained
 * direct-solve residual the paper correlates with kappa * eps. Host outputs.
 * 2 <= iters <= 512. Errors: GF_ERR_STATE without levels == 1 or before
 * gf_set_floor; GF_ERR_NONFINITE if an estimate is not positive. */
int gf_conditioning(gf_grid* g, const double* f, int iters, double* lambda_min, double* lambda_max,
                    double* eta_direct);

/* The floor screen of Sec. 4.1.3 (host-only): with kappa ~ c / rho_min and c = kappa *
 * rho_min measured at rho_min, *rho_screen = c * eps / tau (eps = DBL_EPSILON, 2^-52):
 * floors below it have kappa * eps > tau, the region where the paper's reduced direct
 * solves stop reaching tau. Needs 0 < lambda_min <= lambda_max, rho_min > 0, tau > 0. */
int gf_conditioning_screen(double lambda_min, double lambda_max, double rho_min, double tau,
                           double* rho_screen);

/* ---- host-only policy logic (no device work; usable without a GPU) ----------- */

/* Defaults of Table solver-config / Eq. (trigger) with the given rho0 and ladder. */
void gf_policy_defaults(gf_policy* pol);
/* Eq. (trigger): 1 = escalate, 0 = preserve. */
int gf_trigger_rule(double r50, double r100, const gf_policy* pol);
/* r50 = history[min(a, k_stop)], r100 = history[min(b, k_stop)] (Sec. 3.4). */
int gf_probe_features(const double* history, int k_stop, const gf_policy* pol,
                      double* r50, double* r100);

/* ---- sensitivity (the optimisation loop's consumer of the solve) ------------- */

/* dc_e = -p (1 - rho_min) rho_hat_e^(p-1) u_e^T K0 u_e (Sec. 3.1), FP64, at the
 * grid's current floor. u: n_dof, dc: n_elem doubles. */
int gf_sensitivity(gf_grid* g, const double* u, double* dc);

/* ---- the optimisation loop around the solve (Sec. 3.1) --------------------------- */

/* Linear-hat density filter: xt_e = sum_e' w_ee' x_e' / sum_e' w_ee', with
 * w_ee' = max(0, r_min - |c_e - c_e'|) between element centres in cells (Sec. 3.1,
 * "linear-hat density filter of radius r_min"). x, xt: n_elem doubles, distinct.
 * 1 < r_min <= 8. */
int gf_filter(gf_grid* g, const double* x, double* xt, double r_min);
/* Its adjoint (chain rule of a sensitivity through the filter):
 * out_e' = sum_e w_ee' gs_e / sum_e'' w_ee''. */
int gf_filter_adjoint(gf_grid* g, const double* gs, double* out, double r_min);
/* Optimality-criteria update with move limit and bisection on the volume
 * multiplier (Sec. 3.1): xnew = clip(x sqrt(-dc / (lam dv)), max(0, x-move),
 * min(1, x+move)); lam bisected on [0, 1e9] until (l2-l1)/(l1+l2) <= 1e-3 (at most
 * 200 steps) so that mean(xnew) meets volfrac. All arrays n_elem doubles. */
int gf_oc_update(gf_grid* g, const double* x, const double* dc, const double* dv, double volfrac,
                 double move, double* xnew);
/* *c (host) = f^T u (Eq. to_problem's objective), FP64, fixed summation order. */
int gf_compliance(gf_grid* g, const double* f, const double* u, double* c);
/* One guarded SIMP-OC iteration on the design x (n_elem, in/out): rho_hat =
 * filter(x); gf_set_density(rho_hat, p); gf_select_floor (Algorithm 1) -> u,
 * info; if accepted: *compliance = f^T u, dc = gf_sensitivity, chain both dc and
 * the unit volume sensitivity through the filter adjoint, and x <- OC update.
 * If no floor is admissible, x is left unchanged and *compliance is NaN. */
int gf_oc_iteration(gf_grid* g, double* x, const double* f, double* u, const gf_policy* pol, double p,
                    double volfrac, double r_min, double move, gf_select_info* info, double* compliance);

/* ---- batched frozen states --------------------------------------------------- */

/* Many independent frozen states (grids of uneven size) run Algorithm 1 together.
 * Each FGMRES step of the whole batch is one CUDA graph holding one concurrent
 * chain per state; finished states drop out of the chains; decisions (probe
 * features, Eq. trigger, guard, next floor) are the single-state ones, per state.
 * dims: host array of 3*n_states ints (nx, ny, nz per state); every state shares
 * `levels`, h, E0, nu and `stream`. The batch owns each state's load f and
 * solution u (device). */
typedef struct gf_batch gf_batch;
int gf_create_batch(int n_states, const int* dims, int levels, double h, double E0, double nu,
                    void* stream, gf_batch** out);
int gf_destroy_batch(gf_batch* b);
/* The per-state grid (for sizes; do not destroy it). */
int gf_batch_grid(gf_batch* b, int i, gf_grid** g);
/* State i: density (n_elem doubles, device, copied) with exponent p, load f (n_dof, device, copied). */
int gf_batch_set_state(gf_batch* b, int i, const double* rho_hat, double p, const double* f);
/* Copy state i's current solution into u (n_dof doubles, device); blocks. */
int gf_batch_solution(gf_batch* b, int i, double* u);
/* Coarse-level operators of every state (as gf_set_coarse_operator for one grid):
 * GF_COARSE_REDISCRETISED (default) or GF_COARSE_GALERKIN. The lockstep coarsest
 * inverses then assemble each state's Galerkin coarsest operator, and every state's
 * result stays bit-identical to its single grid's. Drops the captured steps. */
int gf_batch_set_coarse_operator(gf_batch* b, int kind);
/* Launch shapes of every state's grid (as gf_set_sm_share for one grid): 1 = the half-SM
 * shapes, so that the states' chains, which the step graphs run concurrently, share the
 * SMs; 0 = full-SM shapes (default). Clears the floors and drops the captured steps.
 * Errors: GF_ERR_ARG for share outside {0, 1}. */
int gf_batch_set_sm_share(gf_batch* b, int share);
/* Autotuner: time the node stencils at 64/128/256 threads per block once per
 * distinct grid shape and keep the fastest (results do not depend on the pick).
 * tpb_out (host, optional): 2*n_states ints, [FP64, FP32] block size per state. */
int gf_batch_autotune(gf_batch* b, int* tpb_out);
/* Algorithm 1 on every state; infos: host array of n_states. The fused probe is
 * always used for GF_SEL_RULE (requires probe_iters <= kmax). */
int gf_batch_select_floor(gf_batch* b, const gf_policy* pol, gf_select_info* infos);
/* Kernels launched so far on the batch (graph nodes counted per replay). */
int gf_batch_stats(const gf_batch* b, long long* kernel_launches);

/* ---- learned first-floor selector (no counterpart in the paper; its analogue is
 *      the two-feature rule of Eq. trigger) ---------------------------------------- */

/* MLP 6 -> 32 -> 32 -> 4 (tanh hidden layers, softmax), FP32, on the device.
 * Parameters: one flat vector of 1412 floats, W1 (32x6, [out][in]), b1 (32),
 * W2 (32x32), b2, W3 (4x32), b3. Inputs are standardised with (mu, sd) first.
 * theta0: host, 1412 floats (the initial weights; the caller draws them). */
int gf_mlp_create(const float* theta0, void* stream, gf_mlp** out);
int gf_mlp_destroy(gf_mlp* M);
int gf_mlp_set_norm(gf_mlp* M, const float* mu, const float* sd);      /* host, 6 each, sd > 0 */
int gf_mlp_get_params(gf_mlp* M, float* theta);                        /* host, 1412 */
/* logits (device n x 4) for rows of X (device n x 6). */
int gf_mlp_forward(gf_mlp* M, const float* X, int n, float* logits);
/* Mean cross-entropy over the rows (labels y, device ints in [0,4)) and its gradient;
 * loss and grad (1412 floats) are HOST outputs. */
int gf_mlp_loss_grad(gf_mlp* M, const float* X, const int* y, int n, float* loss, float* grad);
/* Adam (beta 0.9/0.999, eps 1e-8) over `epochs` passes of full minibatches of size
 * `batch`; perm (host, epochs*n sample indices, or NULL for the stored order) gives
 * the minibatch order. *final_loss (host, optional) = loss of the last minibatch. */
int gf_mlp_train(gf_mlp* M, const float* X, const int* y, int n, const int* perm, int epochs, int batch,
                 float lr, float* final_loss);
/* Class (argmax logit) for host feature rows (n x 6 doubles), n <= 4096, into cls (host). */
int gf_mlp_predict(gf_mlp* M, const double* feat, int n, int* cls);
/* Softmax probabilities (host, n x 4) for host feature rows, n <= 4096. */
int gf_mlp_probs(gf_mlp* M, const double* feat, int n, double* probs);
/* The selector's 6 inputs for grid g: [log10 r50, log10 r100, r100/r50, fraction of
 * voxels with rho_hat == 0, mean rho_hat, std rho_hat] (x: host, 6 doubles). */
int gf_select_features(const gf_grid* g, double r50, double r100, double* x);

/* ---- the one entry point that allocates nothing -------------------------------- */

/* The paper has no counterpart to this call; it exists for callers that must not
 * allocate device memory: code recorded into a CUDA graph or running under stream
 * capture (cudaMalloc is illegal there), hosts that give the library a fixed,
 * pre-reserved memory budget, and latency-critical loops that must never reach
 * the allocator. It computes the same acceptance residual as gf_true_residual,
 * *eta = ||M(f - K u)||_2 / ||M f||_2 in FP64 with E_e = rho_min + (1 - rho_min)
 * rho_hat_e^p (scaled by E0), but needs no gf_grid: every input is a raw pointer.
 *  - rho_hat: n_elem doubles; f, u: n_dof doubles; eta: ONE double; all DEVICE
 *    pointers, allocated on the device that is current when the call is made: the
 *    call never switches devices, and it launches on, and uses the scratch array
 *    of, the current device. Pointers into another GPU's memory are not detected
 *    and make the kernels fault. *eta is written on `stream` (a cudaStream_t,
 *    NULL = legacy default stream); read it after the stream's work completes.
 *  - Bad values give a non-finite *eta, not an error code: *eta is NaN when
 *    ||M f|| = 0 (a load that is zero on every free DOF; gf_true_residual returns
 *    GF_ERR_ARG there), and NaN or Inf when an input holds NaN or Inf or the sums
 *    overflow (gf_true_residual returns GF_ERR_NONFINITE). A caller must treat a
 *    non-finite *eta as "not accepted"; the comparison *eta <= tau already does.
 *  - Scratch: a static device array inside the library (about 11.2 MB), reserved
 *    on every GPU that loads the library until the process exits. It holds grids
 *    of at most 1,048,576 DOFs; larger grids return GF_ERR_ARG with a message.
 *  - The first call on each device looks up the array's device address (with that
 *    device current); make that first call before any stream capture begins.
 *  - Every call reuses the same array. Calls whose GPU work overlaps (on different
 *    streams or threads) race on it and must be serialised by the caller; each call
 *    writes every scratch word it reads, so nothing has to be cleared between calls.
 *  - No cudaMalloc, cudaFree or other allocating routine is called. */
int gf_true_residual_noalloc(int nx, int ny, int nz, double h, double E0, double nu,
                             const double* rho_hat, double p, double rho_min, const double* f,
                             const double* u, double* eta, void* stream);

/* Node-stencil launch choice: threads per block of the FP64 kernel (64/128/256) and
 * of the FP32 kernel (64/128/256; 0 = the shared-memory-tiled FP32 kernel; -64/-128/
 * -256 = the 27-neighbour register-gather FP32 kernel with that block size).
 * FP64 results do not depend on the choice; FP32 results depend on it only through
 * the summation order of the kernel variant. gf_batch_autotune picks these by timing. */
int gf_set_stencil_blocks(gf_grid* g, int tpb64, int tpb32);

/* ---- diagnostics -------------------------------------------------------------- */
int gf_get_stats(const gf_grid* g, gf_stats* s);
int gf_reset_stats(gf_grid* g);
const char* gf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GF_H */
