/*
 * stmg.h -- C ABI of the GB300 space-time multigrid (STMG) library.
 *
 * The library solves the all-at-once backward-Euler / linear-finite-element system
 * J u = b of the 1D transient heat equation
 *     c dT/dt - d/dx (k dT/dx) = q  on [0, L] x [0, t_T],
 *     T = 0 at t = 0,  T = 0 at x = 0,  dT/dx = 0 at x = L            (Sec. 2, Eq. of the PDE)
 * with element-wise constant k, c, q (Sec. 2.2), and its adjoint J^T Lambda = rhs
 * (Sec. 7.2), by the space-time multigrid V-cycle of Alg. 1: damped pointwise Jacobi
 * (Sec. 3.1), x- or t-semi-coarsening chosen by the effective anisotropy parameter
 * lambda_eff = sqrt(min D_e max D_e) dt / dx^2 (Sec. 4, Alg. 3; Alg. 4 with min_nel),
 * rediscretised coarse operators with conductivity (K) or resistivity (R) averaging
 * (Sec. 3.1, 5.1), causal prolongation with R = s P^T (Sec. 3.1), an exact coarsest
 * solve, and the Dirichlet treatment J = B J_Neu B + W_Diri (I - B) (Appendix A).
 *
 * Grid and layout.  N = nel elements (dx = L/N), NT = nt time steps (dt = t_T/NT).
 * A space-time vector (u, b, Lambda, rhs) is a dense row-major FP64 array of
 * (NT+1) x (N+1) values: row n is time level t_n, column i is node x_i = i dx.
 * Element arrays (k, c, chi, gradient) have N values; element loads q have
 * (NT+1) x N values (row n = load at t_n; row 0 is ignored because b_0 = 0).
 *
 * Memory.  Unless stated otherwise every array argument may be device memory or host
 * memory (pageable or pinned); host arrays are copied through the library's device
 * buffers on the handle's stream.  The caller owns all argument arrays.  The handle
 * owns the level hierarchy and all scratch, allocated at stmg_create and freed by
 * stmg_destroy.
 *
 * Streams and synchronisation.  All device work of a handle is issued on the CUDA
 * stream given to stmg_create (NULL = legacy default stream).  Every call returns only
 * after its outputs are complete.  A handle must not be used by two host threads at
 * once; distinct handles are independent.
 *
 * Errors.  Every call returns a stmg_status; no call exits or traps.  On an error the
 * message is available from stmg_last_error(handle) (or stmg_last_error(NULL) when no
 * handle exists).  A solve that stops on the divergence or cycle limit still returns
 * its last iterate, cycle count and relative residual.
 */
#ifndef STMG_H
#define STMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stmg_handle* stmg_t;

typedef enum {
    STMG_OK = 0,
    STMG_EINVAL = 1,    /* invalid argument (sizes, non-positive k/c/L/t_T, NaN, bad options) */
    STMG_ENOMEM = 2,    /* device or host allocation failed; the handle is unchanged */
    STMG_ECUDA = 3,     /* a CUDA runtime call failed; see stmg_last_error */
    STMG_EDIVERGED = 4, /* relative residual exceeded div_tol (Sec. 3.1 termination rule) */
    STMG_EMAXITER = 5   /* max_cycles reached before tol (Sec. 3.1 termination rule) */
} stmg_status;

enum { STMG_INTERP_CAUSAL = 0, STMG_INTERP_BILINEAR = 1 };  /* Sec. 3.1 / 5.1 "C" and "B" */
enum { STMG_REASM_K = 0, STMG_REASM_R = 1, STMG_REASM_D = 2, /* Sec. 3.1 "K", Sec. 5.1 "R" and "D" */
       STMG_REASM_P = 3 };  /* Sec. 5.1 "P": Galerkin products J_{l+1} = R_l J_l P_l (FP64 only; the
                               coarse k, c that Alg. 3 reads are the K averages, as in Sec. 5.1) */
enum { STMG_FP64 = 0, STMG_MIXED = 1 };                     /* precision of the V-cycle */
enum { STMG_COARSEST = 0, STMG_XCOARSEN = 1, STMG_TCOARSEN = 2 };

/* Solver options; stmg_default_opts fills the defaults given in brackets. */
typedef struct {
    int nu;                    /* [5] pre- and post-smoothing steps of Alg. 1 (paper: 5, and 20 in Sec. 6-7) */
    double omega;              /* [0.5] Jacobi damping (Sec. 3.1) */
    double lambda_crit;        /* [0.25] t-coarsen iff lambda_eff < lambda_crit (Alg. 3; Sec. 5.2 value) */
    int interp;                /* [STMG_INTERP_CAUSAL] prolongation in time: causal (copies forward)
                                  or bilinear 1/2 [1 2 1] (Sec. 5.1); x always 1/2 [1 2 1] */
    int reassembly;            /* [STMG_REASM_R] coarse operators: material averaging K / R / D (D only
                                  through stmg_create_design) or Galerkin products P */
    int min_nel;               /* [0] M of Alg. 4 (t-coarsen when N/2 < M); 0 = Alg. 3 */
    int num_levels;            /* [0] > 0: exactly this many levels N_l */
    int max_levels;            /* [30] cap on N_l when num_levels == 0 */
    long long max_coarse_dofs; /* [512] num_levels == 0: stop at the first level with <= this many DOFs */
    double deff_fixed;         /* [0] > 0: design-independent D_eff on every level (Sec. 7.2) */
    int precision;             /* [STMG_FP64] STMG_FP64: FP64 V-cycles (Alg. 1 as written).
                                  STMG_MIXED: FP64 defect correction around FP32 V-cycles; the fine
                                  residual, the coarse material and the coarsest solve stay FP64.
                                  Both: the FP32 parts (the cycles, the termination norms) run on
                                  copies scaled by a power of two chosen from ||b||, so the solution
                                  of J u = 2^m b is exactly 2^m u for any b whose squares fit FP64. */
    double tol;                /* [1e-10] stop when ||J u - b|| / ||b|| < tol (Sec. 3.1) */
    double div_tol;            /* [1e9] stop (diverged) when the relative residual exceeds this */
    int max_cycles;            /* [100] cycle limit (Sec. 3.1) */
    int mixed_first_cycles;    /* [4] STMG_MIXED: FP32 V-cycles run on the first defect (an inner
                                  iteration) before the first FP64 correction; each counts as a cycle */
    int mixed_inner_cycles;    /* [4] STMG_MIXED: FP32 V-cycles run on every later defect (1..8), the
                                  first from zero and the others continuing the FP32 iterate; the
                                  termination test is then taken every mixed_inner_cycles cycles */
} stmg_opts;

void stmg_default_opts(stmg_opts* opts);

/* Build the level hierarchy for N = nel elements and NT = nt steps on [0, L] x [0, t_end]
 * with element conductivity k_el[nel] > 0 and heat capacity c_el[nel] > 0 (host or
 * device).  Runs the coarsening strategy (Alg. 3/4), averages the coarse materials
 * (Sec. 3.1/5.1), computes W_Diri per level (Appendix A) and allocates every level's
 * vectors.  opts NULL = defaults.  stream: a cudaStream_t or NULL. */
stmg_status stmg_create(stmg_t* handle, int nel, int nt, double L, double t_end, const double* k_el,
                        const double* c_el, const stmg_opts* opts, void* stream);

/* Device memory hooks: alloc(bytes, ctx) returns device memory of the current device,
 * aligned to 256 bytes, or NULL when it has none left (the call then fails with
 * STMG_ENOMEM); free(ptr, ctx) returns it.  Both are called only from the host thread
 * that is inside an stmg call on this handle.  stmg_create_with_allocator is stmg_create
 * with every device allocation of the handle (hierarchy, scratch, staging) taken from
 * the hooks; give both or neither. */
typedef void* (*stmg_alloc_fn)(size_t bytes, void* ctx);
typedef void (*stmg_free_fn)(void* ptr, void* ctx);
stmg_status stmg_create_with_allocator(stmg_t* handle, int nel, int nt, double L, double t_end,
                                       const double* k_el, const double* c_el, const stmg_opts* opts, void* stream,
                                       stmg_alloc_fn alloc, stmg_free_fn free_fn, void* ctx);

/* Issue the handle's future work on another CUDA stream (every call returns with its own
 * work complete, so nothing is pending on the old one). */
stmg_status stmg_set_stream(stmg_t handle, void* stream);

/* Bytes of device memory the handle holds now. */
long long stmg_device_bytes(stmg_t handle);

/* Device bytes that stmg_create would allocate for this problem and these options (the
 * planner runs on the host; nothing is allocated); k_el, c_el are host arrays.  Solves
 * with host element loads, checkpointed sensitivities or the per-level building blocks
 * may add staging buffers.  Returns -1 for invalid arguments. */
long long stmg_footprint(int nel, int nt, double L, double t_end, const double* k_el, const double* c_el,
                         const stmg_opts* opts);

/* Hierarchy for a design field chi[nel] (host or device) with the SIMP model simp6 =
 * {k_ins, k_con, c_ins, c_con, p_k, p_c} (host, Sec. 2.1) and D-reassembly (Sec. 5.1):
 * x-coarsening averages chi over element pairs and re-applies the SIMP model on the coarse
 * level; opts->reassembly is ignored (D is implied).  The only way to use D-reassembly. */
stmg_status stmg_create_design(stmg_t* handle, int nel, int nt, double L, double t_end, const double* chi,
                               const double* simp6, const stmg_opts* opts, void* stream);
/* Replace the design field of a stmg_create_design handle; re-runs the planner. */
stmg_status stmg_update_design(stmg_t handle, const double* chi);

/* Replace k and c (same nel); re-runs the planner.  With deff_fixed > 0 the coarsening
 * path, and so every level size, is unchanged (Sec. 7.2); otherwise levels may be
 * re-allocated. */
stmg_status stmg_update_material(stmg_t handle, const double* k_el, const double* c_el);

void stmg_destroy(stmg_t handle);
const char* stmg_last_error(stmg_t handle);

/* SIMP material model (Sec. 2.1): k = k_ins + (k_con - k_ins) chi^p_k and
 * c = c_ins + (c_con - c_ins) chi^p_c with simp6 = {k_ins, k_con, c_ins, c_con, p_k, p_c}
 * (host array).  chi, k_el, c_el: nel values, all device memory of the current device (or
 * managed memory; anything else gives STMG_EINVAL).  stream may be NULL. */
stmg_status stmg_simp(int nel, const double* chi, const double* simp6, double* k_el, double* c_el, void* stream);

/* Nodal load b = B b_Neu from element loads q_el[(nt+1) x nel] (Sec. 2.2, Appendix A):
 * b[n][i] = dx/2 (q[n][i-1] + q[n][i]) for n >= 1, i >= 1 (q[n][N] taken as 0); 0 on
 * the Dirichlet DOFs.  b: (nt+1) x (nel+1). */
stmg_status stmg_assemble_load(stmg_t handle, const double* q_el, double* b);

/* Solve J u = b (Sec. 2.2) by V-cycles (Alg. 1) until the Sec. 3.1 termination rule.
 * Exactly one of q_el (element loads, assembled as in stmg_assemble_load) and b_nodal
 * ((nt+1) x (nel+1)) is non-NULL.  u: (nt+1) x (nel+1) output; with warm != 0 its
 * content is the initial guess (warm restart, Sec. 7.2), else the guess is 0.
 * cycles / relres (may be NULL) receive the cycle count and ||J u - b|| / ||b||.
 * relres is the termination norm of the Sec. 3.1 rule as the solver evaluates it: ||b||^2
 * is summed in FP64, and the residual's squares are formed from its FP64 value rounded to
 * FP32 (after scaling by a power of two), summed in FP32 within each thread and in FP64
 * across threads, so it agrees with the exact FP64 norm to about 1e-6 relative.
 * Returns STMG_OK, STMG_EDIVERGED or STMG_EMAXITER (u filled in all three cases). */
stmg_status stmg_solve(stmg_t handle, const double* q_el, const double* b_nodal, double* u, int warm, int* cycles,
                       double* relres);

/* Solve the adjoint system J^T lam = rhs (Sec. 7.2) with the same hierarchy, the
 * transposed level operators and the unchanged causal prolongation.  For the
 * compliance objective rhs = b dt / Theta_ref.  Shapes and results as stmg_solve. */
stmg_status stmg_solve_adjoint(stmg_t handle, const double* rhs, double* lam, int warm, int* cycles,
                               double* relres);

/* Design sensitivity of Theta = b^T u dt / Theta_ref (Sec. 7.1) by the discrete adjoint
 * method (Sec. 7.2): dtheta_dchi[e] = -Lambda^T (dJ/dchi_e) u with
 * dJ/dchi_e = k'(chi_e) dJ/dk_e + c'(chi_e) dJ/dc_e from the SIMP model (Sec. 2.1).
 * u solves J u = b and lam solves J^T lam = b dt / Theta_ref.  chi: nel values;
 * simp6: host array as in stmg_simp; dtheta_dchi: nel outputs. */
stmg_status stmg_sensitivity(stmg_t handle, const double* chi, const double* simp6, const double* u,
                             const double* lam, double* dtheta_dchi);

/* ---- time-slab checkpointing of the forward state ------------------------------------ */
/* J is block lower-bidiagonal (Sec. 2.2): every time level of the forward solution follows
 * from the previous one by one implicit step.  A caller that keeps only every K-th time
 * level of a solution (the checkpoints: rows 0, K, 2K, ..., (S-1)K with S = ceil(nt/K),
 * stored as S dense rows of nel+1 values) can rebuild the rest exactly.
 * stmg_recompute_slabs fills u ((nt+1) x (nel+1)) with the checkpoint rows and, for each
 * slab j, rows jK+1 .. min((j+1)K, nt) stepped from row jK with right-hand side b_nodal;
 * all slabs run concurrently.  Requires nel <= 8192. */
stmg_status stmg_recompute_slabs(stmg_t handle, const double* b_nodal, const double* ckpt, int slab_rows,
                                 double* u);
/* The design sensitivity of stmg_sensitivity, with u recomputed slab by slab from the
 * checkpoints inside the same kernel instead of being read from a stored solution. */
stmg_status stmg_sensitivity_slabs(stmg_t handle, const double* chi, const double* simp6, const double* b_nodal,
                                   const double* ckpt, int slab_rows, const double* lam, double* dtheta_dchi);

/* Theta = b^T u dt / theta_ref (Sec. 7.1); theta: host output. */
stmg_status stmg_objective(stmg_t handle, const double* b, const double* u, double theta_ref, double* theta);
/* Gradient of the compliance of Sec. 7.1 with respect to the state, times a seed:
 * grad_u = seed * dTheta/du = seed * b dt / theta_ref (with seed = 1 the right-hand side of
 * the adjoint system of Sec. 7.2).  b, grad_u: (nt+1) x (nel+1) device arrays (grad_u may
 * equal b); host arrays give STMG_EINVAL. */
stmg_status stmg_objective_gradient(stmg_t handle, const double* b, double theta_ref, double seed, double* grad_u);
/* Design-independent effective diffusivity of Sec. 7.2 for the SIMP model simp6 (host
 * array as in stmg_simp): D_eff = sqrt(min D_SIMP * max D_SIMP), D_SIMP(chi) =
 * k(chi) / c(chi), with the extrema taken over chi = j / 10000, j = 0..10000 (they need
 * not lie at chi = 0 or 1).  Host-only arithmetic; deff: host output.  Use it as
 * stmg_opts.deff_fixed for a hierarchy that every design of an optimisation shares. */
stmg_status stmg_deff_simp(const double* simp6, double* deff);

/* ---- optimisation loop (Sec. 7) ------------------------------------------------------ */
/* One design update of the optimisation loop of Sec. 7.2.  The paper updates the design
 * with MMA, a third-party optimiser that is not part of the method; this call is the
 * projected-gradient step that stands in for it:
 *   y = chi - move * (g / max|g|),
 *   chi_new = clamp(y - mu, max(0, chi - move), min(1, chi + move)),
 * with mu >= 0 the smallest shift for which mean(chi_new) <= vol_frac (the volume
 * constraint of Sec. 7.1 for elements of equal size), found by 64 bisection steps on
 * [0, 2] in FP64 (mu = 2, every element on its lower bound, when the move limit keeps the
 * mean above vol_frac).  chi_new is then the Euclidean projection of y onto the box and
 * volume constraints.  g = dtheta (e.g. from stmg_sensitivity); g = 0 gives the projection
 * of chi.  chi, dtheta, chi_new: nel doubles of device memory (chi_new may equal chi);
 * 0 < vol_frac <= 1, 0 < move <= 1; stream may be NULL.  Returns after chi_new is complete;
 * messages go to stmg_last_error(NULL). */
stmg_status stmg_design_update(int nel, const double* chi, const double* dtheta, double vol_frac, double move,
                               double* chi_new, void* stream);

/* ---- hierarchy inspection ------------------------------------------------------------ */
int stmg_num_levels(stmg_t handle);
/* Level l (0 = finest): sizes, how level l+1 is built (STMG_XCOARSEN / STMG_TCOARSEN, or
 * STMG_COARSEST on the last level), mesh widths, W_Diri and lambda_eff.  Any output
 * pointer may be NULL. */
stmg_status stmg_level_info(stmg_t handle, int level, int* nel, int* nt, int* next, double* dx, double* dt,
                            double* w_diri, double* lambda_eff);
/* Coarse-level material of level l into host arrays k[nel_l], c[nel_l]. */
stmg_status stmg_level_material(stmg_t handle, int level, double* k, double* c);

/* ---- building blocks on one level (space-time vectors of level l's shape) ------------- */
/* y = J_l u (adjoint != 0: y = J_l^T u). */
stmg_status stmg_apply(stmg_t handle, int level, int adjoint, const double* u, double* y);
/* nsweeps damped-Jacobi steps u <- u + omega D^-1 (b - J_l u) in place (Sec. 3.1). */
stmg_status stmg_smooth(stmg_t handle, int level, int adjoint, int nsweeps, double* u, const double* b);
/* bc = R_l r = s P_l^T r (level l -> l+1, Sec. 3.1). */
stmg_status stmg_restrict(stmg_t handle, int level, const double* r, double* bc);
/* u += P_l z (level l+1 -> l, Sec. 3.1). */
stmg_status stmg_prolong_add(stmg_t handle, int level, const double* z, double* u);
/* Exact solve of J_l u = b (adjoint: J_l^T u = b) by implicit time stepping with one
 * tridiagonal solve per step; the coarsest-level solver of Alg. 1. */
stmg_status stmg_exact_solve(stmg_t handle, int level, int adjoint, const double* b, double* u);
/* One V-cycle of Alg. 1 on the finest level, u updated in place, in the precision of
 * the options (STMG_MIXED: one FP64 defect-correction step around one FP32 cycle). */
stmg_status stmg_vcycle(stmg_t handle, int adjoint, double* u, const double* b);
/* One step of the mixed scheme's V-cycle (Alg. 1 in FP32 inside FP64 defect correction) on
 * the handle's own level vectors, enqueued on its stream without synchronising, so that the
 * step can be timed on its own: kind 0 = level l's DOWN half (the nu pre-smoothing sweeps
 * from zero, the residual and the restriction into level l+1), kind 1 = level l's UP half
 * (prolongation of level l+1's correction and the nu post-smoothing sweeps; on level 0 added
 * into the FP64 iterate), kind 2 = the FP64 defect of level 0 (the result is then read
 * from the device's scalars, not returned), kind 3 = level l's UP half into the FP32
 * iterate, on level 0 too (the form of every inner FP32 cycle but the last before a
 * defect).  The vectors hold whatever the last solve or V-cycle left in them (zero before
 * the first), and the FP64 iterate is modified.
 * STMG_EINVAL unless the handle is STMG_MIXED with nu > 0, 0 <= level < levels - 1 and
 * kind in 0..3 (kind 2: level 0 only). */
stmg_status stmg_mixed_pass(stmg_t handle, int level, int adjoint, int kind);

/* ---- allocation-free sensitivity ------------------------------------------------------ */
/* The paper has no counterpart to this entry point; it is a deployment variant of
 * stmg_sensitivity for callers that cannot allocate device memory when they need a
 * gradient: cudaMalloc/cudaFree may synchronise the whole device, which a caller that
 * overlaps its own streams with ours cannot afford, and a caller whose device memory is
 * fixed at start-up (a framework-owned pool or a hard budget) may not request more.
 *
 * Same result as stmg_sensitivity, without a handle and without any allocation:
 * nel, nt, L, t_end describe the grid as in stmg_create; chi (nel), u and lam
 * ((nt+1) x (nel+1), dense rows) and dtheta_dchi (nel) must all be device memory of the
 * current device or managed memory (host arrays, and device arrays of another GPU, are
 * rejected with STMG_EINVAL: staging them would need an allocation); simp6 is a host
 * array as in stmg_simp; stream may be NULL.
 * The partial sums live in one fixed array of STMG_NOALLOC_MAX_SCRATCH doubles (8 MiB)
 * inside the library's device image, which every GPU that loads the library keeps until
 * the process exits.  The call needs 2 * (floor(nt/256) + 1) * nel of them and rejects
 * larger problems with STMG_EINVAL (for example nel = 4096 with nt up to 32767); it also
 * rejects nt >= 65535 * 256, whose time chunks exceed one launch's grid.
 * The first call on each device looks up that array's device address; make it before
 * any stream capture.  All calls share the array: calls whose work overlaps on the GPU
 * (different streams or host threads without ordering) race and give wrong results, so
 * serialise them.  Every scratch value read is written earlier in the same call, so a
 * previous call's contents never leak into a result.  The call synchronises its stream
 * (cudaStreamSynchronize) and returns after dtheta_dchi is complete; messages go to
 * stmg_last_error(NULL). */
#define STMG_NOALLOC_MAX_SCRATCH (1 << 20)
stmg_status stmg_sensitivity_noalloc(int nel, int nt, double L, double t_end, const double* chi, const double* simp6,
                                     const double* u, const double* lam, double* dtheta_dchi, void* stream);

/* ---- serving: continuous batching of forward and adjoint solves ----------------------- */
/* A server owns worker threads (one CUDA stream each) and one device memory arena of
 * budget_bytes.  Submitted requests wait in one FIFO queue and start when a worker is free
 * and their footprint (stmg_footprint, plus staging for an element-load array) fits in the
 * budget next to the running requests; several requests run at once and their kernels
 * overlap on the GPU.  A request that the arena cannot place next to the others (its free
 * bytes split into pieces) waits until the running requests finish and runs on the emptied
 * arena.  Finished hierarchies stay resident in the arena and are reused by
 * later requests with the same grid and options (cache != 0) until memory is needed.  A
 * request's result does not depend on what else runs: it is bit-identical alone and in any
 * mix.  Latencies are measured on the server's steady clock (stmg_server_now). */
typedef struct stmg_server_s* stmg_server_t;

typedef struct {
    int workers;            /* [4] concurrent solves */
    long long budget_bytes; /* [0 = half of the free device memory] arena size */
    int cache;              /* [1] keep finished hierarchies for reuse */
    int max_nu;             /* [0] > 0: a request that reaches max_cycles or diverges is solved
                               again with twice the smoothing sweeps, up to max_nu (the decision
                               depends only on the request, so results stay mix-independent) */
} stmg_server_opts;

typedef struct {
    int nel, nt;
    double L, t_end;
    const double* k_el;     /* host, nel values; copied by stmg_server_submit */
    const double* c_el;     /* host, nel values; copied by stmg_server_submit */
    const double* q_el;     /* host element loads (nt+1) x nel, kept alive by the caller until the
                               request completes; or NULL for the uniform load q_value */
    double q_value;
    int adjoint;            /* 0: solve J u = b; 1: solve J^T lam = b dt (the compliance adjoint,
                               Sec. 7.2, with Theta_ref = 1) */
    double* out;            /* (nt+1) x (nel+1) result (host or device), or NULL */
    stmg_opts opts;         /* solver options of this request */
} stmg_request;

typedef struct {
    int status;             /* stmg_status of the solve, or -1 while queued or running */
    int cycles;
    double relres;
    double theta;           /* b^T x dt of the result x: the compliance, for both directions */
    double t_submit, t_start, t_end;  /* seconds on the server clock */
    long long bytes;        /* device bytes the request's hierarchy held */
    int worker;
    int nu;                 /* smoothing sweeps of the solve that produced the result */
} stmg_result;

void stmg_server_default_opts(stmg_server_opts* opts);
stmg_status stmg_server_create(stmg_server_t* server, const stmg_server_opts* opts);
/* Queue one request; ticket receives its id.  Never blocks on the GPU. */
stmg_status stmg_server_submit(stmg_server_t server, const stmg_request* request, long long* ticket);
/* Result of a request; wait != 0 blocks until it is done. */
stmg_status stmg_server_result(stmg_server_t server, long long ticket, int wait, stmg_result* result);
/* Blocks until every submitted request is done. */
stmg_status stmg_server_drain(stmg_server_t server);
double stmg_server_now(stmg_server_t server);
/* Highest arena use so far, in bytes. */
long long stmg_server_peak_bytes(stmg_server_t server);
/* Finishes queued requests, then stops the workers and frees everything. */
void stmg_server_destroy(stmg_server_t server);

/* ---- statistics ------------------------------------------------------------------------ */
/* Number of CUDA kernels this library has launched in this process so far (all handles). */
unsigned long long stmg_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* STMG_H */
