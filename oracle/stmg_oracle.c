/*
 * stmg_oracle.c -- plain, slow, FP64 CPU oracle for the space-time multigrid (STMG)
 * method of Appel & Alexandersen, "Space-Time Multigrid Methods Suitable for Topology
 * Optimisation of Transient Heat Conduction" (arXiv 2505.10168).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that the CUDA
 * library is compared against.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header, table or
 * helper with the CUDA library, and it is deliberately written for readability,
 * not speed: every operator is applied element by element from its finite-element
 * definition, the prolongation is an explicit list of stencil columns, and the
 * restriction is that same list read backwards (R = s P^T).
 *
 * Grid convention (Sec. 2.2): N elements of width dx = L/N, nodes i = 0..N at
 * x_i = i dx; NT backward-Euler steps of dt = t_T/NT, time levels n = 0..NT.  A
 * space-time vector holds all (NT+1)(N+1) nodal values, row n (time level) by row,
 * node index fastest: v[n*(N+1) + i].  The Dirichlet DOFs are the initial row n = 0
 * and the node i = 0 of every row (Sec. 2, boundary conditions; Appendix A treats the
 * initial condition as a Dirichlet condition).
 *
 * Parity status: every exported function is pinned by tests/test_oracle_*.py against
 * the printed stencil, the W_Diri formula, dense direct solves, the separable modal
 * closed form, the printed lambda_eff examples, a dense-matrix brute-force V-cycle,
 * the adjoint identity and central finite differences.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no fused multiply-add contraction,
 * so every product is rounded on its own as written).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_LEVELS 64

enum { OR_COARSEST = 0, OR_XCOARSEN = 1, OR_TCOARSEN = 2 };
enum { OR_INTERP_C = 0, OR_INTERP_B = 1 };
enum { OR_REASM_K = 0, OR_REASM_R = 1, OR_REASM_D = 2 };
enum { OR_CONVERGED = 0, OR_DIVERGED = 1, OR_MAXCYCLES = 2, OR_EINVAL = 3 };

/* Solver settings.  Field meaning follows the paper's parameter names. */
typedef struct {
    int nu;                 /* smoothing steps before and after the coarse correction (Alg. 1) */
    double omega;           /* Jacobi damping, 1/2 in the paper (Sec. 3.1) */
    double lambda_crit;     /* coarsening threshold of Alg. 2-4 */
    int interp;             /* OR_INTERP_C (causal) or OR_INTERP_B (bilinear), Sec. 5.1 */
    int reassembly;         /* OR_REASM_K, _R or _D, Sec. 5.1 */
    int min_nel;            /* M of Alg. 4; 0 gives Alg. 3 */
    int num_levels;         /* > 0: exactly this many levels N_l (as in the paper's tests) */
    int max_levels;         /* cap on N_l when num_levels == 0 */
    long long max_coarse_dofs; /* num_levels == 0: stop once a level has at most this many DOFs */
    double deff_fixed;      /* > 0: design-independent D_eff on every level (Sec. 7.2) */
} or_opts;

typedef struct {
    int N, NT;              /* elements and time steps on this level */
    double dx, dt;
    double *k, *c, *chi;    /* per element; chi only with D-reassembly */
    double W;               /* W_Diri of this level (Appendix A) */
    double lambda_eff;      /* lambda_eff of this level (Alg. 3) */
    int next;               /* how level l+1 is built from this one; OR_COARSEST on the last */
} or_level;

typedef struct {
    int nlev;
    or_level lev[OR_MAX_LEVELS];
    or_opts o;
    double simp[6];         /* k_ins, k_con, c_ins, c_con, p_k, p_c (Sec. 2.1) */
    double *u[OR_MAX_LEVELS], *b[OR_MAX_LEVELS], *r[OR_MAX_LEVELS];
} or_hier;

static size_t nvec(const or_level* L) { return (size_t)(L->NT + 1) * (size_t)(L->N + 1); }
static size_t at(const or_level* L, int n, int i) { return (size_t)n * (size_t)(L->N + 1) + (size_t)i; }
static int is_dirichlet(int n, int i) { return n == 0 || i == 0; }

/* ------------------------------------------------------------------------------ */
/* Material model, Sec. 2.1: k = k_ins + (k_con - k_ins) chi^p_k, same form for c. */
/* ------------------------------------------------------------------------------ */
static double simp_k(const double* s, double chi) { return s[0] + (s[1] - s[0]) * pow(chi, s[4]); }
static double simp_c(const double* s, double chi) { return s[2] + (s[3] - s[2]) * pow(chi, s[5]); }
static double simp_dk(const double* s, double chi) { return s[4] * (s[1] - s[0]) * pow(chi, s[4] - 1.0); }
static double simp_dc(const double* s, double chi) { return s[5] * (s[3] - s[2]) * pow(chi, s[5] - 1.0); }

void or_simp(int N, const double* chi, const double* simp, double* k, double* c) {
    for (int e = 0; e < N; ++e) {
        k[e] = simp_k(simp, chi[e]);
        c[e] = simp_c(simp, chi[e]);
    }
}

/* ------------------------------------------------------------------------------ */
/* Element matrices of the linear Galerkin discretisation, Sec. 2.2:              */
/*   mass   M_e = c_e dx / 6 [[2,1],[1,2]],  stiffness K_e = k_e / dx [[1,-1],[-1,1]] */
/* ------------------------------------------------------------------------------ */
static double elem_M(const or_level* L, int e, int a, int b) { return L->c[e] * L->dx / 6.0 * (a == b ? 2.0 : 1.0); }
static double elem_K(const or_level* L, int e, int a, int b) { return L->k[e] / L->dx * (a == b ? 1.0 : -1.0); }

/* W_Diri = max_e c_e dx/dt + max_e k_e/dx (Appendix A, last equation). */
static double w_diri(const or_level* L) {
    double cmax = L->c[0], kmax = L->k[0];
    for (int e = 1; e < L->N; ++e) {
        if (L->c[e] > cmax) cmax = L->c[e];
        if (L->k[e] > kmax) kmax = L->k[e];
    }
    return cmax * L->dx / L->dt + kmax / L->dx;
}

/* Nodal load b = B b_Neu, with b_Neu,i = integral of q N_i over the two elements that
 * touch node i for an element-wise constant q (Sec. 2.2 and Appendix A).  q is given
 * per element and time level, q[n*N + e]; row 0 is unused because b_0 = 0. */
void or_assemble_load(int N, int NT, double dx, const double* q, double* b) {
    or_level L;
    memset(&L, 0, sizeof L);
    L.N = N; L.NT = NT;
    memset(b, 0, nvec(&L) * sizeof(double));
    for (int n = 1; n <= NT; ++n)
        for (int e = 0; e < N; ++e)
            for (int a = 0; a < 2; ++a) {
                int i = e + a;
                if (is_dirichlet(n, i)) continue;
                b[at(&L, n, i)] += q[(size_t)n * N + e] * dx / 2.0;
            }
}

/* ------------------------------------------------------------------------------ */
/* All-at-once operator J (Sec. 2.2) with the Dirichlet treatment of Appendix A:   */
/*   J = B J_Neu B + W_Diri (I - B).                                               */
/* Block row n >= 1 of J_Neu is  -M/dt T_{n-1} + (M/dt + K) T_n.  The product B..B */
/* drops every row and every column that belongs to a Dirichlet DOF; the identity   */
/* part puts W_Diri on their diagonal.  adj != 0 applies the transpose J^T (Sec. 7.2). */
/* ------------------------------------------------------------------------------ */
static void apply_op(const or_level* L, int adj, const double* u, double* y) {
    int N = L->N, NT = L->NT;
    memset(y, 0, nvec(L) * sizeof(double));
    for (int n = 1; n <= NT; ++n)
        for (int e = 0; e < N; ++e)
            for (int a = 0; a < 2; ++a)
                for (int bb = 0; bb < 2; ++bb) {
                    int row = e + a, col = e + bb;
                    if (row == 0 || col == 0) continue; /* node 0 is Dirichlet */
                    double m = elem_M(L, e, a, bb) / L->dt;
                    double kk = elem_K(L, e, a, bb);
                    /* entry J[(n,row),(n,col)] = m + kk; entry J[(n,row),(n-1,col)] = -m,
                     * present only if row n-1 is not the Dirichlet row 0. */
                    if (!adj) {
                        y[at(L, n, row)] += (m + kk) * u[at(L, n, col)];
                        if (n - 1 >= 1) y[at(L, n, row)] += -m * u[at(L, n - 1, col)];
                    } else {
                        y[at(L, n, col)] += (m + kk) * u[at(L, n, row)];
                        if (n - 1 >= 1) y[at(L, n - 1, col)] += -m * u[at(L, n, row)];
                    }
                }
    for (int n = 0; n <= NT; ++n)
        for (int i = 0; i <= N; ++i)
            if (is_dirichlet(n, i)) y[at(L, n, i)] = L->W * u[at(L, n, i)];
}

/* Main diagonal of J (the matrix D of the smoother, Sec. 3.1). */
static void diag_op(const or_level* L, double* d) {
    int N = L->N, NT = L->NT;
    memset(d, 0, nvec(L) * sizeof(double));
    for (int n = 1; n <= NT; ++n)
        for (int e = 0; e < N; ++e)
            for (int a = 0; a < 2; ++a) {
                int row = e + a;
                if (row == 0) continue;
                d[at(L, n, row)] += elem_M(L, e, a, a) / L->dt + elem_K(L, e, a, a);
            }
    for (int n = 0; n <= NT; ++n)
        for (int i = 0; i <= N; ++i)
            if (is_dirichlet(n, i)) d[at(L, n, i)] = L->W;
}

/* r = b - J u (or b - J^T u). */
static void residual(const or_level* L, int adj, const double* u, const double* b, double* r) {
    size_t nv = nvec(L);
    apply_op(L, adj, u, r);
    for (size_t p = 0; p < nv; ++p) r[p] = b[p] - r[p];
}

static double norm2(const double* v, size_t n) {
    double s = 0.0;
    for (size_t p = 0; p < n; ++p) s += v[p] * v[p];
    return sqrt(s);
}

/* Damped pointwise Jacobi, Sec. 3.1: u <- u + omega D^{-1} (b - J u), nsweeps times. */
static void jacobi(const or_level* L, int adj, double omega, int nsweeps, double* u, const double* b) {
    size_t nv = nvec(L);
    double* r = (double*)malloc(nv * sizeof(double));
    double* d = (double*)malloc(nv * sizeof(double));
    diag_op(L, d);
    for (int s = 0; s < nsweeps; ++s) {
        residual(L, adj, u, b, r);
        for (size_t p = 0; p < nv; ++p) u[p] += omega * r[p] / d[p];
    }
    free(r);
    free(d);
}

/* ------------------------------------------------------------------------------ */
/* Prolongation P (Sec. 3.1, stencils of the three coarsening types; Sec. 5.1 for   */
/* the bilinear variant).  p_column lists the fine points that the coarse point    */
/* (m, j) is sent to and the weight of each: this is column (m, j) of P.           */
/* ------------------------------------------------------------------------------ */
static int p_column(const or_level* F, int type, int interp, int m, int j, int* fn, int* fi, double* w) {
    int cnt = 0;
    if (type == OR_XCOARSEN) {
        /* x: 1/2 [1 2 1] within the time row; coarse node j sits on fine node 2j. */
        fn[cnt] = m; fi[cnt] = 2 * j; w[cnt] = 1.0; ++cnt;
        if (2 * j - 1 >= 0) { fn[cnt] = m; fi[cnt] = 2 * j - 1; w[cnt] = 0.5; ++cnt; }
        if (2 * j + 1 <= F->N) { fn[cnt] = m; fi[cnt] = 2 * j + 1; w[cnt] = 0.5; ++cnt; }
    } else if (interp == OR_INTERP_C) {
        /* t, causal: the coarse value at t_{2m} is copied to fine levels 2m and 2m+1
         * (the stencil's centre and the row above it, i.e. forward in time only). */
        fn[cnt] = 2 * m; fi[cnt] = j; w[cnt] = 1.0; ++cnt;
        if (2 * m + 1 <= F->NT) { fn[cnt] = 2 * m + 1; fi[cnt] = j; w[cnt] = 1.0; ++cnt; }
    } else {
        /* t, bilinear: 1/2 [1 2 1] along time. */
        fn[cnt] = 2 * m; fi[cnt] = j; w[cnt] = 1.0; ++cnt;
        if (2 * m - 1 >= 0) { fn[cnt] = 2 * m - 1; fi[cnt] = j; w[cnt] = 0.5; ++cnt; }
        if (2 * m + 1 <= F->NT) { fn[cnt] = 2 * m + 1; fi[cnt] = j; w[cnt] = 0.5; ++cnt; }
    }
    return cnt;
}

/* Restriction scale s of R = s P^T: 1 for x-coarsening, 1/2 for t-coarsening (Sec. 3.1). */
static double r_scale(int type) { return type == OR_XCOARSEN ? 1.0 : 0.5; }

/* u_fine += P z_coarse */
static void prolong_add(const or_level* F, const or_level* C, int type, int interp, const double* z, double* u) {
    int fn[3], fi[3];
    double w[3];
    for (int m = 0; m <= C->NT; ++m)
        for (int j = 0; j <= C->N; ++j) {
            int cnt = p_column(F, type, interp, m, j, fn, fi, w);
            for (int q = 0; q < cnt; ++q) u[at(F, fn[q], fi[q])] += w[q] * z[at(C, m, j)];
        }
}

/* b_coarse = s P^T r_fine */
static void restrict_to(const or_level* F, const or_level* C, int type, int interp, const double* r, double* bc) {
    int fn[3], fi[3];
    double w[3];
    double s = r_scale(type);
    for (int m = 0; m <= C->NT; ++m)
        for (int j = 0; j <= C->N; ++j) {
            int cnt = p_column(F, type, interp, m, j, fn, fi, w);
            double acc = 0.0;
            for (int q = 0; q < cnt; ++q) acc += w[q] * r[at(F, fn[q], fi[q])];
            bc[at(C, m, j)] = s * acc;
        }
}

/* ------------------------------------------------------------------------------ */
/* Exact solve of J u = b (or J^T u = b) by implicit time stepping (Sec. 2.2): the */
/* block bidiagonal structure gives (M/dt + K) T_n = q_n + M/dt T_{n-1} on the     */
/* non-Dirichlet nodes 1..N; the adjoint runs backwards with T_{n+1}.  Each step is */
/* a tridiagonal solve by the Thomas algorithm.  Dirichlet DOFs: u = b / W_Diri.   */
/* Used as the coarsest-level solver of Alg. 1 and as the exact discrete solution. */
/* ------------------------------------------------------------------------------ */
static void time_stepping(const or_level* L, int adj, const double* b, double* u) {
    int N = L->N, NT = L->NT;
    double *lo = calloc((size_t)N + 2, sizeof(double)), *di = calloc((size_t)N + 2, sizeof(double));
    double *up = calloc((size_t)N + 2, sizeof(double)), *f = calloc((size_t)N + 2, sizeof(double));
    double *cp = calloc((size_t)N + 2, sizeof(double)), *dp = calloc((size_t)N + 2, sizeof(double));
    for (int n = 0; n <= NT; ++n)
        for (int i = 0; i <= N; ++i)
            if (is_dirichlet(n, i)) u[at(L, n, i)] = b[at(L, n, i)] / L->W;
    /* tridiagonal A = (M/dt + K) on nodes 1..N, built element by element */
    for (int e = 0; e < N; ++e)
        for (int a = 0; a < 2; ++a)
            for (int bb = 0; bb < 2; ++bb) {
                int row = e + a, col = e + bb;
                if (row == 0 || col == 0) continue;
                double v = elem_M(L, e, a, bb) / L->dt + elem_K(L, e, a, bb);
                if (col == row) di[row] += v;
                else if (col == row - 1) lo[row] += v;
                else up[row] += v;
            }
    for (int step = 1; step <= NT; ++step) {
        int n = adj ? NT + 1 - step : step;
        int nprev = adj ? n + 1 : n - 1; /* the coupled time level */
        int has_prev = adj ? (nprev <= NT) : (nprev >= 1);
        for (int i = 1; i <= N; ++i) f[i] = b[at(L, n, i)];
        if (has_prev)
            for (int e = 0; e < N; ++e)
                for (int a = 0; a < 2; ++a)
                    for (int bb = 0; bb < 2; ++bb) {
                        int row = e + a, col = e + bb;
                        if (row == 0 || col == 0) continue;
                        f[row] += elem_M(L, e, a, bb) / L->dt * u[at(L, nprev, col)];
                    }
        /* Thomas: forward elimination then back substitution on unknowns 1..N */
        cp[1] = up[1] / di[1];
        dp[1] = f[1] / di[1];
        for (int i = 2; i <= N; ++i) {
            double den = di[i] - lo[i] * cp[i - 1];
            cp[i] = up[i] / den;
            dp[i] = (f[i] - lo[i] * dp[i - 1]) / den;
        }
        u[at(L, n, N)] = dp[N];
        for (int i = N - 1; i >= 1; --i) u[at(L, n, i)] = dp[i] - cp[i] * u[at(L, n, i + 1)];
    }
    free(lo); free(di); free(up); free(f); free(cp); free(dp);
}

/* ------------------------------------------------------------------------------ */
/* Coarse-level material (Sec. 3.1 for K; Sec. 5.1 for D and R).  t-coarsening     */
/* keeps k and c; x-coarsening merges elements 2e and 2e+1 into coarse element e.   */
/* ------------------------------------------------------------------------------ */
static void coarse_material(const or_hier* H, const or_level* F, or_level* C, int type) {
    if (type == OR_TCOARSEN) {
        for (int e = 0; e < C->N; ++e) {
            C->k[e] = F->k[e];
            C->c[e] = F->c[e];
            if (F->chi) C->chi[e] = F->chi[e];
        }
        return;
    }
    for (int e = 0; e < C->N; ++e) {
        double k0 = F->k[2 * e], k1 = F->k[2 * e + 1];
        double c0 = F->c[2 * e], c1 = F->c[2 * e + 1];
        if (H->o.reassembly == OR_REASM_D) {
            double chi = (F->chi[2 * e] + F->chi[2 * e + 1]) / 2.0;
            C->chi[e] = chi;
            C->k[e] = simp_k(H->simp, chi);
            C->c[e] = simp_c(H->simp, chi);
        } else if (H->o.reassembly == OR_REASM_R) {
            double rho0 = 1.0 / k0, rho1 = 1.0 / k1; /* thermal resistivity */
            double rho = (rho0 + rho1) / 2.0;
            C->k[e] = 1.0 / rho;
            C->c[e] = (c0 + c1) / 2.0;
        } else {
            C->k[e] = (k0 + k1) / 2.0;
            C->c[e] = (c0 + c1) / 2.0;
        }
    }
}

/* lambda_eff = D_eff dt / dx^2 with D_eff = sqrt(min_e D_e max_e D_e), D_e = k_e / c_e
 * (Sec. 4, Alg. 3), or with the fixed design-independent D_eff of Sec. 7.2. */
static double lambda_eff(const or_hier* H, const or_level* L) {
    double deff;
    if (H->o.deff_fixed > 0.0) {
        deff = H->o.deff_fixed;
    } else {
        double dmin = L->k[0] / L->c[0], dmax = dmin;
        for (int e = 1; e < L->N; ++e) {
            double d = L->k[e] / L->c[e];
            if (d < dmin) dmin = d;
            if (d > dmax) dmax = d;
        }
        deff = sqrt(dmin * dmax);
    }
    return deff * L->dt / (L->dx * L->dx);
}

static void alloc_level(or_level* L, int with_chi) {
    L->k = (double*)calloc((size_t)L->N, sizeof(double));
    L->c = (double*)calloc((size_t)L->N, sizeof(double));
    L->chi = with_chi ? (double*)calloc((size_t)L->N, sizeof(double)) : NULL;
}

/* ------------------------------------------------------------------------------ */
/* Hierarchy construction: Alg. 3 (Alg. 4 when min_nel > 0).                        */
/* Per level: t-coarsen iff lambda_eff < lambda_crit (or N/2 < M), else x-coarsen. */
/* Where the paper leaves the depth open it is set by num_levels, else coarsening  */
/* stops once a level holds at most max_coarse_dofs DOFs.  A direction that cannot */
/* halve its size (odd count or a single interval) is replaced by the other one.   */
/* ------------------------------------------------------------------------------ */
or_hier* or_create(int N, int NT, double Ldom, double tT, const double* k, const double* c, const double* chi,
                   const double* simp, const or_opts* o) {
    if (N < 1 || NT < 1 || !(Ldom > 0) || !(tT > 0) || !o || o->nu < 0) return NULL;
    for (int e = 0; e < N; ++e)
        if (!(k[e] > 0) || !(c[e] > 0)) return NULL;
    if (o->reassembly == OR_REASM_D && (!chi || !simp)) return NULL;
    or_hier* H = (or_hier*)calloc(1, sizeof(or_hier));
    H->o = *o;
    if (simp) memcpy(H->simp, simp, sizeof H->simp);
    int with_chi = (o->reassembly == OR_REASM_D);
    or_level* L0 = &H->lev[0];
    L0->N = N; L0->NT = NT; L0->dx = Ldom / N; L0->dt = tT / NT;
    alloc_level(L0, with_chi);
    for (int e = 0; e < N; ++e) {
        L0->k[e] = k[e];
        L0->c[e] = c[e];
        if (with_chi) L0->chi[e] = chi[e];
    }
    int cap = o->num_levels > 0 ? o->num_levels : (o->max_levels > 0 ? o->max_levels : OR_MAX_LEVELS);
    if (cap > OR_MAX_LEVELS) cap = OR_MAX_LEVELS;
    int l = 0;
    for (;;) {
        or_level* L = &H->lev[l];
        L->W = w_diri(L);
        L->lambda_eff = lambda_eff(H, L);
        L->next = OR_COARSEST;
        if (l + 1 >= cap) break;
        if (o->num_levels <= 0 && (long long)nvec(L) <= o->max_coarse_dofs) break;
        int can_x = (L->N % 2 == 0) && L->N >= 2;
        int can_t = (L->NT % 2 == 0) && L->NT >= 2;
        int want_t = (L->lambda_eff < o->lambda_crit) || (o->min_nel > 0 && L->N / 2 < o->min_nel);
        int type;
        if (want_t) type = can_t ? OR_TCOARSEN : (can_x ? OR_XCOARSEN : OR_COARSEST);
        else type = can_x ? OR_XCOARSEN : (can_t ? OR_TCOARSEN : OR_COARSEST);
        if (type == OR_COARSEST) break;
        L->next = type;
        or_level* C = &H->lev[l + 1];
        C->N = type == OR_XCOARSEN ? L->N / 2 : L->N;
        C->NT = type == OR_TCOARSEN ? L->NT / 2 : L->NT;
        C->dx = type == OR_XCOARSEN ? 2.0 * L->dx : L->dx;
        C->dt = type == OR_TCOARSEN ? 2.0 * L->dt : L->dt;
        alloc_level(C, with_chi);
        coarse_material(H, L, C, type);
        ++l;
    }
    H->nlev = l + 1;
    for (int q = 0; q < H->nlev; ++q) {
        size_t nv = nvec(&H->lev[q]);
        H->u[q] = (double*)calloc(nv, sizeof(double));
        H->b[q] = (double*)calloc(nv, sizeof(double));
        H->r[q] = (double*)calloc(nv, sizeof(double));
    }
    return H;
}

void or_destroy(or_hier* H) {
    if (!H) return;
    for (int q = 0; q < H->nlev; ++q) {
        free(H->lev[q].k); free(H->lev[q].c); free(H->lev[q].chi);
        free(H->u[q]); free(H->b[q]); free(H->r[q]);
    }
    free(H);
}

/* ------------------------------------------------------------------------------ */
/* Alg. 1, VCycle(l, u, b), followed literally.                                     */
/* ------------------------------------------------------------------------------ */
static void vcycle(or_hier* H, int l, int adj, double* u, const double* b) {
    or_level* L = &H->lev[l];
    if (l == H->nlev - 1) {
        time_stepping(L, adj, b, u);
        return;
    }
    or_level* C = &H->lev[l + 1];
    jacobi(L, adj, H->o.omega, H->o.nu, u, b);
    residual(L, adj, u, b, H->r[l]);
    restrict_to(L, C, L->next, H->o.interp, H->r[l], H->b[l + 1]);
    memset(H->u[l + 1], 0, nvec(C) * sizeof(double));
    vcycle(H, l + 1, adj, H->u[l + 1], H->b[l + 1]);
    prolong_add(L, C, L->next, H->o.interp, H->u[l + 1], u);
    jacobi(L, adj, H->o.omega, H->o.nu, u, b);
}

/* ------------------------------------------------------------------------------ */
/* Exported entry points (ctypes).                                                  */
/* ------------------------------------------------------------------------------ */
int or_nlevels(const or_hier* H) { return H->nlev; }

/* info[6*l ..]: N, NT, next, dx, dt, W   lam[l]: lambda_eff */
void or_level_info(const or_hier* H, int l, int* ints, double* dbl) {
    const or_level* L = &H->lev[l];
    ints[0] = L->N; ints[1] = L->NT; ints[2] = L->next;
    dbl[0] = L->dx; dbl[1] = L->dt; dbl[2] = L->W; dbl[3] = L->lambda_eff;
}

void or_level_material(const or_hier* H, int l, double* k, double* c) {
    const or_level* L = &H->lev[l];
    memcpy(k, L->k, (size_t)L->N * sizeof(double));
    memcpy(c, L->c, (size_t)L->N * sizeof(double));
}

void or_apply(const or_hier* H, int l, int adj, const double* u, double* y) { apply_op(&H->lev[l], adj, u, y); }
void or_diag(const or_hier* H, int l, double* d) { diag_op(&H->lev[l], d); }
void or_residual(const or_hier* H, int l, int adj, const double* u, const double* b, double* r) {
    residual(&H->lev[l], adj, u, b, r);
}
void or_smooth(const or_hier* H, int l, int adj, int nsweeps, double* u, const double* b) {
    jacobi(&H->lev[l], adj, H->o.omega, nsweeps, u, b);
}
void or_restrict(const or_hier* H, int l, const double* r, double* bc) {
    restrict_to(&H->lev[l], &H->lev[l + 1], H->lev[l].next, H->o.interp, r, bc);
}
void or_prolong_add(const or_hier* H, int l, const double* z, double* u) {
    prolong_add(&H->lev[l], &H->lev[l + 1], H->lev[l].next, H->o.interp, z, u);
}
void or_exact_level(const or_hier* H, int l, int adj, const double* b, double* u) {
    time_stepping(&H->lev[l], adj, b, u);
}
void or_vcycle(or_hier* H, int adj, double* u, const double* b) { vcycle(H, 0, adj, u, b); }

/* Solver loop, Sec. 3.1: start from u (zero unless warm), run V-cycles and stop after
 * cycle n when r_n < tol, r_n > div_tol or n = max_cycles, where
 * r_n = ||J u_n - b|| / ||b|| (Euclidean norm over all DOFs).  hist[0..cycles] gets r_n.
 * Returns OR_CONVERGED, OR_DIVERGED or OR_MAXCYCLES. */
int or_solve(or_hier* H, int adj, const double* b, double* u, int warm, double tol, double div_tol, int max_cycles,
             int* cycles, double* hist) {
    const or_level* L = &H->lev[0];
    size_t nv = nvec(L);
    if (!warm) memset(u, 0, nv * sizeof(double));
    double nb = norm2(b, nv);
    *cycles = 0;
    if (nb == 0.0) {
        memset(u, 0, nv * sizeof(double));
        if (hist) hist[0] = 0.0;
        return OR_CONVERGED;
    }
    double* r = (double*)malloc(nv * sizeof(double));
    residual(L, adj, u, b, r);
    double rn = norm2(r, nv) / nb;
    if (hist) hist[0] = rn;
    int status = OR_MAXCYCLES;
    for (int n = 1; n <= max_cycles; ++n) {
        vcycle(H, 0, adj, u, b);
        residual(L, adj, u, b, r);
        rn = norm2(r, nv) / nb;
        if (hist) hist[n] = rn;
        *cycles = n;
        if (rn < tol) { status = OR_CONVERGED; break; }
        if (rn > div_tol) { status = OR_DIVERGED; break; }
    }
    free(r);
    return status;
}

/* Exact discrete solution on an arbitrary fine grid without building a hierarchy. */
int or_exact(int N, int NT, double Ldom, double tT, const double* k, const double* c, int adj, const double* b,
             double* u) {
    if (N < 1 || NT < 1) return OR_EINVAL;
    or_level L;
    memset(&L, 0, sizeof L);
    L.N = N; L.NT = NT; L.dx = Ldom / N; L.dt = tT / NT;
    L.k = (double*)k; L.c = (double*)c;
    L.W = w_diri(&L);
    time_stepping(&L, adj, b, u);
    return OR_CONVERGED;
}

/* Objective of Sec. 7.1: Theta = b^T u dt / Theta_ref. */
double or_objective(int N, int NT, double dt, double theta_ref, const double* b, const double* u) {
    size_t nv = (size_t)(NT + 1) * (size_t)(N + 1);
    double s = 0.0;
    for (size_t p = 0; p < nv; ++p) s += b[p] * u[p];
    return s * dt / theta_ref;
}

/* Sensitivity of Theta with respect to the design field (Sec. 7.2, discrete adjoint
 * method): with J u = b, J^T Lambda = b dt / Theta_ref and b independent of chi,
 *   dTheta/dchi_e = -Lambda^T (dJ/dchi_e) u,
 *   dJ/dchi_e = k'(chi_e) dJ/dk_e + c'(chi_e) dJ/dc_e,
 * where dJ/dk_e and dJ/dc_e are read off the element loop of apply_op: element e adds
 * (M_e/dt + K_e) to block (n, n) and -M_e/dt to block (n, n-1) for n-1 >= 1, with the
 * Dirichlet rows and columns removed.  W_Diri only touches Dirichlet DOFs, where the
 * exact u and Lambda vanish, so its (non-smooth) dependence on chi is left out. */
void or_sensitivity(int N, int NT, double Ldom, double tT, const double* chi, const double* simp, const double* u,
                    const double* lam, double* g) {
    or_level L;
    memset(&L, 0, sizeof L);
    L.N = N; L.NT = NT; L.dx = Ldom / N; L.dt = tT / NT;
    for (int e = 0; e < N; ++e) {
        double sk = 0.0, sc = 0.0;
        for (int n = 1; n <= NT; ++n)
            for (int a = 0; a < 2; ++a)
                for (int bb = 0; bb < 2; ++bb) {
                    int row = e + a, col = e + bb;
                    if (row == 0 || col == 0) continue;
                    double dK = (a == bb ? 1.0 : -1.0) / L.dx;          /* dK_e/dk_e */
                    double dM = L.dx / 6.0 * (a == bb ? 2.0 : 1.0);     /* dM_e/dc_e */
                    double lr = lam[at(&L, n, row)];
                    sk += lr * dK * u[at(&L, n, col)];
                    sc += lr * dM / L.dt * u[at(&L, n, col)];
                    if (n - 1 >= 1) sc += lr * (-dM / L.dt) * u[at(&L, n - 1, col)];
                }
        g[e] = -(simp_dk(simp, chi[e]) * sk + simp_dc(simp, chi[e]) * sc);
    }
}
