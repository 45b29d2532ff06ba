/*
 * Plain FP64 CPU oracle for the parallel-in-time sparse-grid combination
 * method (Griebel, Schweitzer, Troska, arXiv 2509.22156).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header or constant table with the CUDA library under
 * paper_2509_22156_gb300/csrc; the two are compared on the same seeded inputs.
 *
 * Everything here is written for clarity, not speed: one grid point at a time,
 * textbook Krylov methods, all time points stored, no blocking or fusion.
 * The only concession to speed is an OpenMP loop over the independent
 * component grids (Sec. 2.1: "all subproblems are independent"), which does
 * not change any arithmetic.
 *
 * Citations name the paper's sections, equations and algorithms.
 *
 * Parity status of each function (which test pins it):
 *   or_enumerate / grid sizes      Table 1 process counts (exact integers)
 *   or_coefficient                 sum of coefficients = 1; d-linear exactness
 *   or_apply (heat)                discrete eigenfunction closed form
 *   or_apply (OU)                  consistency order 1 vs analytic operator,
 *                                  discrete mass balance, M-matrix sign pattern
 *   or_apply (var. coeff. heat)    consistency order 2 vs analytic operator,
 *                                  symmetry, reduction to heat at amplitude 0
 *   or_apply (CME, toggle switch)  order 2 (central) / 1 (donor cell) vs the
 *                                  analytic Fokker-Planck operator (sympy);
 *                                  mass balance; the immigration-death special
 *                                  case follows its closed-form mean
 *   or_apply (linear SDE)          reduction to OU for diagonal drift; order 1
 *                                  (donor cell) and order 2 (central) vs the
 *                                  analytic operator on a full-covariance
 *                                  normal density; mass balance; central
 *                                  drift: symmetric part diagonal (trace A);
 *                                  closed-form normal law approached
 *   or_cg / or_bicgstab            dense direct solve (numpy) on tiny grids
 *   or_phi / or_sequential         heat closed form per mode; OU Gaussian trend
 *   or_mgrit                       converged = sequential; FCF exactness after
 *                                  ceil(Nc/2) cycles, F exactness after Nc
 *                                  cycles; one cycle with Phi^m
 *   or_combine                     interpolation property at sparse-grid nodes
 *   or_hierarchize                 inverse pair; a hierarchical hat function
 *                                  sampled on a grid has one unit surplus
 *   or_recombine                   equals the combined solution (or_combine)
 *                                  at every node of every grid; a projection
 *                                  (Q Q = Q); fixes sparse-grid functions
 *   or_initial                     direct evaluation at node coordinates
 *   or_net_forward / backward      finite-difference gradient check; linear
 *                                  special cases; single-tap, s-channel,
 *                                  coefficient-channel and hidden-channel
 *                                  closed forms; an array restatement
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXD 6

enum { OR_HEAT = 0, OR_VARHEAT = 1, OR_OU = 2, OR_LSDE = 3, OR_CME = 4 };
enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOCONV = 4, OR_EBREAK = 5 };

typedef struct {
    int d, n, L0, op;
    double lo[OR_MAXD], hi[OR_MAXD];
    double theta, sigma, vamp;       /* OU drift/diffusion; var-coef amplitude */
    double sde_A[OR_MAXD * OR_MAXD]; /* linear SDE dX = A X dt + sigma dW: drift matrix */
    double sde_H[OR_MAXD * OR_MAXD]; /* H = 2 sigma D sigma^T (row major)              */
    int sde_central;                 /* drift flux: 0 donor cell, 1 central average   */
    /* chemical master equation, toggle-switch network (Sec. 4.3): species i
     * is produced at rate cme_p[i] / (cme_s[i] + (sum_{k != i} x_k)^cme_b[i])
     * and degraded at rate cme_g[i] x_i                                     */
    double cme_p[OR_MAXD], cme_s[OR_MAXD], cme_b[OR_MAXD], cme_g[OR_MAXD];
    int G;
    int *lev;                        /* G*d level multi-indices               */
    long long *off;                  /* G+1 packed offsets                    */
    double *coef;                    /* G combination coefficients            */
} or_problem;

/* ------------------------------------------------------------------------ */
/* Grid set of the combination formula (Eq. "combination_technique_solution",
 * Sec. 2.1.1): all l >= L0 componentwise with |l|_1 = n + (d-1) - w,
 * w = 0..d-1.  Order: w ascending, then l lexicographically ascending.     */

static long long binom(int a, int b)
{
    long long r = 1;
    if (b < 0 || b > a) return 0;
    for (int k = 1; k <= b; ++k) r = r * (a - b + k) / k;
    return r;
}

double or_coefficient(int d, int w)
{
    double s = (w % 2 == 0) ? 1.0 : -1.0;
    return s * (double)binom(d - 1, w);
}

/* Recursive lexicographic enumeration of l in [L0, inf)^d with sum = target. */
static int enum_rec(int d, int L0, int target, int pos, int *cur, int *out, int count, int cap)
{
    if (pos == d - 1) {
        if (target >= L0) {
            cur[pos] = target;
            if (out && count < cap) memcpy(out + (size_t)count * d, cur, sizeof(int) * d);
            return count + 1;
        }
        return count;
    }
    int remaining = d - 1 - pos;
    for (int v = L0; target - v >= remaining * L0; ++v) {
        cur[pos] = v;
        count = enum_rec(d, L0, target - v, pos + 1, cur, out, count, cap);
    }
    return count;
}

/* Returns the number of grids; writes levels (G*d) and layers (G) when the
 * buffers are non-NULL and large enough (cap grids). */
int or_enumerate(int d, int n, int L0, int *lev_out, int *layer_out, int cap)
{
    if (d < 1 || d > OR_MAXD || L0 < 1 || n < L0) return -1;
    int cur[OR_MAXD];
    int count = 0;
    for (int w = 0; w <= d - 1; ++w) {
        int target = n + (d - 1) - w;
        int before = count;
        count = enum_rec(d, L0, target, 0, cur, lev_out, count, cap);
        if (layer_out)
            for (int k = before; k < count && k < cap; ++k) layer_out[k] = w;
    }
    return count;
}

/* Interior nodes of Omega_l: prod_i (2^{l_i} - 1)  (Eq. "spatial_speedup_factor_new"). */
long long or_grid_points(int d, const int *l)
{
    long long n = 1;
    for (int i = 0; i < d; ++i) n *= ((1LL << l[i]) - 1);
    return n;
}

/* ------------------------------------------------------------------------ */
/* Problem object                                                           */

void *or_create(int d, int n, int L0, int op, const double *lo, const double *hi,
                double theta, double sigma, double vamp)
{
    if (d < 1 || d > OR_MAXD || L0 < 1 || n < L0 || op < 0 || op > 4) return NULL;
    or_problem *P = (or_problem *)calloc(1, sizeof(or_problem));
    P->d = d; P->n = n; P->L0 = L0; P->op = op;
    for (int i = 0; i < d; ++i) { P->lo[i] = lo[i]; P->hi[i] = hi[i]; }
    P->theta = theta; P->sigma = sigma; P->vamp = vamp;
    P->G = or_enumerate(d, n, L0, NULL, NULL, 0);
    P->lev = (int *)malloc(sizeof(int) * (size_t)P->G * d);
    int *layer = (int *)malloc(sizeof(int) * (size_t)P->G);
    or_enumerate(d, n, L0, P->lev, layer, P->G);
    P->off = (long long *)malloc(sizeof(long long) * (size_t)(P->G + 1));
    P->coef = (double *)malloc(sizeof(double) * (size_t)P->G);
    P->off[0] = 0;
    for (int g = 0; g < P->G; ++g) {
        P->off[g + 1] = P->off[g] + or_grid_points(d, P->lev + (size_t)g * d);
        P->coef[g] = or_coefficient(d, layer[g]);
    }
    free(layer);
    return P;
}

/* Drift matrix A and diffusion matrix H (row major, d x d) of the linear SDE
 * operator (op 3), and its drift flux: central = 0 donor cell (first order),
 * 1 the central average of the two neighbours (second order). */
int or_set_sde(void *vp, const double *A, const double *H, int central)
{
    or_problem *P = (or_problem *)vp;
    if (central != 0 && central != 1) return OR_EINVAL;
    memcpy(P->sde_A, A, sizeof(double) * P->d * P->d);
    memcpy(P->sde_H, H, sizeof(double) * P->d * P->d);
    P->sde_central = central;
    return OR_OK;
}

/* Reaction rates of the toggle-switch chemical master equation operator
 * (op 4, Sec. 4.3) per species: production p[i] / (s[i] + y^b[i]) with y
 * the sum of the other species' counts, degradation g[i] x_i; drift flux as
 * for the linear SDE (central = 1: central average). */
int or_set_cme(void *vp, const double *p, const double *s, const double *b, const double *g, int central)
{
    or_problem *P = (or_problem *)vp;
    if (central != 0 && central != 1) return OR_EINVAL;
    for (int i = 0; i < P->d; ++i) {
        P->cme_p[i] = p[i]; P->cme_s[i] = s[i]; P->cme_b[i] = b[i]; P->cme_g[i] = g[i];
    }
    P->sde_central = central;
    return OR_OK;
}

void or_destroy(void *vp)
{
    or_problem *P = (or_problem *)vp;
    if (!P) return;
    free(P->lev); free(P->off); free(P->coef); free(P);
}

int or_info(void *vp, int *G, long long *ntot, int *lev, double *coef, long long *off)
{
    or_problem *P = (or_problem *)vp;
    if (G) *G = P->G;
    if (ntot) *ntot = P->off[P->G];
    if (lev) memcpy(lev, P->lev, sizeof(int) * (size_t)P->G * P->d);
    if (coef) memcpy(coef, P->coef, sizeof(double) * (size_t)P->G);
    if (off) memcpy(off, P->off, sizeof(long long) * (size_t)(P->G + 1));
    return OR_OK;
}

void or_set_threads(int nt)
{
#ifdef _OPENMP
    if (nt > 0) omp_set_num_threads(nt);
#else
    (void)nt;
#endif
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Geometry of one grid: N_i interior nodes per axis, C-order strides with the
 * last axis fastest, mesh widths h_i = (b_i - a_i) / 2^{l_i}, interior node
 * coordinate x_{i,c} = a_i + (c+1) h_i for c = 0..N_i-1.                   */
typedef struct {
    int d;
    long long n, N[OR_MAXD], S[OR_MAXD];
    double h[OR_MAXD], lo[OR_MAXD];
} geom;

static geom grid_geom(const or_problem *P, int g)
{
    geom G;
    G.d = P->d;
    const int *l = P->lev + (size_t)g * P->d;
    for (int i = 0; i < P->d; ++i) {
        G.N[i] = (1LL << l[i]) - 1;
        G.h[i] = (P->hi[i] - P->lo[i]) / (double)(1LL << l[i]);
        G.lo[i] = P->lo[i];
    }
    long long s = 1;
    for (int i = P->d - 1; i >= 0; --i) { G.S[i] = s; s *= G.N[i]; }
    G.n = s;
    return G;
}

static void coords(const geom *G, long long j, long long *c)
{
    for (int i = 0; i < G->d; ++i) { c[i] = (j / G->S[i]) % G->N[i]; }
}

/* Variable diffusion coefficient a(x) = 1 + A * f_1(x_1) f_2(x_2) ... with
 * f alternating sin(2 pi x), cos(2 pi x), sin(2 pi x), ...; for d = 3 this is
 * 1 + A sin(2 pi x1) cos(2 pi x2) sin(2 pi x3). */
static double varcoef(const or_problem *P, const double *x)
{
    double prod = 1.0;
    for (int i = 0; i < P->d; ++i)
        prod *= (i % 2 == 0) ? sin(2.0 * M_PI * x[i]) : cos(2.0 * M_PI * x[i]);
    return 1.0 + P->vamp * prod;
}

/* ------------------------------------------------------------------------ */
/* Operator: q = (I + dt L_l) p on grid g, zero Dirichlet values outside
 * (Eq. "parabolic_problem_time_propagation_LES" multiplied by dt).
 *   heat:       (L p)_j = sum_i (2 p_j - p_{j-e_i} - p_{j+e_i}) / h_i^2
 *   var. coef.: (L p)_j = sum_i [a_{j+1/2}(p_j - p_{j+e_i})
 *                               + a_{j-1/2}(p_j - p_{j-e_i})] / h_i^2,
 *               a evaluated at the face midpoints
 *   OU (Fokker-Planck of dX = -theta X dt + sigma dW, Eq. "sde_fokker_planck"
 *   with diagonal drift): (L p)_j = sum_i (F_{j+1/2} - F_{j-1/2}) / h_i
 *               + (sigma^2/2)(2 p_j - p_{j-e_i} - p_{j+e_i}) / h_i^2,
 *               donor-cell flux F_{j+1/2} = v+ p_j + v- p_{j+e_i},
 *               face velocity v = -theta x_{j+1/2}.
 *   linear SDE (Eq. "sde_fokker_planck", dX = A X dt + sigma dW, H = 2 sigma
 *   D sigma^T): L p = sum_i d_i((A x)_i p) - (1/2) sum_ij H_ij d_i d_j p:
 *               drift as the donor-cell flux above with face velocity
 *               v = (A x)_i at the face x_{j+1/2 e_i}, or (central) the
 *               flux F_{j+1/2} = v (p_j + p_{j+e_i}) / 2; diagonal diffusion
 *               (H_ii / 2)(2 p_j - p_{j-e_i} - p_{j+e_i}) / h_i^2; for i < k
 *               the mixed term -((H_ik + H_ki) / 2) (p_{++} - p_{+-} - p_{-+}
 *               + p_{--}) / (4 h_i h_k) over the four diagonal neighbours
 *               j +- e_i +- e_k (zero outside the grid).
 *   chemical master equation, Fokker-Planck form (Sec. 4.3, Eq. "cme_fp"),
 *   toggle-switch network: species i has a production reaction (nu = +e_i,
 *   propensity a_i(x)) and a degradation reaction (nu = -e_i, b_i(x) =
 *   g_i x_i), so u_t = sum_i [-d_i((a_i - b_i) u) + (1/2) d_i^2((a_i + b_i) u)]
 *   and L u = sum_i d_i(v_i u) - (1/2) d_i^2(D_i u), v_i = a_i - b_i,
 *   D_i = a_i + b_i: drift as the linear SDE's flux with the face velocity
 *   v_i(x_{j+1/2 e_i}), diffusion the second difference of D_i u,
 *   -(D_i(x_{j+e_i}) p_{j+e_i} - 2 D_i(x_j) p_j + D_i(x_{j-e_i}) p_{j-e_i})
 *   / (2 h_i^2).                                                            */
static double cme_production(const or_problem *P, int i, const double *x)
{
    double y = 0.0;
    for (int k = 0; k < P->d; ++k)
        if (k != i) y += x[k];
    return P->cme_p[i] / (P->cme_s[i] + pow(y, P->cme_b[i]));
}

static void apply_grid(const or_problem *P, int g, double dt, const double *p, double *q)
{
    geom G = grid_geom(P, g);
    long long c[OR_MAXD];
    double x[OR_MAXD];
    for (long long j = 0; j < G.n; ++j) {
        coords(&G, j, c);
        for (int i = 0; i < G.d; ++i) x[i] = G.lo[i] + (double)(c[i] + 1) * G.h[i];
        double Lp = 0.0;
        for (int i = 0; i < G.d; ++i) {
            double pm = (c[i] > 0) ? p[j - G.S[i]] : 0.0;
            double pp = (c[i] < G.N[i] - 1) ? p[j + G.S[i]] : 0.0;
            double h = G.h[i];
            if (P->op == OR_HEAT) {
                Lp += (2.0 * p[j] - pm - pp) / (h * h);
            } else if (P->op == OR_VARHEAT) {
                double xf[OR_MAXD];
                memcpy(xf, x, sizeof(double) * G.d);
                xf[i] = x[i] + 0.5 * h;
                double ap = varcoef(P, xf);
                xf[i] = x[i] - 0.5 * h;
                double am = varcoef(P, xf);
                Lp += (ap * (p[j] - pp) + am * (p[j] - pm)) / (h * h);
            } else if (P->op == OR_OU) {
                double vp = -P->theta * (x[i] + 0.5 * h);
                double vm = -P->theta * (x[i] - 0.5 * h);
                double Fp = fmax(vp, 0.0) * p[j] + fmin(vp, 0.0) * pp;
                double Fm = fmax(vm, 0.0) * pm + fmin(vm, 0.0) * p[j];
                Lp += (Fp - Fm) / h + 0.5 * P->sigma * P->sigma * (2.0 * p[j] - pm - pp) / (h * h);
            } else if (P->op == OR_CME) {
                /* a_i does not depend on x_i; b_i = g_i x_i does */
                double a = cme_production(P, i, x), gi = P->cme_g[i];
                double vp = a - gi * (x[i] + 0.5 * h), vm = a - gi * (x[i] - 0.5 * h);
                double Fp, Fm;
                if (P->sde_central) {
                    Fp = vp * 0.5 * (p[j] + pp);
                    Fm = vm * 0.5 * (pm + p[j]);
                } else {
                    Fp = fmax(vp, 0.0) * p[j] + fmin(vp, 0.0) * pp;
                    Fm = fmax(vm, 0.0) * pm + fmin(vm, 0.0) * p[j];
                }
                double Dm = a + gi * (x[i] - h), D0 = a + gi * x[i], Dp = a + gi * (x[i] + h);
                Lp += (Fp - Fm) / h - 0.5 * (Dp * pp - 2.0 * D0 * p[j] + Dm * pm) / (h * h);
            } else {
                /* face velocities (A x)_i at x -+ h/2 e_i */
                double ax = 0.0;
                for (int k = 0; k < G.d; ++k) ax += P->sde_A[i * G.d + k] * x[k];
                double vp = ax + 0.5 * h * P->sde_A[i * G.d + i];
                double vm = ax - 0.5 * h * P->sde_A[i * G.d + i];
                double Fp, Fm;
                if (P->sde_central) {
                    Fp = vp * 0.5 * (p[j] + pp);
                    Fm = vm * 0.5 * (pm + p[j]);
                } else {
                    Fp = fmax(vp, 0.0) * p[j] + fmin(vp, 0.0) * pp;
                    Fm = fmax(vm, 0.0) * pm + fmin(vm, 0.0) * p[j];
                }
                Lp += (Fp - Fm) / h + 0.5 * P->sde_H[i * G.d + i] * (2.0 * p[j] - pm - pp) / (h * h);
                for (int k = i + 1; k < G.d; ++k) {
                    double hik = 0.5 * (P->sde_H[i * G.d + k] + P->sde_H[k * G.d + i]);
                    if (hik == 0.0) continue;
                    double corner[4];  /* (+,+) (+,-) (-,+) (-,-) in (i, k) */
                    for (int q2 = 0; q2 < 4; ++q2) {
                        int si = (q2 < 2) ? 1 : -1, sk = (q2 % 2 == 0) ? 1 : -1;
                        long long ci = c[i] + si, ck = c[k] + sk;
                        corner[q2] = (ci >= 0 && ci < G.N[i] && ck >= 0 && ck < G.N[k])
                                         ? p[j + si * G.S[i] + sk * G.S[k]] : 0.0;
                    }
                    Lp -= hik * (corner[0] - corner[1] - corner[2] + corner[3]) / (4.0 * h * G.h[k]);
                }
            }
        }
        q[j] = p[j] + dt * Lp;
    }
}

int or_apply(void *vp, double dt, int n_batch, const double *p, double *q)
{
    or_problem *P = (or_problem *)vp;
    long long nt = P->off[P->G];
    for (int b = 0; b < n_batch; ++b)
        for (int g = 0; g < P->G; ++g)
            apply_grid(P, g, dt, p + b * nt + P->off[g], q + b * nt + P->off[g]);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Krylov solvers (textbook forms).                                         */

static double dot(long long n, const double *a, const double *b)
{
    double s = 0.0;
    for (long long j = 0; j < n; ++j) s += a[j] * b[j];
    return s;
}

/* Conjugate gradients (Hestenes-Stiefel) for the symmetric operators
 * (Sec. 4.1 solver parameters).  x holds the initial guess on entry.
 * Stops when ||b - A x||_2 <= rtol ||b||_2. */
static int cg_grid(const or_problem *P, int g, double dt, const double *b, double *x,
                   double rtol, int maxit, int *iters)
{
    long long n = P->off[g + 1] - P->off[g];
    double *r = malloc(sizeof(double) * n), *p = malloc(sizeof(double) * n),
           *q = malloc(sizeof(double) * n);
    apply_grid(P, g, dt, x, q);
    for (long long j = 0; j < n; ++j) { r[j] = b[j] - q[j]; p[j] = r[j]; }
    double bb = dot(n, b, b), rr = dot(n, r, r);
    double stop = rtol * rtol * bb;
    int k = 0, st = OR_OK;
    while (rr > stop) {
        if (k >= maxit) { st = OR_ENOCONV; break; }
        apply_grid(P, g, dt, p, q);
        double pq = dot(n, p, q);
        if (!(pq > 0.0)) { st = OR_EBREAK; break; }
        double alpha = rr / pq;
        for (long long j = 0; j < n; ++j) { x[j] += alpha * p[j]; r[j] -= alpha * q[j]; }
        double rr_new = dot(n, r, r);
        double beta = rr_new / rr;
        for (long long j = 0; j < n; ++j) p[j] = r[j] + beta * p[j];
        rr = rr_new;
        ++k;
    }
    if (iters) *iters = k;
    free(r); free(p); free(q);
    return st;
}

/* BiCGStab (van der Vorst, 1992) for the non-symmetric drift operator
 * (Sec. 4.1 solver parameters), shadow residual r^ = r_0. */
static int bicgstab_grid(const or_problem *P, int g, double dt, const double *b, double *x,
                         double rtol, int maxit, int *iters)
{
    long long n = P->off[g + 1] - P->off[g];
    double *r = malloc(sizeof(double) * n), *rh = malloc(sizeof(double) * n),
           *p = malloc(sizeof(double) * n), *v = malloc(sizeof(double) * n),
           *s = malloc(sizeof(double) * n), *t = malloc(sizeof(double) * n);
    apply_grid(P, g, dt, x, v);
    for (long long j = 0; j < n; ++j) { r[j] = b[j] - v[j]; rh[j] = r[j]; p[j] = 0.0; v[j] = 0.0; }
    double bb = dot(n, b, b), rr = dot(n, r, r);
    double stop = rtol * rtol * bb;
    double rho = 1.0, alpha = 1.0, omega = 1.0;
    int k = 0, st = OR_OK;
    while (rr > stop) {
        if (k >= maxit) { st = OR_ENOCONV; break; }
        double rho_new = dot(n, rh, r);
        if (rho_new == 0.0 || omega == 0.0) { st = OR_EBREAK; break; }
        double beta = (rho_new / rho) * (alpha / omega);
        for (long long j = 0; j < n; ++j) p[j] = r[j] + beta * (p[j] - omega * v[j]);
        apply_grid(P, g, dt, p, v);
        double rhv = dot(n, rh, v);
        if (rhv == 0.0) { st = OR_EBREAK; break; }
        alpha = rho_new / rhv;
        for (long long j = 0; j < n; ++j) s[j] = r[j] - alpha * v[j];
        apply_grid(P, g, dt, s, t);
        double tt = dot(n, t, t);
        double ts = dot(n, t, s);
        omega = (tt > 0.0) ? ts / tt : 0.0;
        for (long long j = 0; j < n; ++j) { x[j] += alpha * p[j] + omega * s[j]; r[j] = s[j] - omega * t[j]; }
        rr = dot(n, r, r);
        rho = rho_new;
        ++k;
        if (omega == 0.0 && rr > stop) { st = OR_EBREAK; break; }
    }
    if (iters) *iters = k;
    free(r); free(rh); free(p); free(v); free(s); free(t);
    return st;
}

/* One backward-Euler step on grid g (Eq. "parabolic_problem_time_propagation"
 * and its linear system): solve (I + dt L) u_next = u_prev + dt f,
 * initial guess u_prev.  CG for heat operators, BiCGStab for OU. */
static int phi_grid(const or_problem *P, int g, double dt, const double *u_prev, const double *f,
                    double *u_next, double rtol, int maxit, int *iters)
{
    long long n = P->off[g + 1] - P->off[g];
    double *b = malloc(sizeof(double) * n);
    for (long long j = 0; j < n; ++j) b[j] = u_prev[j] + (f ? dt * f[j] : 0.0);
    if (u_next != u_prev) memcpy(u_next, u_prev, sizeof(double) * n);
    int st = (P->op == OR_OU || P->op == OR_LSDE || P->op == OR_CME) ? bicgstab_grid(P, g, dt, b, u_next, rtol, maxit, iters)
                                                   : cg_grid(P, g, dt, b, u_next, rtol, maxit, iters);
    free(b);
    return st;
}

int or_phi(void *vp, double dt, int n_batch, const double *u_prev, const double *f,
           double *u_next, double rtol, int maxit, int *iters /* n_batch*G or NULL */)
{
    or_problem *P = (or_problem *)vp;
    long long nt = P->off[P->G];
    int worst = OR_OK;
    int items = n_batch * P->G;
#pragma omp parallel for schedule(dynamic)
    for (int it = 0; it < items; ++it) {
        int b = it / P->G, g = it % P->G;
        int k = 0;
        int st = phi_grid(P, g, dt, u_prev + b * nt + P->off[g], f ? f + b * nt + P->off[g] : NULL,
                          u_next + b * nt + P->off[g], rtol, maxit, &k);
        if (iters) iters[it] = k;
        if (st != OR_OK) {
#pragma omp critical
            worst = st;
        }
    }
    return worst;
}

/* Dense direct solve of (I + dt L) x = b on a tiny grid: the matrix is built
 * column by column from the operator and factored by Gaussian elimination
 * with partial pivoting.  Used only to pin the Krylov solvers. */
int or_dense_solve(void *vp, int g, double dt, const double *b, double *x)
{
    or_problem *P = (or_problem *)vp;
    long long n = P->off[g + 1] - P->off[g];
    if (n > 4096) return OR_EINVAL;
    double *A = malloc(sizeof(double) * n * n), *e = calloc(n, sizeof(double)),
           *col = malloc(sizeof(double) * n), *rhs = malloc(sizeof(double) * n);
    for (long long k = 0; k < n; ++k) {
        e[k] = 1.0;
        apply_grid(P, g, dt, e, col);
        e[k] = 0.0;
        for (long long i = 0; i < n; ++i) A[i * n + k] = col[i];
    }
    memcpy(rhs, b, sizeof(double) * n);
    for (long long k = 0; k < n; ++k) {
        long long piv = k;
        for (long long i = k + 1; i < n; ++i)
            if (fabs(A[i * n + k]) > fabs(A[piv * n + k])) piv = i;
        if (piv != k) {
            for (long long c = 0; c < n; ++c) { double t = A[k * n + c]; A[k * n + c] = A[piv * n + c]; A[piv * n + c] = t; }
            double t = rhs[k]; rhs[k] = rhs[piv]; rhs[piv] = t;
        }
        for (long long i = k + 1; i < n; ++i) {
            double m = A[i * n + k] / A[k * n + k];
            for (long long c = k; c < n; ++c) A[i * n + c] -= m * A[k * n + c];
            rhs[i] -= m * rhs[k];
        }
    }
    for (long long k = n - 1; k >= 0; --k) {
        double s = rhs[k];
        for (long long c = k + 1; c < n; ++c) s -= A[k * n + c] * x[c];
        x[k] = s / A[k * n + k];
    }
    free(A); free(e); free(col); free(rhs);
    return OR_OK;
}

/* Time-sequential solution (Alg. 1 with s = 1): nsteps backward-Euler steps
 * on every grid.  F (or NULL: f = 0) holds the forcing f_n of step n =
 * 1..nsteps, packed like nsteps states (Eq. "parabolic_problem_time_
 * propagation_LES": (I + dt L) u_n = u_{n-1} + dt f_n).  tmul (or NULL: all
 * 1) gives every grid its own time partition (Sec. 2.2.1): grid g takes
 * tmul[g] steps of dt / tmul[g] inside each step n, all with f_n. */
int or_sequential(void *vp, const double *u0, double dt, int nsteps, double rtol, int maxit,
                  double *uT, const unsigned char *gmask /* G or NULL: grids to compute */,
                  const double *F, const int *tmul)
{
    or_problem *P = (or_problem *)vp;
    long long nt = P->off[P->G];
    int worst = OR_OK;
#pragma omp parallel for schedule(dynamic)
    for (int g = 0; g < P->G; ++g) {
        if (gmask && !gmask[g]) continue;
        long long n = P->off[g + 1] - P->off[g];
        int tm = tmul ? tmul[g] : 1;
        double *u = uT + P->off[g];
        memcpy(u, u0 + P->off[g], sizeof(double) * n);
        for (int s = 0; s < nsteps; ++s) {
            const double *f = F ? F + (long long)s * nt + P->off[g] : NULL;
            for (int q = 0; q < tm; ++q) {
                int st = phi_grid(P, g, dt / tm, u, f, u, rtol, maxit, NULL);
                if (st != OR_OK) {
#pragma omp critical
                    worst = st;
                }
            }
        }
    }
    return worst;
}

/* ------------------------------------------------------------------------ */
/* Learned coarse propagator: axis-separable 1-D convolutional network.
 * Not part of the paper; it replaces the coarse propagator Phi_coarse of
 * Sec. 3.3.1 inside MGRIT.  Layout of the weights (all FP64 here; callers
 * pass BF16-rounded values):
 *   layer k (k = 0..3) maps Cin_k -> Cout_k channels with Cin = {3,16,16,16}
 *   (input channels u, a(x), and the per-axis constant s_i = 1/(1 + 4 dT/h_i^2)
 *   for layer 0; hidden channels plus s_i for layers 1..3 -> Cin =
 *   {3,17,17,17}); s_i is the backward-Euler damping factor of the highest
 *   grid mode along axis i, a bounded stand-in for dT/h_i^2,
 *   Cout = {16,16,16,1}; W_k[o][c][t] with t = 0..4 the tap for offset t-2;
 *   bias_k[o].  h^{k+1}_o(j) = act(b_o + sum_i sum_c sum_t W[o][c][t] *
 *   in_c(j + (t-2) e_i)), zero padding outside the grid (Dirichlet zero),
 *   with in_c = (h^k channels, s_i) along axis i.  act = ReLU on layers 0..2,
 *   identity on layer 3.  The state enters normalised, u / sigma with
 *   sigma = sqrt(mean_j u_j^2) over the grid's nodes, and the output is
 *   u + sigma * h^4 (u itself when sigma = 0), so that the map is scale-
 *   equivariant like the linear propagator it replaces.                    */
#define NET_W 5
static const int NET_CIN[4] = {3, 17, 17, 17};
static const int NET_COUT[4] = {16, 16, 16, 1};

long long or_net_param_count(void)
{
    long long s = 0;
    for (int k = 0; k < 4; ++k) s += (long long)NET_COUT[k] * NET_CIN[k] * NET_W + NET_COUT[k];
    return s;
}

/* Parameter block layout: for k = 0..3: W_k (Cout*Cin*5) then b_k (Cout). */
static void net_offsets(long long *wo, long long *bo)
{
    long long s = 0;
    for (int k = 0; k < 4; ++k) {
        wo[k] = s; s += (long long)NET_COUT[k] * NET_CIN[k] * NET_W;
        bo[k] = s; s += NET_COUT[k];
    }
}

/* Feature input of a grid: channel 0 = u, channel 1 = a(x) (ones for the
 * constant-coefficient operators), and per axis the constant mu_i. */
static void net_layer_forward(const geom *G, int k, const double *theta, long long wo, long long bo,
                              const double *in /* Cin_k-1 channels (mu excluded) x n */,
                              const double *mu, double *pre /* Cout x n */)
{
    int cin = NET_CIN[k], cout = NET_COUT[k];
    long long n = G->n;
    long long c[OR_MAXD];
    for (long long j = 0; j < n; ++j) {
        coords(G, j, c);
        for (int o = 0; o < cout; ++o) {
            double acc = theta[bo + o];
            for (int i = 0; i < G->d; ++i) {
                for (int t = 0; t < NET_W; ++t) {
                    long long cc = c[i] + (t - 2);
                    if (cc < 0 || cc >= G->N[i]) continue;
                    long long jj = j + (t - 2) * G->S[i];
                    for (int ch = 0; ch < cin - 1; ++ch)
                        acc += theta[wo + ((long long)o * cin + ch) * NET_W + t] * in[ch * n + jj];
                    acc += theta[wo + ((long long)o * cin + (cin - 1)) * NET_W + t] * mu[i];
                }
            }
            pre[o * n + j] = acc;
        }
    }
}

/* Forward pass on one grid: out = u + h^4.  acts (optional) receives the
 * post-activation hidden states of layers 0..2 (3 x 16 x n) and pre the
 * pre-activations of layers 0..3 (16+16+16+1 channels x n). */
/* RMS of a grid vector (the network's input scale). */
static double rms(long long n, const double *u)
{
    double s = 0.0;
    for (long long j = 0; j < n; ++j) s += u[j] * u[j];
    return sqrt(s / (double)n);
}

static void net_forward_grid(const or_problem *P, int g, double dT, const double *theta,
                             const double *u, double *out, double *acts, double *pres)
{
    geom G = grid_geom(P, g);
    long long n = G.n;
    long long wo[4], bo[4];
    net_offsets(wo, bo);
    double mu[OR_MAXD];
    for (int i = 0; i < G.d; ++i) mu[i] = 1.0 / (1.0 + 4.0 * dT / (G.h[i] * G.h[i]));
    const double sigma = rms(n, u);
    if (!(sigma > 0.0)) {
        memcpy(out, u, sizeof(double) * n);
        if (acts) memset(acts, 0, sizeof(double) * 3 * 16 * n);
        if (pres) memset(pres, 0, sizeof(double) * 49 * n);
        return;
    }
    double *in0 = malloc(sizeof(double) * 2 * n);
    long long c[OR_MAXD];
    double x[OR_MAXD];
    for (long long j = 0; j < n; ++j) {
        in0[j] = u[j] / sigma;
        coords(&G, j, c);
        for (int i = 0; i < G.d; ++i) x[i] = G.lo[i] + (double)(c[i] + 1) * G.h[i];
        in0[n + j] = (P->op == OR_VARHEAT) ? varcoef(P, x) : 1.0;
    }
    double *pre = malloc(sizeof(double) * 16 * n);
    double *h = malloc(sizeof(double) * 16 * n);
    const double *in = in0;
    long long pre_off = 0;
    for (int k = 0; k < 4; ++k) {
        net_layer_forward(&G, k, theta, wo[k], bo[k], in, mu, pre);
        int cout = NET_COUT[k];
        if (pres) memcpy(pres + pre_off, pre, sizeof(double) * cout * n);
        pre_off += (long long)cout * n;
        if (k < 3) {
            for (long long t = 0; t < (long long)cout * n; ++t) h[t] = pre[t] > 0.0 ? pre[t] : 0.0;
            if (acts) memcpy(acts + (long long)k * 16 * n, h, sizeof(double) * 16 * n);
            in = h;
            /* next layer reads h while writing pre: distinct buffers */
        } else {
            for (long long j = 0; j < n; ++j) out[j] = u[j] + sigma * pre[j];
        }
    }
    free(in0); free(pre); free(h);
}

int or_net_forward(void *vp, double dT, const double *theta, int n_batch, const double *u, double *out)
{
    or_problem *P = (or_problem *)vp;
    long long nt = P->off[P->G];
    int items = n_batch * P->G;
#pragma omp parallel for schedule(dynamic)
    for (int it = 0; it < items; ++it) {
        int b = it / P->G, g = it % P->G;
        net_forward_grid(P, g, dT, theta, u + b * nt + P->off[g], out + b * nt + P->off[g], NULL, NULL);
    }
    return OR_OK;
}

/* Loss of one pair set: sum over items of ||out - y||^2 / ||y||^2, and its
 * gradient with respect to all parameters (reverse mode written out layer by
 * layer).  Returns the loss; grad (param_count) is overwritten. */
double or_net_loss_grad(void *vp, double dT, const double *theta, int n_batch, const double *u,
                        const double *y, double *grad)
{
    or_problem *P = (or_problem *)vp;
    long long nt = P->off[P->G];
    long long np = or_net_param_count();
    long long wo[4], bo[4];
    net_offsets(wo, bo);
    memset(grad, 0, sizeof(double) * np);
    double loss = 0.0;
    for (int b = 0; b < n_batch; ++b) {
        for (int g = 0; g < P->G; ++g) {
            geom G = grid_geom(P, g);
            long long n = G.n;
            const double *ub = u + b * nt + P->off[g];
            const double *yb = y + b * nt + P->off[g];
            double *out = malloc(sizeof(double) * n);
            double *acts = malloc(sizeof(double) * 3 * 16 * n);
            double *pres = malloc(sizeof(double) * 49 * n);
            net_forward_grid(P, g, dT, theta, ub, out, acts, pres);
            double yy = dot(n, yb, yb);
            if (yy <= 0.0) yy = 1.0;
            const double sigma = rms(n, ub);
            double *dpre = malloc(sizeof(double) * 16 * n); /* grad wrt pre-activation of layer k */
            double *dh = malloc(sizeof(double) * 16 * n);   /* grad wrt input hidden of layer k */
            for (long long j = 0; j < n; ++j) {
                double e = out[j] - yb[j];
                loss += e * e / yy;
                dpre[j] = 2.0 * e / yy * sigma;
            }
            if (!(sigma > 0.0)) {
                free(out); free(acts); free(pres); free(dpre); free(dh);
                continue;
            }
            double mu[OR_MAXD];
            for (int i = 0; i < G.d; ++i) mu[i] = 1.0 / (1.0 + 4.0 * dT / (G.h[i] * G.h[i]));
            /* layer inputs: layer 0 reads (u, a), layer k>0 reads acts[k-1] */
            double *in0 = malloc(sizeof(double) * 2 * n);
            long long c[OR_MAXD];
            double x[OR_MAXD];
            for (long long j = 0; j < n; ++j) {
                in0[j] = ub[j] / sigma;
                coords(&G, j, c);
                for (int i = 0; i < G.d; ++i) x[i] = G.lo[i] + (double)(c[i] + 1) * G.h[i];
                in0[n + j] = (P->op == OR_VARHEAT) ? varcoef(P, x) : 1.0;
            }
            long long pre_off[4] = {0, 16 * n, 32 * n, 48 * n};
            for (int k = 3; k >= 0; --k) {
                int cin = NET_CIN[k], cout = NET_COUT[k];
                const double *in = (k == 0) ? in0 : acts + (long long)(k - 1) * 16 * n;
                /* dpre holds dL/dpre_k (cout x n) */
                for (long long t = 0; t < (long long)(cin - 1) * n; ++t) dh[t] = 0.0;
                for (long long j = 0; j < n; ++j) {
                    coords(&G, j, c);
                    for (int o = 0; o < cout; ++o) {
                        double go = dpre[o * n + j];
                        if (go == 0.0) continue;
                        grad[bo[k] + o] += go;
                        for (int i = 0; i < G.d; ++i) {
                            for (int t = 0; t < NET_W; ++t) {
                                long long cc = c[i] + (t - 2);
                                if (cc < 0 || cc >= G.N[i]) continue;
                                long long jj = j + (t - 2) * G.S[i];
                                for (int ch = 0; ch < cin - 1; ++ch) {
                                    long long wi = wo[k] + ((long long)o * cin + ch) * NET_W + t;
                                    grad[wi] += go * in[ch * n + jj];
                                    dh[ch * n + jj] += go * theta[wi];
                                }
                                grad[wo[k] + ((long long)o * cin + (cin - 1)) * NET_W + t] += go * mu[i];
                            }
                        }
                    }
                }
                if (k > 0) {
                    /* through the ReLU of layer k-1 */
                    const double *pk = pres + pre_off[k - 1];
                    for (long long t = 0; t < 16 * n; ++t) dpre[t] = pk[t] > 0.0 ? dh[t] : 0.0;
                }
            }
            free(out); free(acts); free(pres); free(dpre); free(dh); free(in0);
        }
    }
    return loss;
}

/* ------------------------------------------------------------------------ */
/* Multigrid reduction in time (Sec. 3.3, Alg. 2), per grid, all time points
 * stored.  A level problem reads v_0 given, v_k = Phi_level(v_{k-1}) + g_k
 * for k = 1..N (Eq. "iterative_temporal_solution"); g == NULL means g = 0.
 * Phi_level is backward Euler with step dt_level (level 0: the fine step;
 * level q: dt * m^q), or on the level below the finest, optionally, the
 * learned network or m exact fine steps (used to pin the algorithm).       */

typedef struct {
    const or_problem *P;
    int g;
    double dt;          /* fine step */
    int m;              /* coarsening factor */
    int nlev;           /* number of levels (>= 2) */
    double rtol;        /* Krylov tolerance */
    int maxit;
    int coarse_kind;    /* 0 implicit BE, 1 m exact fine steps, 2 learned net,
                           3 two-stage SDIRK, 4 extrapolated BE (3 and 4 on
                           every coarse level) */
    const double *theta;/* net parameters (coarse_kind 2) */
    int relax_f;        /* 1: F-relaxation on the finest level, 2: on every level, 0: FCF */
    int status;
    const double *F;    /* forcing of the common steps 1..N (grid's part), stride nt, or NULL */
    long long nt;
    int tm;             /* the grid's steps per common step (its own time partition) */
} mg_ctx;

/* Coarsening factor between `level` and level + 1: the finest level of a
 * grid with its own time partition (tm steps per common step) has tm m
 * steps per coarse interval; the coarser levels m. */
static int mg_factor(const mg_ctx *C, int level) { return level == 0 ? C->m * C->tm : C->m; }

/* v_out = Phi_level(v_in) (+ g if non-NULL); k = index (1-based) of the step
 * on the finest level, which selects its forcing (the coarser levels carry no
 * forcing: FAS cancels it, Alg. 2). */
static void mg_step(mg_ctx *C, int level, int k, const double *v_in, const double *gk, double *v_out)
{
    long long n = C->P->off[C->g + 1] - C->P->off[C->g];
    double dtl = C->dt / C->tm;
    for (int q = 0; q < level; ++q) dtl *= mg_factor(C, q);
    int st = OR_OK;
    if (level == 1 && C->coarse_kind == 1) {
        memcpy(v_out, v_in, sizeof(double) * n);
        for (int s = 0; s < mg_factor(C, 0); ++s) {
            int s2 = phi_grid(C->P, C->g, C->dt / C->tm, v_out, NULL, v_out, C->rtol, C->maxit, NULL);
            if (s2 != OR_OK) st = s2;
        }
    } else if (level == 1 && C->coarse_kind == 2) {
        net_forward_grid(C->P, C->g, dtl, C->theta, v_in, v_out, NULL, NULL);
    } else if (level >= 1 && C->coarse_kind == 3) {
        /* Two-stage singly diagonally implicit Runge-Kutta step of order 2,
         * stiffly accurate and L-stable (Alexander's scheme, gamma =
         * 1 - 1/sqrt 2): for u' = -L u the stages solve
         *   (I + gamma dT L) U1 = u_n,
         *   (I + gamma dT L) U2 = u_n - (1 - gamma) dT L U1
         *                       = (1 - beta) u_n + beta U1,  beta = (1 - gamma) / gamma,
         * (dT L U1 = (u_n - U1) / gamma) and u_{n+1} = U2; stability function
         * (1 + (1 - 2 gamma) z) / (1 - gamma z)^2.  A coarse propagator of
         * higher order than the fine backward Euler, closer to Phi^m for the
         * smooth modes; the fixed point of MGRIT stays the fine solution. */
        const double gam = 1.0 - 1.0 / sqrt(2.0), beta = (1.0 - gam) / gam;
        double *u1 = malloc(sizeof(double) * n), *b2 = malloc(sizeof(double) * n);
        st = phi_grid(C->P, C->g, gam * dtl, v_in, NULL, u1, C->rtol, C->maxit, NULL);
        for (long long j = 0; j < n; ++j) b2[j] = (1.0 - beta) * v_in[j] + beta * u1[j];
        int s2 = phi_grid(C->P, C->g, gam * dtl, b2, NULL, v_out, C->rtol, C->maxit, NULL);
        if (s2 != OR_OK) st = s2;
        free(u1); free(b2);
    } else if (level >= 1 && C->coarse_kind == 4) {
        /* Extrapolated backward Euler (Richardson extrapolation of two half
         * steps against one full step): 2 BE(dT/2)^2 - BE(dT), second order
         * and A-stable, stability function 2 / (1 - z/2)^2 - 1 / (1 - z).
         * It approximates m fine backward-Euler steps closely over the whole
         * decaying spectrum (smooth modes to second order, stiff ones damped
         * like 1/z), which makes MGRIT's coarse correction accurate. */
        double *h = malloc(sizeof(double) * n), *f1 = malloc(sizeof(double) * n);
        st = phi_grid(C->P, C->g, 0.5 * dtl, v_in, NULL, h, C->rtol, C->maxit, NULL);
        int s2 = phi_grid(C->P, C->g, 0.5 * dtl, h, NULL, h, C->rtol, C->maxit, NULL);
        if (s2 != OR_OK) st = s2;
        s2 = phi_grid(C->P, C->g, dtl, v_in, NULL, f1, C->rtol, C->maxit, NULL);
        if (s2 != OR_OK) st = s2;
        for (long long j = 0; j < n; ++j) v_out[j] = 2.0 * h[j] - f1[j];
        free(h); free(f1);
    } else {
        const double *f = (level == 0 && C->F) ? C->F + (long long)((k - 1) / C->tm) * C->nt : NULL;
        st = phi_grid(C->P, C->g, dtl, v_in, f, v_out, C->rtol, C->maxit, NULL);
    }
    if (st != OR_OK) C->status = st;
    if (gk)
        for (long long j = 0; j < n; ++j) v_out[j] += gk[j];
}

/* One step of the level-`level` propagator of the MGRIT hierarchy (fine step
 * dt, coarsening m, coarse kind 0 or 3) on every grid: out = Phi_level(in).
 * Exposed to pin the coarse propagators against their closed forms.      */
int or_coarse_step(void *vp, double dt, int m, int level, int coarse_kind, double rtol, const double *in,
                   double *out)
{
    or_problem *P = (or_problem *)vp;
    if (level < 0 || m < 1 || (coarse_kind != 0 && coarse_kind != 3 && coarse_kind != 4)) return OR_EINVAL;
    int worst = OR_OK;
    for (int g = 0; g < P->G; ++g) {
        mg_ctx C = {P, g, dt, m, level + 1, rtol, 100000, coarse_kind, NULL, 0, OR_OK, NULL, P->off[P->G], 1};
        mg_step(&C, level, 1, in + P->off[g], NULL, out + P->off[g]);
        if (C.status != OR_OK) worst = C.status;
    }
    return worst;
}

/* One two-level FAS cycle on level `level` (Alg. 2 with FCF relaxation),
 * recursing on the coarse problem when level + 1 < nlev - 1, and solving the
 * coarsest level by a sequential sweep.  v has N+1 states, g has N+1
 * (entry 0 unused) or is NULL.  Returns max_j ||r_j||_2 over the C-points,
 * measured after the FCF relaxation (Sec. 4.1 stopping rule).             */
static double mg_cycle(mg_ctx *C, int level, int N, double *v, const double *g)
{
    long long n = C->P->off[C->g + 1] - C->P->off[C->g];
    int m = mg_factor(C, level);
    int Nc = N / m;
#define V(k) (v + (long long)(k) * n)
#define GF(k) (g ? g + (long long)(k) * n : NULL)
    /* F-relaxation: inside every coarse interval j, propagate from the
     * C-point jm over the F-points jm+1 .. jm+m-1. */
    for (int j = 0; j < Nc; ++j)
        for (int i = 1; i < m; ++i) mg_step(C, level, j * m + i, V(j * m + i - 1), GF(j * m + i), V(j * m + i));
    /* relax_f = 1: F-relaxation on the finest level; 2: on every level */
    if (!((level == 0 || C->relax_f == 2) && C->relax_f)) {
        /* C-relaxation: one step into every C-point. */
        for (int j = 1; j <= Nc; ++j) mg_step(C, level, j * m, V(j * m - 1), GF(j * m), V(j * m));
        /* F-relaxation again (FCF, Sec. 4.1). */
        for (int j = 0; j < Nc; ++j)
            for (int i = 1; i < m; ++i) mg_step(C, level, j * m + i, V(j * m + i - 1), GF(j * m + i), V(j * m + i));
    }
    /* C-point residual r_j = Phi(v_{jm-1}) + g_{jm} - v_{jm}; utilde_j keeps
     * Phi(v_{jm-1}) + g_{jm}. */
    double *ut = malloc(sizeof(double) * (size_t)(Nc + 1) * n);
    double rmax = 0.0;
    for (int j = 1; j <= Nc; ++j) {
        double *u_j = ut + (long long)j * n;
        mg_step(C, level, j * m, V(j * m - 1), GF(j * m), u_j);
        double rr = 0.0;
        for (long long t = 0; t < n; ++t) { double r = u_j[t] - V(j * m)[t]; rr += r * r; }
        double rn = sqrt(rr);
        if (rn > rmax || rn != rn) rmax = rn;
    }
    /* Coarse FAS problem (Alg. 2, restriction + coarse solve):
     *   w_0 = v_0,  w_j = Phi_c(w_{j-1}) + gc_j,
     *   gc_j = utilde_j - Phi_c(v_{(j-1)m})   (restricted solution + residual). */
    double *w = malloc(sizeof(double) * (size_t)(Nc + 1) * n);
    double *gc = malloc(sizeof(double) * (size_t)(Nc + 1) * n);
    double *tmp = malloc(sizeof(double) * n);
    for (int j = 0; j <= Nc; ++j) memcpy(w + (long long)j * n, V(j * m), sizeof(double) * n);
    for (int j = 1; j <= Nc; ++j) {
        mg_step(C, level + 1, 0, V((j - 1) * m), NULL, tmp);
        for (long long t = 0; t < n; ++t) gc[(long long)j * n + t] = ut[(long long)j * n + t] - tmp[t];
    }
    if (level + 1 == C->nlev - 1) {
        for (int j = 1; j <= Nc; ++j)
            mg_step(C, level + 1, 0, w + (long long)(j - 1) * n, gc + (long long)j * n, w + (long long)j * n);
    } else {
        mg_cycle(C, level + 1, Nc, w, gc);
    }
    /* Correction at the C-points: v_{jm} <- v_{jm} + (w_j - v_{jm}) = w_j.
     * The F-points are refreshed by the F-relaxation that opens the next
     * cycle (prolongation = injection + F-relaxation). */
    for (int j = 1; j <= Nc; ++j) memcpy(V(j * m), w + (long long)j * n, sizeof(double) * n);
    free(ut); free(w); free(gc); free(tmp);
#undef V
#undef GF
    return rmax;
}

/* CTMGRIT^loc with s = 1 (Alg. 3): independent MGRIT on every grid, each
 * stopping when all its C-point residual norms are <= tol (Sec. 4.1), then
 * the caller combines.  The initial guess is u0 at every time point, or
 * (init = 1) one sweep of the level-1 propagator over the C-points.
 * Returns u_N on every grid in uT; iters[g] = cycles used; res_hist[g*maxit+k]
 * = residual measured in cycle k (when non-NULL). */
int or_mgrit(void *vp, const double *u0, double dt, int nsteps, int m, int nlev, double tol,
             int maxit, int coarse_kind, const double *theta, double rtol, int krylov_maxit,
             double *uT, int *iters, double *res_hist, const unsigned char *gmask /* G or NULL */,
             int relax_f /* 1: F-relaxation on the finest level instead of FCF, 2: on every level */,
             int init /* 1: initial C-points from one sweep of the level-1 propagator;
                         2: that sweep with the extrapolated backward Euler */,
             const double *F /* forcing f_n, n = 1..nsteps, packed like states, or NULL */,
             const int *tmul /* per grid steps per common step (own time partition), or NULL */)
{
    or_problem *P = (or_problem *)vp;
    if (m < 2 || nlev < 2) return OR_EINVAL;
    long long div = 1;
    for (int q = 0; q < nlev - 1; ++q) div *= m;
    if (nsteps % div != 0) return OR_EINVAL;
    long long ntot = P->off[P->G];
    int worst = OR_OK;
#pragma omp parallel for schedule(dynamic)
    for (int g = 0; g < P->G; ++g) {
        if (gmask && !gmask[g]) continue;
        long long n = P->off[g + 1] - P->off[g];
        int tm = tmul ? tmul[g] : 1;
        int Ng = nsteps * tm;   /* steps of the grid's own partition */
        double *v = malloc(sizeof(double) * (size_t)(Ng + 1) * n);
        for (int k = 0; k <= Ng; ++k) memcpy(v + (long long)k * n, u0 + P->off[g], sizeof(double) * n);
        mg_ctx C = {P, g, dt, m, nlev, rtol, krylov_maxit, coarse_kind, theta, relax_f, OR_OK,
                    F ? F + P->off[g] : NULL, ntot, tm};
        int m0 = m * tm;
        if (init) {
            /* initial guess at the C-points: u_{jm} = Phi_c(u_{(j-1)m}); the
             * F-points follow from the first relaxation */
            /* init = 2: this sweep with the extrapolated backward Euler
             * (coarse kind 4); the cycles keep their coarse propagator */
            const int ck = C.coarse_kind;
            if (init == 2) C.coarse_kind = 4;
            for (int j = 1; j <= Ng / m0; ++j)
                mg_step(&C, 1, 0, v + (long long)(j - 1) * m0 * n, NULL, v + (long long)j * m0 * n);
            C.coarse_kind = ck;
        }
        int it = 0, conv = 0;
        while (it < maxit) {
            double r = mg_cycle(&C, 0, Ng, v, NULL);
            if (res_hist) res_hist[(long long)g * maxit + it] = r;
            ++it;
            if (r <= tol) { conv = 1; break; }
        }
        memcpy(uT + P->off[g], v + (long long)Ng * n, sizeof(double) * n);
        if (iters) iters[g] = it;
        int st = C.status != OR_OK ? C.status : (conv ? OR_OK : OR_ENOCONV);
        if (st != OR_OK) {
#pragma omp critical
            worst = st;
        }
        free(v);
    }
    return worst;
}

/* ------------------------------------------------------------------------ */
/* Combination (Eq. "combination_technique_solution"): u^(c)(x) =
 * sum_l c_l I_l[u_l](x) with I_l the piecewise d-linear interpolant on
 * Omega_l, zero on the boundary (Sec. 2.2.2, interior nodal basis).       */
static double interp_grid(const or_problem *P, int g, const double *u, const double *x)
{
    geom G = grid_geom(P, g);
    const int *l = P->lev + (size_t)g * P->d;
    long long cell[OR_MAXD];
    double t[OR_MAXD];
    for (int i = 0; i < G.d; ++i) {
        long long M = 1LL << l[i];           /* nodes 0..M, 0 and M on the boundary */
        double s = (x[i] - G.lo[i]) / G.h[i];
        long long k = (long long)floor(s);
        if (k < 0) k = 0;
        if (k > M - 1) k = M - 1;
        cell[i] = k;
        t[i] = s - (double)k;
    }
    double val = 0.0;
    for (int corner = 0; corner < (1 << G.d); ++corner) {
        double w = 1.0;
        long long idx = 0;
        int inside = 1;
        for (int i = 0; i < G.d; ++i) {
            int bit = (corner >> i) & 1;
            long long node = cell[i] + bit;   /* paper numbering 0..M */
            w *= bit ? t[i] : (1.0 - t[i]);
            if (node <= 0 || node >= (1LL << l[i])) { inside = 0; }
            else idx += (node - 1) * G.S[i];
        }
        if (inside) val += w * u[idx];
    }
    return val;
}

int or_combine(void *vp, const double *u, int npts, const double *pts, double *out)
{
    or_problem *P = (or_problem *)vp;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < npts; ++k) {
        double acc = 0.0;
        for (int g = 0; g < P->G; ++g)
            acc += P->coef[g] * interp_grid(P, g, u + P->off[g], pts + (long long)k * P->d);
        out[k] = acc;
    }
    return OR_OK;
}

/* Interpolation of one grid's nodal vector at points (used by the tests). */
int or_interp(void *vp, int g, const double *ug, int npts, const double *pts, double *out)
{
    or_problem *P = (or_problem *)vp;
    for (int k = 0; k < npts; ++k) out[k] = interp_grid(P, g, ug, pts + (long long)k * P->d);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Recombination (Sec. 2.2.2).  Hierarchical basis of one axis of a grid of
 * level l: the interior node with 1-based index J (x = a + J h) has
 * hierarchical level l - t, t the number of trailing zero bits of J, and
 * hierarchical parents J - 2^t and J + 2^t (index 0 or 2^l lies on the
 * boundary, value 0).  Hierarchization replaces every nodal value by its
 * surplus over the linear interpolant of its two parents,
 *   s_J = u_J - (u_{J - 2^t} + u_{J + 2^t}) / 2,
 * finest level first (the parents still hold nodal values); the inverse adds
 * the parents' mean back, coarsest level first.  In d dimensions the 1-D
 * transform is applied along every axis in turn (H_l of Eq.
 * "overall_combination_operator" is their tensor product).                 */
static int trailing_zeros(long long J)
{
    int t = 0;
    while (!(J & 1)) { J >>= 1; ++t; }
    return t;
}

static void hier_axis(const geom *G, int i, int lev, double *v, int inverse)
{
    long long N = G->N[i], S = G->S[i];
    for (long long j0 = 0; j0 < G->n; ++j0) {
        if ((j0 / S) % N != 0) continue;            /* first node of a line along axis i */
        for (int k = 0; k < lev; ++k) {
            int t = inverse ? lev - 1 - k : k;
            long long step = 1LL << t;
            for (long long J = step; J <= N; J += 2 * step) {  /* odd multiples of 2^t */
                double left = (J - step >= 1) ? v[j0 + (J - step - 1) * S] : 0.0;
                double right = (J + step <= N) ? v[j0 + (J + step - 1) * S] : 0.0;
                double mean = 0.5 * (left + right);
                v[j0 + (J - 1) * S] += inverse ? mean : -mean;
            }
        }
    }
}

/* out = H_l u (inverse = 0) or H_l^{-1} u (inverse = 1) on every grid. */
int or_hierarchize(void *vp, const double *u, double *out, int inverse)
{
    or_problem *P = (or_problem *)vp;
    memmove(out, u, sizeof(double) * P->off[P->G]);
#pragma omp parallel for schedule(dynamic)
    for (int g = 0; g < P->G; ++g) {
        geom G = grid_geom(P, g);
        const int *l = P->lev + (size_t)g * P->d;
        for (int i = 0; i < P->d; ++i) hier_axis(&G, i, l[i], out + P->off[g], inverse);
    }
    return OR_OK;
}

/* out = Q u = H^{-1} Qbar H u (Eq. "overall_combination_operator"): the
 * surplus of node i of grid l becomes the sum, over every grid m that has a
 * node at the same coordinates (the set S(i, Omega_l)), of m's combination
 * coefficient times m's surplus there (Eq. "recombination_operator").  The
 * node with 1-based indices J on grid l sits at J_k / 2^{l_k} of the box
 * along axis k; grid m has it where J_k 2^{m_k - l_k} is an integer.
 * out may alias u.                                                         */
int or_recombine(void *vp, const double *u, double *out)
{
    or_problem *P = (or_problem *)vp;
    long long nt = P->off[P->G];
    double *hat = malloc(sizeof(double) * nt);
    double *sum = malloc(sizeof(double) * nt);
    or_hierarchize(vp, u, hat, 0);
#pragma omp parallel for schedule(dynamic)
    for (int g = 0; g < P->G; ++g) {
        geom G = grid_geom(P, g);
        const int *l = P->lev + (size_t)g * P->d;
        long long c[OR_MAXD];
        for (long long j = 0; j < G.n; ++j) {
            coords(&G, j, c);
            double acc = 0.0;
            for (int m = 0; m < P->G; ++m) {
                geom Gm = grid_geom(P, m);
                const int *lm = P->lev + (size_t)m * P->d;
                long long idx = 0;
                int found = 1;
                for (int k = 0; k < P->d; ++k) {
                    long long J = c[k] + 1, Jm;
                    if (lm[k] >= l[k]) {
                        Jm = J << (lm[k] - l[k]);
                    } else {
                        long long q = 1LL << (l[k] - lm[k]);
                        if (J % q) { found = 0; break; }
                        Jm = J / q;
                    }
                    idx += (Jm - 1) * Gm.S[k];
                }
                if (found) acc += P->coef[m] * hat[P->off[m] + idx];
            }
            sum[P->off[g] + j] = acc;
        }
    }
    or_hierarchize(vp, sum, out, 1);
    free(hat);
    free(sum);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Manufactured solution of the heat experiment (Sec. 4.2, Eq. "heat_equation"):
 *   u*(x, t) = rho e^{-t} S(x),  rho = sqrt(|x|^2 + t^2),
 *   S(x) = prod_i sin(pi xi_i),  xi_i = (x_i - a_i) / (b_i - a_i),
 * and the forcing f = d(u^*)/dt - Laplace u* that makes it the exact solution:
 *   d(u^*)/dt = e^{-t} S (t / rho - rho),
 *   Laplace u* = e^{-t} (S Laplace rho + 2 grad rho . grad S + rho Laplace S),
 *   grad rho = x / rho,  Laplace rho = d / rho - |x|^2 / rho^3,
 *   d S / d x_i = (pi / w_i) cos(pi xi_i) prod_{k != i} sin(pi xi_k),
 *   Laplace S = -pi^2 sum_i S / w_i^2,  w_i = b_i - a_i.                   */
static double manufactured(const or_problem *P, const double *x, double t, int forcing)
{
    int d = P->d;
    double r2 = 0.0, S = 1.0;
    for (int i = 0; i < d; ++i) {
        r2 += x[i] * x[i];
        S *= sin(M_PI * (x[i] - P->lo[i]) / (P->hi[i] - P->lo[i]));
    }
    double rho = sqrt(r2 + t * t);
    double et = exp(-t);
    if (!forcing) return rho * et * S;
    double ut = et * S * (t / rho - rho);
    double lap_rho = d / rho - r2 / (rho * rho * rho);
    double grad = 0.0, lapS = 0.0;
    for (int i = 0; i < d; ++i) {
        double w = P->hi[i] - P->lo[i];
        double dS = (M_PI / w) * cos(M_PI * (x[i] - P->lo[i]) / w);
        for (int k = 0; k < d; ++k)
            if (k != i) dS *= sin(M_PI * (x[k] - P->lo[k]) / (P->hi[k] - P->lo[k]));
        grad += (x[i] / rho) * dS;
        lapS -= M_PI * M_PI * S / (w * w);
    }
    double lap = et * (S * lap_rho + 2.0 * grad + rho * lapS);
    return ut - lap;
}

/* ------------------------------------------------------------------------ */
/* Initial values sampled at the interior nodes of every grid.
 * kind 0: sum of K product-sine modes, params = [K, (A_k, m_k1..m_kd)_k]:
 *         u0(x) = sum_k A_k prod_i sin(pi m_ki (x_i - a_i)/(b_i - a_i))
 * kind 1: product Gaussian, params = [mean_1..mean_d, std_1..std_d]:
 *         u0(x) = prod_i exp(-(x_i - mean_i)^2 / (2 std_i^2)) / (std_i sqrt(2 pi))
 * kind 2: the manufactured solution u*(x, t) of the heat experiment, params = [t]
 * kind 3: its forcing f(x, t) = d(u^*)/dt - Laplace u*, params = [t]
 * kind 4: normal density with mean M and covariance C (the law of the
 *         linear SDE, Eq. "sde_analytical_solution"), params = [M (d), C (d x d,
 *         row major)]: (2 pi)^{-d/2} det(C)^{-1/2} exp(-(x - M)^T C^{-1} (x - M) / 2),
 *         evaluated with the Cholesky factor C = R R^T                           */
int or_initial(void *vp, int kind, const double *params, int nparams, double *out)
{
    or_problem *P = (or_problem *)vp;
    int d = P->d;
    if (kind == 0) {
        int K = (int)params[0];
        if (nparams < 1 + K * (d + 1)) return OR_EINVAL;
    } else if (kind == 1) {
        if (nparams < 2 * d) return OR_EINVAL;
    } else if (kind == 2 || kind == 3) {
        if (nparams < 1) return OR_EINVAL;
    } else if (kind == 4) {
        if (nparams < d + d * d) return OR_EINVAL;
    } else {
        return OR_EINVAL;
    }
    double R[OR_MAXD * OR_MAXD] = {0.0}, logdet = 0.0;
    if (kind == 4) {
        const double *C = params + d;
        for (int i = 0; i < d; ++i) {
            for (int k = 0; k <= i; ++k) {
                double v = C[i * d + k];
                for (int q = 0; q < k; ++q) v -= R[i * d + q] * R[k * d + q];
                if (i == k) {
                    if (!(v > 0.0)) return OR_EINVAL;
                    R[i * d + i] = sqrt(v);
                    logdet += log(R[i * d + i]);
                } else {
                    R[i * d + k] = v / R[k * d + k];
                }
            }
        }
    }
    for (int g = 0; g < P->G; ++g) {
        geom G = grid_geom(P, g);
        long long c[OR_MAXD];
        for (long long j = 0; j < G.n; ++j) {
            coords(&G, j, c);
            double x[OR_MAXD];
            for (int i = 0; i < d; ++i) x[i] = G.lo[i] + (double)(c[i] + 1) * G.h[i];
            double v = 0.0;
            if (kind == 0) {
                int K = (int)params[0];
                for (int k = 0; k < K; ++k) {
                    const double *pk = params + 1 + k * (d + 1);
                    double prod = pk[0];
                    for (int i = 0; i < d; ++i)
                        prod *= sin(M_PI * pk[1 + i] * (x[i] - P->lo[i]) / (P->hi[i] - P->lo[i]));
                    v += prod;
                }
            } else if (kind == 1) {
                v = 1.0;
                for (int i = 0; i < d; ++i) {
                    double z = (x[i] - params[i]) / params[d + i];
                    v *= exp(-0.5 * z * z) / (params[d + i] * sqrt(2.0 * M_PI));
                }
            } else if (kind == 4) {
                double z[OR_MAXD], q = 0.0;
                for (int i = 0; i < d; ++i) {
                    double r = x[i] - params[i];
                    for (int k = 0; k < i; ++k) r -= R[i * d + k] * z[k];
                    z[i] = r / R[i * d + i];
                    q += z[i] * z[i];
                }
                v = exp(-0.5 * q - logdet - 0.5 * d * log(2.0 * M_PI));
            } else {
                v = manufactured(P, x, params[0], kind == 3);
            }
            out[P->off[g] + j] = v;
        }
    }
    return OR_OK;
}
