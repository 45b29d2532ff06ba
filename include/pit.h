/*
 * pit.h -- C ABI of libpit.so, a single-GPU (GB300, sm_103a) implementation of
 * the hot path of the parallel-in-time sparse-grid combination method of
 * Griebel, Schweitzer and Troska (arXiv 2509.22156, "A parallel-in-time
 * combination method for parabolic problems"):
 *
 *   - the fine propagator Phi, one backward-Euler step (I + dt L) u = u_prev + dt f
 *     (Sec. 2, Eqs. "parabolic_problem_time_propagation" and "..._LES"),
 *     solved matrix-free by CG (symmetric operators) or BiCGStab (drift
 *     operators) as in Sec. 4.1;
 *   - on every component grid of the combination technique
 *     (Sec. 2.1.1, Eq. "combination_technique_solution");
 *   - inside two- or three-level FAS multigrid reduction in time with FCF
 *     relaxation, independently per grid (Sec. 3.3, Alg. 2; Sec. 3.4, Alg. 3);
 *   - followed by the weighted combination sum (Eq. "combination_technique_solution").
 *
 * Conventions shared by every entry point:
 *   - Vectors are FP64 in the canonical packed layout: grid g occupies
 *     [offsets[g], offsets[g+1]) of a vector of n_total values; grids are
 *     ordered by layer w ascending, then by level multi-index l
 *     lexicographically; inside a grid the interior nodes are in C order with
 *     the last axis fastest; node c_i (0-based) on axis i sits at
 *     lo_i + (c_i + 1) h_i with h_i = (hi_i - lo_i) / 2^{l_i}.  A batch of
 *     n_batch vectors is n_batch consecutive packed vectors.
 *   - Pointers are caller-owned.  Where a parameter says "host or device", the
 *     library detects the memory kind (cudaPointerGetAttributes) and stages
 *     host data through its own device buffers.  Where it says "device", it
 *     must be device memory of the problem's GPU.
 *   - All work is ordered on the CUDA stream given at creation.  Functions
 *     that return statistics or decide on convergence synchronise that stream
 *     before returning; the others are asynchronous.
 *   - No C++ exception crosses the ABI.  Every function returns a pit_status;
 *     pit_last_error() gives a thread-local message for the last failure.
 *     Invalid sizes, levels and options are rejected before any launch.
 *   - The library never falls back to a CPU path: without a usable CUDA device
 *     pit_problem_create returns PIT_ERR_CUDA.
 */
#ifndef PIT_H
#define PIT_H

#ifdef __cplusplus
extern "C" {
#endif

#define PIT_MAX_DIM 6
#define PIT_MAX_HIST 64

typedef struct pit_problem *pit_problem_t; /* opaque, owned by the library */

typedef enum {
    PIT_OK = 0,
    PIT_ERR_INVALID_ARG = 1,
    PIT_ERR_CUDA = 2,
    PIT_ERR_OOM = 3,
    PIT_ERR_NOCONV = 4,     /* a Krylov solve or MGRIT hit its iteration cap   */
    PIT_ERR_BREAKDOWN = 5,  /* Krylov breakdown (zero denominator)              */
    PIT_ERR_NONFINITE = 6,  /* NaN or Inf met in a residual or input            */
    PIT_ERR_TIMEOUT = 7,    /* a bounded device-side wait gave up               */
    PIT_ERR_UNSUPPORTED = 8 /* valid request outside what this build supports   */
} pit_status;

typedef enum {
    PIT_OP_HEAT = 0,    /* L = -Laplace (Sec. 4.2, Eq. "heat_equation"), (2d+1)-point stencil */
    PIT_OP_VARHEAT = 1, /* L = -div(a grad), a = 1 + A sin(2 pi x1) cos(2 pi x2) sin(2 pi x3)...
                           evaluated at face midpoints; symmetric, CG                        */
    PIT_OP_OU = 2,      /* Fokker-Planck operator of dX = -theta X dt + sigma dW
                           (Sec. 4.4, Eq. "sde_fokker_planck" with diagonal drift):
                           donor-cell upwind drift + central diffusion; BiCGStab            */
    PIT_OP_LSDE = 3,    /* Fokker-Planck operator of the linear SDE dX = A X dt + sigma dW
                           (Sec. 4.4, Eqs. "sde", "sde_fokker_planck"), A = drift (d x d),
                           H = 2 sigma D sigma^T = diffusion (d x d):
                           L p = sum_i d_i((A x)_i p) - (1/2) sum_ij H_ij d_i d_j p, drift
                           flux with face velocity (A x)_i (donor cell or central, see
                           pit_drift_scheme), central diagonal diffusion, and for i != k the
                           four-point mixed stencil
                           (p_{++} - p_{+-} - p_{-+} + p_{--}) / (4 h_i h_k); BiCGStab      */
    PIT_OP_CME = 4      /* Fokker-Planck form of the chemical master equation (Sec. 4.3,
                           Eq. "cme_fp") of the toggle-switch networks (Tables
                           "toggle_switch_2d", "toggle_switch_3d"): species i is produced at
                           a_i = cme_prod[i] / (cme_sat[i] + y_i^cme_exp[i]), y_i the sum of
                           the other species' counts, and degraded at b_i = cme_deg[i] x_i:
                           L u = sum_i d_i((a_i - b_i) u) - (1/2) d_i^2((a_i + b_i) u), drift
                           flux as for PIT_OP_LSDE (pit_drift_scheme) with the face velocity
                           a_i - b_i, diffusion the second difference of (a_i + b_i) u;
                           the box must lie in x >= 0; BiCGStab                              */
} pit_op;

/* Drift flux of the linear-SDE operator at the face x_{j+1/2 e_i} with face
 * velocity v = (A x)_i there:
 *   PIT_DRIFT_UPWIND   donor cell, F = max(v,0) p_j + min(v,0) p_{j+e_i}
 *                      (first order; monotone)
 *   PIT_DRIFT_CENTRAL  F = v (p_j + p_{j+e_i}) / 2 (second order, the paper's
 *                      "second order finite difference" of Sec. 4.4.1; the
 *                      drift part of L is then skew up to its diagonal
 *                      trace(A) / 2 per axis sum)
 * for PIT_OP_LSDE and PIT_OP_CME; the OU operator always uses the donor cell. */
typedef enum { PIT_DRIFT_UPWIND = 0, PIT_DRIFT_CENTRAL = 1 } pit_drift_scheme;

typedef enum { PIT_PREC_FP64 = 0, PIT_PREC_MIXED = 1, PIT_PREC_FP32 = 2, PIT_PREC_MIXED_PAIR = 3 } pit_prec;

typedef enum {
    PIT_COARSE_IMPLICIT = 0, /* Phi_coarse = backward Euler with dT = m dt (Sec. 3.3.1)  */
    PIT_COARSE_EXACT = 1,    /* Phi_coarse = m fine steps (exact coarse correction)        */
    PIT_COARSE_LEARNED = 2,  /* learned network (not in the paper; see pit_train_coarse); the
                                implicit step replaces it when it was not accepted, and for
                                the remaining cycles when a cycle's residual fails to drop
                                below 0.9 times the previous one or is not finite          */
    PIT_COARSE_SDIRK2 = 3,   /* not in the paper: every coarse level steps with the two-stage
                                L-stable SDIRK scheme of order 2 (gamma = 1 - 1/sqrt 2):
                                (I + gamma dT L) U1 = u_n, (I + gamma dT L) U2 = -sqrt 2 u_n
                                + (1 + sqrt 2) U1, u_{n+1} = U2.  Two solves per coarse step,
                                closer to m fine backward-Euler steps than one with dT for
                                the smooth modes, so MGRIT needs fewer cycles; its fixed
                                point is still the fine solution.  The coarse solves must be
                                PIT_PREC_MIXED or PIT_PREC_FP32 (PIT_ERR_UNSUPPORTED
                                otherwise); not with the residual mode or global MGRIT    */
    PIT_COARSE_EXTRAP = 4    /* not in the paper: every coarse level steps with the
                                extrapolated backward Euler 2 BE(dT/2)^2 - BE(dT) (three
                                solves per coarse step, second order, A-stable).  Its
                                error against m fine backward-Euler steps is small over the
                                whole decaying spectrum (smooth modes to second order, stiff
                                ones damped like 1/(lambda dT)), so MGRIT needs fewer
                                cycles; its fixed point is still the fine solution.  Heat
                                operators (constant and variable coefficient; the latter's
                                coefficient table is switched to the full step in place)
                                with PIT_PREC_MIXED or PIT_PREC_FP32 coarse solves
                                (PIT_ERR_UNSUPPORTED otherwise; the FP32 form keeps u_n and
                                the second half step's result in a library-owned global
                                slab of n_batch x n_total floats); not with the residual
                                mode or global MGRIT                                      */
} pit_coarse;

/* Problem: d-dimensional box [lo, hi], zero Dirichlet values, combination
 * level level_n (the paper's L) with minimum level level0 (the paper's L0,
 * Sec. 2.1.1), operator op with parameters theta, sigma (OU), vamp
 * (variable-coefficient amplitude A), and drift, diffusion (linear SDE: the
 * d x d matrices A and H, row major, first d*d entries used), the reaction
 * rates cme_prod, cme_sat, cme_exp, cme_deg of the toggle-switch chemical
 * master equation (one entry per species; finite, cme_prod and cme_deg >= 0,
 * cme_sat > 0, and lo >= 0 on every axis, else PIT_ERR_INVALID_ARG), and the
 * drift flux drift_scheme (pit_drift_scheme; must be PIT_DRIFT_UPWIND for the
 * heat, variable-coefficient and OU operators, else PIT_ERR_INVALID_ARG). */
typedef struct {
    int d;
    int level_n;
    int level0;
    int op;
    double lo[PIT_MAX_DIM];
    double hi[PIT_MAX_DIM];
    double theta;
    double sigma;
    double vamp;
    double drift[PIT_MAX_DIM * PIT_MAX_DIM];
    double diffusion[PIT_MAX_DIM * PIT_MAX_DIM];
    int drift_scheme;
    double cme_prod[PIT_MAX_DIM];
    double cme_sat[PIT_MAX_DIM];
    double cme_exp[PIT_MAX_DIM];
    double cme_deg[PIT_MAX_DIM];
} pit_problem_desc;

/* Options of one batched backward-Euler solve.
 *   prec = PIT_PREC_FP64:  Krylov in FP64 until ||b - A x||_2 <= rtol ||b||_2
 *                          or maxit iterations.
 *   prec = PIT_PREC_MIXED: FP64 iterative refinement: r = b - A x in FP64,
 *                          FP32 Krylov on A e = r to relative
 *                          max(inner_rtol, 0.5 rtol ||b|| / ||r||) (at most maxit
 *                          iterations), x += e in FP64; at most ir_maxit
 *                          passes; the same FP64 stopping rule.
 *   prec = PIT_PREC_FP32:  Krylov in FP32 on a copy of the state scaled by a
 *                          power of two (inputs and outputs stay FP64) until
 *                          the FP32 recurrence residual meets rtol; for solves
 *                          whose tolerance lies far above FP32 rounding, such
 *                          as the coarse correction solves of MGRIT (rtol of
 *                          1e-5 or looser).  Values below 2^-126 of the largest
 *                          input are flushed to zero.  Grids whose FP32 state
 *                          does not fit in shared memory are solved in the
 *                          PIT_PREC_MIXED form with their FP64 state in global
 *                          memory, to the same rtol on the true residual.
 *   prec = PIT_PREC_MIXED_PAIR: the refinement of PIT_PREC_MIXED with the
 *                          state held as pairs of FP32 numbers (hi + lo, about
 *                          48 significant bits, scaled by a power of two) and
 *                          the residual b - A x formed from the pairs by
 *                          error-free FP32 transformations (two-sum, two-product
 *                          by FMA) with one compensation term, without FP64
 *                          arithmetic (which GB300 runs at 1/58 of the FP32
 *                          rate).  The residual's floor is about 2^-48 (1 + 4
 *                          sum_i dt / h_i^2) |x|, 32 times the FP64 residual's
 *                          (2^-53 for 2^-48): about 1e-14 of ||b|| where
 *                          dt / h^2 is of order one, near 1e-12 where it is in
 *                          the hundreds; choose rtol above it.  Same options and stopping rule as
 *                          PIT_PREC_MIXED.  Heat and variable-coefficient
 *                          operators (the latter through its face coefficients
 *                          dt a / h^2, also held as pairs); the drift operator
 *                          gives PIT_ERR_UNSUPPORTED.  Grids whose state does
 *                          not fit in shared memory keep their pairs in global
 *                          memory, as PIT_PREC_MIXED keeps its FP64 state.
 *                          Inputs and outputs stay FP64; values below 2^-102 of
 *                          the state's norm lose their low part. */
/* Preconditioner of the Krylov solves (the paper preconditions its CG and
 * BiCGStab by domain decomposition, Sec. 2.1.2 and Sec. 4.1; on one GPU the
 * grid-resident solver offers these):
 *   DEFAULT  heat operator: the line preconditioner (tridiagonal along the
 *            finest axis, in the FP32 Krylov forms on anisotropic grids at
 *            stiff steps); other operators: none.
 *   NONE     no preconditioner.
 *   JACOBI   diagonal (Jacobi) preconditioning of the FP32 correction solves
 *            of the refinement forms (PIT_PREC_MIXED, PIT_PREC_MIXED_PAIR) for
 *            the variable-coefficient and drift (OU) operators, applied as
 *            the symmetric scaling D^{-1/2} A D^{-1/2}; elsewhere as NONE. */
typedef enum { PIT_PRECOND_DEFAULT = 0, PIT_PRECOND_NONE = 1, PIT_PRECOND_JACOBI = 2 } pit_precond;

/* Initial guess of each backward-Euler step's solve in the refinement form
 * PIT_PREC_MIXED (the paper fixes none; it changes how many refinement passes
 * a step takes, not the stopping rule or the fixed point):
 *   DEFAULT      EXTRAPOLATE.
 *   PREVIOUS     the previous state x_{s-1}.
 *   EXTRAPOLATE  from the third step of a call on, when a step has no forcing
 *                and no caller guess: the linear extrapolation
 *                2 x_{s-1} - x_{s-2}.  Its initial residual is formed without
 *                a stencil pass from the FP64 residuals of the two previous
 *                steps (A (x_{s-1} - x_{s-2}) = A x_{s-1} - A x_{s-2}, each
 *                known from its step's check), so for smooth solutions a step
 *                starts near (dt lambda)^2 |x| instead of dt lambda |x| and
 *                often needs one FP32 correction instead of two.
 * Other precision forms ignore it. */
typedef enum { PIT_GUESS_DEFAULT = 0, PIT_GUESS_PREVIOUS = 1, PIT_GUESS_EXTRAPOLATE = 2 } pit_guess;

typedef struct {
    int prec;
    double rtol;
    int maxit;
    double inner_rtol;
    int ir_maxit;
    int precond;          /* pit_precond */
    int guess;            /* pit_guess */
} pit_solve_opts;

typedef struct {
    int n_items;          /* (batch entry, grid) pairs solved                  */
    int n_failed;         /* items that did not meet rtol                      */
    int max_iters;        /* largest Krylov iteration count of one item        */
    long long sum_iters;  /* Krylov iterations summed over items               */
    int max_refine;       /* largest number of refinement passes (mixed)       */
    int status;           /* worst item status as a pit_status                  */
} pit_phi_stats;

/* Relaxation of the finest MGRIT level (Sec. 3.3.1 defines F- and C-relaxation;
 * the experiments of Sec. 4.1 use FCF).  Coarser levels of a three-level
 * hierarchy use FCF, except with PIT_RELAX_F_ALL. */
typedef enum {
    PIT_RELAX_FCF = 0,  /* F-, C- and F-relaxation before the residual (Sec. 4.1) */
    PIT_RELAX_F = 1,    /* F-relaxation only: half the fine steps per cycle, exactness
                           advances one coarse interval per cycle instead of two    */
    PIT_RELAX_F_ALL = 2 /* F-relaxation on the finest and on the middle level of a
                           three-level hierarchy                                      */
} pit_relax;

/* MGRIT options (Sec. 3.3, Alg. 2; Sec. 4.1 stopping rule: a grid stops when
 * all its C-point residual l2 norms are <= tol).
 * nsteps must be a multiple of m^(levels-1). */
typedef struct {
    double t0, t1;
    int nsteps;
    int m;
    int levels;           /* 2 or 3 */
    double tol;
    int maxit;            /* MGRIT cycle cap */
    int coarse;           /* pit_coarse */
    int fas;              /* 1: FAS form of Alg. 2 as printed; 0: with a linear coarse
                             propagator (implicit), solve the coarse problem for the
                             correction (Sec. 3.3.1 notes this for linear problems), so
                             that crs.rtol is relative to the correction            */
    pit_solve_opts fine;  /* options of every fine-level Phi solve   */
    pit_solve_opts crs;   /* options of every coarse-level Phi solve */
    int relax;            /* pit_relax of the finest level           */
    int lanes;            /* concurrent grid groups (Alg. 3 runs MGRIT per grid): 0 = library
                             default (5), 1 = all grids in lockstep; more than one lane is
                             used with the correction form and the implicit coarse step only
                             (a learned propagator that was not accepted counts as implicit),
                             other forms run as one lane                                    */
    int init;             /* initial guess: 0 = u0 at every time point; 1 = one sweep of the
                             level-1 coarse propagator from u0 over the C-points (the paper
                             leaves the initial guess open; the fixed point is the same);
                             2 = that sweep with the extrapolated backward Euler of
                             PIT_COARSE_EXTRAP while the cycles keep `coarse` (heat
                             operators, PIT_PREC_MIXED or PIT_PREC_FP32 coarse solves,
                             any coarse propagator but PIT_COARSE_EXACT;
                             PIT_ERR_UNSUPPORTED otherwise)                                 */
    int recomb;           /* recombination steps s of Alg. 3 (Sec. 2.2.1): 0 = none (one MGRIT
                             solve over [t0, t1], combined afterwards by pit_combine); s >= 1:
                             [t0, t1] is split at tau_k = t0 + k (t1 - t0) / s, and before each
                             of the s intervals every grid's state is replaced by the projection
                             of the combined solution onto its grid (pit_recombine); nsteps
                             must then be a multiple of s m^(levels-1)                        */
    const double *forcing; /* device, nsteps packed states or NULL: f_n of the fine steps
                             n = 1..nsteps in (I + dt L) u_n = u_{n-1} + dt f_n (Eq.
                             "parabolic_problem_time_propagation_LES"); the coarse levels
                             carry none (the FAS / correction coarse problem cancels it)     */
    const int *tmul;      /* host, G ints in 1..4096, or NULL: each grid's own time partition
                             (Sec. 2.2.1): grid g takes tmul[g] steps of dt / tmul[g] inside
                             each fine step n, all with f_n; the coarse step dT = m dt is
                             common.  Grids with different tmul run as separate lanes, which
                             needs the correction form with the implicit coarse step        */
    int global_every;     /* 0: MGRIT on every subproblem independently (CTMGRIT^loc, Alg. 3).
                             r >= 1: global MGRIT (Sec. 3.4: MGRIT on the whole combination
                             problem): the propagator of r fine steps is Phi^r o Q, Q the
                             recombination (pit_recombine), so all grids are coupled every r
                             steps and iterate together until the largest C-point residual
                             of all grids meets tol; its fixed point is Alg. 1 with a
                             recombination step every r fine steps.  r must divide m; two
                             levels, F-relaxation, implicit coarse step Phi_c o Q in the
                             correction form, no tmul or recomb                              */
    int residual;         /* 1: residual mode (the XBraid option of Sec. 4.4.1): the fine
                             steps of the F-relaxation are the fine solves as configured, for
                             instance a fixed small number of Krylov iterations (fine.rtol 0,
                             fine.maxit k; hitting the caps is then not a failure), the C-point
                             residual is the space-time residual of the backward-Euler
                             equation rho_j = u_{jm-1} + dt f_{jm} - (I + dt L) u_{jm}, the
                             coarse problem (I + dT L) e_j = e_{j-1} + rho_j, and MGRIT stops
                             when every ||rho_j||_2 <= tol.  With exact fine solves its fixed
                             point is the sequential solution.  Two levels, F-relaxation,
                             implicit coarse step, correction form, no tmul                  */
} pit_mgrit_opts;

typedef struct {
    int max_cycles;                 /* cycles of the slowest grid                   */
    int n_converged;                /* grids that met tol                           */
    double res_hist[PIT_MAX_HIST];  /* max over grids of the residual, per cycle    */
    long long phi_items;            /* (state, grid) backward-Euler solves executed  */
    long long krylov_iters;         /* Krylov iterations summed over all solves      */
    long long point_iters;          /* Krylov iterations weighted by grid nodes      */
    int learned_used;               /* 1 if the learned coarse propagator was used   */
    int fallback;                   /* 1 if it was replaced by the implicit one      */
    double ms;                      /* wall time of the call                        */
} pit_mgrit_stats;

/* ---------------------------------------------------------------------------
 * Learned coarse propagator (not in the paper): an axis-separable network that
 * replaces the coarse-level backward-Euler step Phi_c of MGRIT (Sec. 3.3.1).
 * Phi_hat(u) = u + sigma h4(u / sigma), sigma the RMS of u on the grid; four
 * layers of width-5 convolutions along every axis with weights shared by all
 * axes, channels (u, a, s_i) -> 16 -> 16 -> 16 -> 1, ReLU on the hidden
 * layers; a = diffusion coefficient at the nodes (1 for constant-coefficient
 * operators), s_i = 1 / (1 + 4 dT / h_i^2) per axis; taps outside the grid read
 * zero.  Parameter block (PIT_NET_PARAMS floats): for layer k = 0..3 the
 * weights W_k[o][c][t] (Cout x Cin x 5, Cin = 3, 17, 17, 17; c = Cin-1 is the
 * s channel; t = 0..4 is the tap at offset t-2), then the biases b_k[o].
 * Weights are used rounded to BF16 (nearest even); activations and
 * accumulation are FP32, the state FP64.  MGRIT never converges to anything
 * but the fine solution whatever the coarse propagator (Alg. 2): the network
 * only changes how many cycles are needed. */
#define PIT_NET_PARAMS 3094

typedef struct {
    double dt_fine;        /* fine step of the pairs                            */
    int m;                 /* pairs are (u, Phi^m u): coarse step dT = m dt_fine */
    int n_pairs;           /* training pairs (one pair = one grid's state)     */
    int n_holdout;         /* held-out pairs judged against the implicit Phi_c  */
    int epochs;
    int batch;             /* pairs per Adam step                              */
    double lr;             /* Adam learning rate (beta1 0.9, beta2 0.999, eps 1e-8) */
    unsigned long long seed;
    int ic_modes;          /* random initial values: sums of ic_modes product-sine */
    int ic_fmax;           /* modes, N(0,1) amplitudes, frequencies 1..ic_fmax     */
    int traj_len;          /* pairs taken along each fine trajectory           */
    pit_solve_opts fine;   /* solver of the fine steps that make the targets   */
    pit_solve_opts crs;    /* solver of the implicit Phi_c used as the judge   */
    double accept_ratio;   /* the network is accepted when its held-out error is
                              at most accept_ratio x that of the implicit step
                              (0 < accept_ratio <= 1; 1: not larger)          */
} pit_train_opts;

typedef struct {
    double loss_first_epoch;     /* mean relative squared loss, first epoch */
    double loss_last_epoch;      /* same, last epoch                         */
    double holdout_err_learned;  /* mean ||Phi_hat u - Phi^m u|| / ||Phi^m u|| on held-out pairs */
    double holdout_err_implicit; /* same for the implicit coarse step        */
    int accepted;                /* 1 when the learned error is at most
                                    accept_ratio x the implicit one        */
    int adam_steps;
    double ms_data;              /* generating the pairs                    */
    double ms_train;             /* forward/backward/Adam                   */
} pit_train_stats;

/* Sets (host, n == PIT_NET_PARAMS floats; rounded to BF16 here) or reads the
 * network parameters of the problem.  Setting marks the network accepted. */
pit_status pit_net_set_params(pit_problem_t p, const float *w, int n);
pit_status pit_net_get_params(pit_problem_t p, float *w, int n);

/* out = Phi_hat(u) for n_batch packed states with coarse step dT.
 * u, out: device, n_batch * n_total doubles, must not overlap. */
pit_status pit_net_forward(pit_problem_t p, double dT, int n_batch, const double *u, double *out);

/* Training loss sum over all (state, grid) items of ||Phi_hat(u) - y||^2 /
 * ||y||^2 and its gradient with respect to the parameters (as used: BF16-
 * rounded).  u, y: device, n_batch * n_total doubles; loss: host double;
 * grad: host, PIT_NET_PARAMS floats. */
pit_status pit_net_loss_grad(pit_problem_t p, double dT, int n_batch, const double *u, const double *y,
                             double *loss, float *grad);

/* Trains the network on the GPU: pairs (u, Phi^m u) from fine trajectories
 * of seeded random initial values (training and held-out), Adam on FP32
 * master weights with BF16 forward/backward weights, then judges it against
 * the implicit coarse step on the held-out pairs.  The trained parameters are
 * kept; MGRIT with PIT_COARSE_LEARNED uses them only when accepted. */
pit_status pit_train_coarse(pit_problem_t p, const pit_train_opts *opts, pit_train_stats *stats);

/* Creates a problem on the current CUDA device: enumerates the component
 * grids (Eq. "combination_technique_solution"; l >= level0 componentwise,
 * |l|_1 = level_n + d - 1 - w, w = 0..d-1), uploads the grid table, makes the
 * launch plan of every precision form the operator and grid sizes support,
 * and allocates the solvers' workspaces lazily.  stream is a cudaStream_t (NULL = legacy
 * default stream).  Errors: PIT_ERR_INVALID_ARG (d outside 1..6, level0 < 1,
 * level_n < level0, hi <= lo, unknown op), PIT_ERR_CUDA (no device). */
pit_status pit_problem_create(const pit_problem_desc *desc, void *stream, pit_problem_t *out);

/* Releases every device buffer, graph and stream object of the problem. */
pit_status pit_problem_destroy(pit_problem_t p);

/* Grid table (host pointers, each optional): number of grids G, n_total,
 * levels (G*d ints), combination coefficients (-1)^w C(d-1, w) (G doubles),
 * offsets (G+1 long longs). */
pit_status pit_problem_info(pit_problem_t p, int *n_grids, long long *n_total, int *levels,
                            double *coef, long long *offsets);

/* Samples an initial value at every interior node of every grid.
 * kind 0: sum of K product-sine modes, params = [K, (A_k, m_k1..m_kd) for k < K]:
 *         u0(x) = sum_k A_k prod_i sin(pi m_ki (x_i - lo_i) / (hi_i - lo_i))
 * kind 1: product Gaussian, params = [mean_1..mean_d, std_1..std_d].
 * kind 2: the manufactured solution of the heat experiment (Sec. 4.2, Eq.
 *         "heat_equation"), params = [t]: u*(x, t) = sqrt(|x|^2 + t^2) e^{-t}
 *         prod_i sin(pi (x_i - lo_i) / (hi_i - lo_i)).
 * kind 3: its forcing for the heat operator, params = [t]:
 *         f(x, t) = du*(x, t)/dt - Laplace u*(x, t).
 * kind 4: normal density with mean M and covariance C (the law of the linear
 *         SDE, Eq. "sde_analytical_solution"), params = [M (d), C (d x d, row
 *         major, symmetric positive definite)].
 * params: host, n_params doubles.  u0: host or device, n_total doubles. */
pit_status pit_sample_initial(pit_problem_t p, int kind, const double *params, int n_params, double *u0);

/* Stencil application q = (I + dt L) p for a batch (the matrix of
 * Eq. "parabolic_problem_time_propagation_LES" times dt).  p, q: device,
 * n_batch * n_total doubles, must not overlap. */
pit_status pit_apply(pit_problem_t p, double dt, int n_batch, const double *pv, double *qv);

/* Batched backward-Euler step Phi (Sec. 2, Eq. "parabolic_problem_time_propagation"):
 * for every batch entry b and grid g solve (I + dt L) x = u_prev + dt f with
 * initial guess u_prev, write x to u_next.  f may be NULL (f = 0).
 * u_prev, f, u_next: device, n_batch * n_total doubles; u_next may alias
 * u_prev exactly (in-place step), no other overlap.  stats may be NULL; when
 * given, the call synchronises and fills it, and returns PIT_ERR_NOCONV,
 * PIT_ERR_BREAKDOWN or PIT_ERR_NONFINITE if any item failed. */
pit_status pit_phi_batch(pit_problem_t p, double dt, int n_batch, const double *u_prev,
                         const double *f, double *u_next, const pit_solve_opts *opts,
                         pit_phi_stats *stats);

/* Time-sequential stepping (Alg. 1 with s = 1): nsteps backward-Euler steps
 * of size dt from u0 on every grid.  u0, uT: host or device, n_total doubles,
 * may alias.  Synchronises; stats may be NULL. */
pit_status pit_sequential_solve(pit_problem_t p, const double *u0, double dt, int nsteps,
                                const pit_solve_opts *opts, double *uT, pit_phi_stats *stats);

/* Time-sequential stepping with forcing and per-grid time partitions (Alg. 1
 * with s = 1; Sec. 2.2.1): grid g takes nsteps x tmul[g] steps of
 * dt / tmul[g]; the steps inside fine step n use f_n.  forcing: device,
 * nsteps packed states (f_n, n = 1..nsteps) or NULL; tmul: host, G ints in
 * 1..4096 or NULL (all 1).  Otherwise as pit_sequential_solve. */
pit_status pit_sequential_solve_forced(pit_problem_t p, const double *u0, double dt, int nsteps,
                                       const double *forcing, const int *tmul, const pit_solve_opts *opts,
                                       double *uT, pit_phi_stats *stats);

/* CTMGRIT^loc with s = 1 (Alg. 3): independent MGRIT (Alg. 2, FCF, FAS) on
 * every grid from u0 over [t0, t1] with nsteps fine steps, returning the
 * final state of every grid.  The initial guess at every time point is u0.
 * u0, uT: host or device, n_total doubles.  Synchronises once per cycle to
 * read the residual norms.  Returns PIT_ERR_NOCONV if a grid did not meet
 * tol within maxit cycles (uT then holds the last iterate). */
pit_status pit_mgrit_solve(pit_problem_t p, const double *u0, const pit_mgrit_opts *opts,
                           double *uT, pit_mgrit_stats *stats);

/* Combination sum (Eq. "combination_technique_solution"):
 * out[k] = sum_g coef_g * I_g[u_g](pts[k]), I_g the piecewise d-linear
 * interpolant on grid g with zero boundary values (Sec. 2.2.2).
 * u: host or device, n_total doubles; pts: host or device, n_pts * d doubles
 * (row-major); out: host or device, n_pts doubles.  Points outside the box
 * are clamped to its boundary cell. */
pit_status pit_combine(pit_problem_t p, const double *u, int n_pts, const double *pts, double *out);

/* Recombination (Sec. 2.2.2, Eq. "overall_combination_operator"):
 * out = Q u = H^{-1} Qbar H u.  Every grid's nodal values are hierarchized
 * (surplus of each node over the linear interpolant of its two hierarchical
 * parents, along every axis in turn), the surplus at every node becomes the
 * sum over all grids that have a node at the same coordinates of their
 * combination coefficient times their surplus there (Eq.
 * "recombination_operator"), and the grids are dehierarchized.  The result on
 * grid l is the nodal interpolant on Omega_l of the combined solution
 * sum_m c_m I_m[u_m].  u, out: device, n_total doubles; out may alias u
 * exactly.  The sparse grid's block plan is built, and its scratch (n_total
 * plus the number of sparse-grid nodes doubles) allocated, on the first call.
 * PIT_ERR_UNSUPPORTED when (largest level + 1)^d exceeds 2^24. */
pit_status pit_recombine(pit_problem_t p, const double *u, double *out);

/* Kernel timing of a problem: while enabled, every library call that launches
 * device work is bracketed by CUDA events recorded on the problem's stream
 * (one timed call may launch several kernels: a multi-step solve launches one
 * kernel per shared-memory bucket, concurrently on forked streams, and the
 * events span them all).  pit_profile_read synchronises the stream and
 * returns, since the last enable, per kernel family: timed calls, their summed
 * device milliseconds, the kernels launched, and for the backward-Euler
 * kernels the work done (Krylov iterations and refinement passes weighted by
 * grid nodes).  Family 0 = backward-Euler solver on batches of 8 or more
 * entries per grid (relaxation), 1 = backward-Euler solver on fewer
 * (sequential sweeps, time stepping), 2 = combination sum, 3 = other. */
typedef struct {
    long long launches[4];   /* timed calls                                       */
    double ms[4];            /* device time of the timed calls                    */
    long long phi_items;
    long long point_iters;   /* sum over items of nodes x Krylov iterations       */
    long long point_passes;  /* sum over items of nodes x refinement residual passes */
    long long point_steps;   /* sum over items of nodes x backward-Euler steps    */
    long long kernels[4];    /* kernel launches, including those of the
                                launch-shape tuner on a first call              */
    long long point_iters_f[2];   /* point_iters of family 0 and of family 1     */
    long long point_passes_f[2];  /* point_passes of family 0 and of family 1    */
    long long point_steps_f[2];   /* point_steps of family 0 and of family 1     */
    long long device_allocs;      /* device allocations (cudaMalloc) the library made
                                     since pit_profile_enable, counted over every
                                     problem of the process                       */
} pit_profile;

pit_status pit_profile_enable(pit_problem_t p, int on);
pit_status pit_profile_read(pit_problem_t p, pit_profile *out);

/* In-place backward-Euler step that allocates nothing.  The paper has no
 * counterpart; this is a service to callers that cannot allocate device
 * memory while they run: an application whose GPU memory is entirely reserved
 * by another allocator (a framework's caching pool that owns the device), or
 * a control loop that forbids any allocation after start-up.  It computes
 * what pit_phi_batch computes with u_next == u_prev: u <- Phi(u) (+ dt f in the
 * right-hand side) for n_batch packed states, but stages the result in one
 * static device array of PIT_STATIC_SCRATCH_DOUBLES doubles (8 MiB) that the
 * library holds on every GPU that loads it, until the process exits, instead
 * of a buffer it would allocate.
 *   - u, f: device, n_batch * n_total doubles (f may be NULL); the caller owns
 *     them.  Requires n_batch * n_total <= PIT_STATIC_SCRATCH_DOUBLES, else
 *     PIT_ERR_INVALID_ARG before any device work.
 *   - The problem's device must be current.  The first call on a device looks
 *     up the array's device address (cudaGetSymbolAddress) and caches it; make
 *     that first call before any stream capture.
 *   - All calls on a device share the one array, and every call overwrites it
 *     entirely before reading it.  Calls whose work overlaps on the GPU (on
 *     different streams, or from several threads) race on it: order them.
 *   - Calls no cudaMalloc, cudaFree or allocating library routine: the launch
 *     plan comes from pit_problem_create, so the first call on a new problem
 *     allocates nothing either (pit_profile_read's device_allocs counts the
 *     library's allocations).  With profiling enabled (pit_profile_enable) the
 *     timing events of the call may be created on first use.
 *   - One launch covers every grid, with the shared memory of the largest and
 *     the CTA size the autotuner chose for the first shared-memory bucket of
 *     this problem and batch width (else 128 threads).
 *   - PIT_ERR_UNSUPPORTED for problems with grids too large for the on-chip
 *     solve (their solver state needs global scratch), and for any precision
 *     form that pit_phi_batch rejects on this problem (such as the pair form
 *     on the drift operator).
 *   - stats as in pit_phi_batch (NULL skips the synchronisation); the step
 *     counts in pit_profile_read like a pit_phi_batch call. */
#define PIT_STATIC_SCRATCH_DOUBLES (1 << 20)
pit_status pit_phi_batch_inplace_static(pit_problem_t p, double dt, int n_batch, double *u, const double *f,
                                        const pit_solve_opts *opts, pit_phi_stats *stats);

/* Thread-local text of the last error. */
const char *pit_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PIT_H */
