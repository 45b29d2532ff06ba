// Internal declarations of libpit: device-side grid table, operator
// coefficients, launch arguments and the launchers shared by the API and the
// kernels.  Method: Griebel, Schweitzer, Troska, arXiv 2509.22156.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pit.h"

#define PIT_D PIT_MAX_DIM

namespace pit {

// One component grid Omega_l (Sec. 2.1.1): N_i = 2^{l_i} - 1 interior nodes per
// axis, C-order strides S_i with the last axis fastest, mesh width h_i.
struct GridInfo {
    long long off;      // packed offset of the grid in a state vector
    int n;              // interior nodes
    int pad;
    int N[PIT_D];
    int S[PIT_D];
    double h[PIT_D];
};

struct OpParams {
    int op;             // pit_op
    int d;
    double lo[PIT_D];
    double theta, sigma, vamp;
    double A[PIT_D * PIT_D];  // linear SDE: drift matrix (row major, d x d)
    double H[PIT_D * PIT_D];  // linear SDE: H = 2 sigma D sigma^T (row major, d x d)
    int central;              // linear SDE, CME: central drift flux (else donor cell)
    // CME toggle network: production cp / (cs + y^cb), y the other species'
    // total, degradation cg x_i (per species)
    double cp[PIT_D], cs[PIT_D], cb[PIT_D], cg[PIT_D];
};

// Drift part of one axis of the flux-form operator (F_+ - F_-) / h at node j,
// face velocities vp at x + h/2 e_i and vm at x - h/2 e_i: coefficients of
// p_j, p_{j-e_i}, p_{j+e_i}.  Donor cell: F_+ = max(vp,0) p_j + min(vp,0)
// p_{j+e_i}; central: F_+ = vp (p_j + p_{j+e_i}) / 2.
__host__ __device__ __forceinline__ void drift_coef(double vp, double vm, double h, bool central, double &dd,
                                                    double &dm, double &dp)
{
    if (central) {
        dd = 0.5 * (vp - vm) / h;
        dm = -0.5 * vm / h;
        dp = 0.5 * vp / h;
    } else {
        dd = (fmax(vp, 0.0) - fmin(vm, 0.0)) / h;
        dm = -fmax(vm, 0.0) / h;
        dp = fmin(vp, 0.0) / h;
    }
}

// Production propensity of species i of the CME toggle network at x.
template <typename X>
__host__ __device__ __forceinline__ double cme_production(const OpParams &op, int i, const X &x, int d)
{
    double y = 0.0;
    for (int k = 0; k < d; ++k)
        if (k != i) y += x[k];
    return op.cp[i] / (op.cs[i] + pow(y, op.cb[i]));
}

// Coefficients of axis i of the CME operator at a node with coordinate xi on
// that axis and production a (which does not depend on x_i): drift flux with
// face velocities a - g (xi +- h/2), diffusion -(D_+ p_+ - 2 D_0 p_j + D_- p_-)
// / (2 h^2) with D = a + g x.
__host__ __device__ __forceinline__ void cme_coef(double a, double g, double xi, double h, bool central,
                                                  double &dd, double &dm, double &dp)
{
    drift_coef(a - g * (xi + 0.5 * h), a - g * (xi - 0.5 * h), h, central, dd, dm, dp);
    const double ih2 = 0.5 / (h * h);
    dd += 2.0 * (a + g * xi) * ih2;
    dm -= (a + g * (xi - h)) * ih2;
    dp -= (a + g * (xi + h)) * ih2;
}

// Global counters filled by the backward-Euler kernels (one atomic per item).
struct DevStats {
    unsigned long long sum_iters;
    unsigned long long items;
    unsigned long long point_iters;   // sum of nodes x Krylov iterations
    unsigned long long point_passes;  // sum of nodes x refinement residual passes
    unsigned long long point_steps;   // sum of nodes x backward-Euler steps
    int max_iters;
    int n_failed;
    int max_refine;
    int worst;          // largest pit_status code seen
};

// Arguments of one multi-step backward-Euler launch.  Item k = item0 +
// blockIdx.x is grid order[k / n_batch] of batch entry b = k % n_batch.  Entry b starts
// from in + b*in_stride (+ grid offset) and takes nsteps steps of size dt;
// the forcing of step s (1-based) is f + b*f_stride + ((s-1)/f_div)*f_step
// (f may be NULL: no forcing);
// after step s (1-based) x <- x + g_s with g_s = g + b*g_stride + (s-1)*g_step
// (g may be NULL); states after steps 1..nsteps-1 are written to out_steps +
// b*os_stride + (s-1)*os_step when out_steps is non-NULL; the final state x is
// written as out_scale * x + out_hscale * h_b to out_last + b*ol_stride; when
// hs is non-NULL every stored state (steps and last) also gets hs_s =
// hs + b*hs_stride + (s-1)*hs_step added; when cmp is
// non-NULL, norms[b*n_grids + g] = ||x - cmp_b||_2.  When guess is non-NULL
// the Krylov solve of step s starts from guess_s - g_s instead of x_{s-1}
// (guess_s = guess + b*guess_stride + (s-1)*guess_step); the right-hand side is
// unchanged, so only the iteration count depends on it.  No output may overlap
// the input of the same item.
struct StepArgs {
    int item0;              // first item of this launch (launches may be split in chunks)
    const GridInfo *grids;
    const uint16_t *masks;  // neighbour mask of every node, packed like a state
    const int *order;       // the launch's grids, by decreasing size
    int n_order;            // grids in order
    int n_grids;            // all grids of the problem (row length of norms)
    int n_batch;
    int nsteps;
    double dt;
    const double *in;        long long in_stride;
    const double *f;         long long f_stride, f_step;
    int f_div;
    const double *g;         long long g_stride, g_step;
    double *out_steps;       long long os_stride, os_step;
    double *out_last;        long long ol_stride;
    double out_scale;
    double out_hscale;
    const double *h;         long long h_stride;
    const double *hs;        long long hs_stride, hs_step;
    const double *cmp;       long long cmp_stride;
    double *norms;
    const double *guess;     long long guess_stride, guess_step;
    double *xg;              // state in global memory (grids too large for shared memory):
    double *bg;              //   x and b (MIXED) of entry b at xg/bg + b*n_total + grid offset, the
                             //   carried x - A x (MIXED, FP64) at slab 2;
                             //   PLAIN: Krylov vector k at xg + ((1+k) n_batch + b) n_total + offset,
                             //   then (table operators) coefficient row k of the item at
                             //   xg + ((1+NKV+k) n_batch + b) n_total + offset
    long long n_total;
    const int *active;       // per grid, NULL = all active
    const double *faces;     // variable coefficient at the 2d faces of every node, or NULL
    OpParams op;
    double rtol;
    int maxit;
    float inner_rtol;
    int ir_maxit;
    int inexact;             // 1: a solve stopped by its iteration caps is not a failure
    int precond;             // pit_precond of the Krylov solves
    int predict;             // MIXED without forcing: extrapolated initial guess 2 x_s - x_{s-1}
    int sdirk;               // MIXED or SINGLE: every step is a two-stage SDIRK step, dt its stage step
    int ext;                 // heat, MIXED or SINGLE: every step is an extrapolated backward-Euler step, dt its half step
    float *scr;              // SINGLE extrapolated steps: n_batch x n_total FP32 scratch (u_n, then U2)
    DevStats *stats;
};

// Precision forms of the multi-step kernel: PLAIN = FP64 Krylov, MIXED = FP32
// Krylov in FP64 refinement, SINGLE = FP32 Krylov on a power-of-two-scaled
// FP32 copy of the state (FP64 input and output), PAIR = FP32 Krylov in a
// refinement whose state and residual are FP32 pairs (symmetric operators).
enum Prec { PLAIN = 0, MIXED = 1, SINGLE = 2, PAIR = 3 };
constexpr int NPREC = 4;
// Launch parts of one multi-step call: NBKT shared-memory buckets of the
// grids whose state fits on chip, then the grids with global-memory state.
constexpr int NBKT = 4;
constexpr int NPART = NBKT + 1;
inline int prec_form(int pit_prec)
{
    return pit_prec == PIT_PREC_MIXED        ? MIXED
           : pit_prec == PIT_PREC_FP32       ? SINGLE
           : pit_prec == PIT_PREC_MIXED_PAIR ? PAIR
                                             : PLAIN;
}

// Learned coarse propagator: parameter block (BF16-rounded values held as
// FP32) passed by value to the inference kernel, and one training item.
struct NetWeights {
    float w[PIT_NET_PARAMS];
};
struct NetTrainItem {
    int g;          // grid
    int pad;
    long long off;  // offset of the grid's values in the packed u and y arrays
};

size_t net_smem_bytes(int n);
size_t net_act_floats(int n, bool train);
cudaError_t net_kernels_init(size_t max_smem);
// Launches items a.item0 .. a.item0 + n_items - 1.
cudaError_t launch_net_steps(const StepArgs &a, const NetWeights &W, float *act, long long act_stride, size_t smem,
                             cudaStream_t s, int n_items);
cudaError_t launch_net_train(const GridInfo *grids, const NetTrainItem *items, int n_items, const double *u,
                             const double *y, double dT, const float *w, float *act, long long act_stride,
                             float *grad_rows, double *loss_items, OpParams op, cudaStream_t s);
// Sums n_rows gradient rows (item order) into grad_out (if non-NULL) and, when
// master is non-NULL, takes one Adam step on the master weights (gradient
// scaled by `scale`) and writes their BF16 rounding to w_bf16.
cudaError_t launch_net_adam(const float *grad_rows, int n_rows, float scale, float *master, float *m, float *v,
                            float *w_bf16, float lr, float b1, float b2, float eps, int t, float *grad_out,
                            cudaStream_t s);

// Shared-memory bytes a backward-Euler item of n nodes needs.
// (na: nodes of the grid's longest axis, for the heat line preconditioner)
size_t phi_smem_bytes(int prec, int op, int d, int n, int na);
// Launch one multi-step batch (grid-per-CTA, every Krylov solve on chip);
// xg selects the variant whose FP64 state lives in global memory.
cudaError_t launch_steps(int prec, const StepArgs &a, int threads, size_t smem, cudaStream_t s, bool xg = false);
// Shared memory per item of the global-state variant (PLAIN or MIXED), and
// the number of n_batch x n_total FP64 slabs of global workspace it uses
// (x, b and the carried x - A x for MIXED; x and the Krylov vectors for
// PLAIN).
size_t phi_smem_bytes_xg(int prec, int op, int d, int n);
int xg_slabs(int prec, int op, int d);
// Raise the dynamic shared-memory limit of every backward-Euler kernel.
cudaError_t phi_kernels_init(size_t max_smem);
// Neighbour masks of every node (bit 2i: interior neighbour at -e_i, 2i+1: at +e_i).
cudaError_t launch_masks(const GridInfo *grids, int G, int d, uint16_t *masks, cudaStream_t s);

cudaError_t launch_apply(const GridInfo *grids, int G, long long ntot, int n_batch, double dt,
                         const double *p, double *q, const double *faces, OpParams op, cudaStream_t s);
// Space-time residual rho_b = x_b + dt f_b - (I + dt L) u_b at nb C-points
// (strides xs, fs, us, os in doubles; f may be NULL), written as scale * rho_b;
// ||rho_b||_2 per grid in norms[b * G + g]; active grids only.
cudaError_t launch_st_resid(const GridInfo *grids, int G, long long ntot, int nb, double dt, const double *x,
                            long long xs, const double *f, long long fs, const double *u, long long us, double scale,
                            double *out, long long os, double *norms, const int *active, const double *faces,
                            OpParams op, cudaStream_t s);
cudaError_t launch_initial(const GridInfo *grids, int G, OpParams op, const double *hi, int kind,
                           const double *params_dev, int n_params, double *u, cudaStream_t s);
cudaError_t launch_faces(const GridInfo *grids, int G, OpParams op, double *faces, cudaStream_t s);
// Number of grid chunks the combination sum splits into (one kernel per
// chunk set, partial sums in part[chunk * n_pts + k], n_chunks x n_pts doubles,
// then added in chunk order); 1 means a single kernel writing out directly.
int combine_chunks(int G, int n_pts, int n_sm);
cudaError_t launch_combine(const GridInfo *grids, const double *coef, const int *levels, int G, OpParams op,
                           const double *u, int n_pts, const double *pts, double *out, int n_chunks, double *part,
                           cudaStream_t s);
// resid[j*G + g] = || a_j - b_j ||_2 on grid g, for active grids; j < nb.
cudaError_t launch_resid_norms(const GridInfo *grids, int G, long long ntot, int nb, const double *a,
                               long long a_stride, const double *b, long long b_stride, const int *active,
                               double *resid, cudaStream_t s);
// rmax[g] = max_j resid[j*G + g] (NaN propagates), active grids only.
// out_k = x_k + y_k on the active grids of nb consecutive states.
cudaError_t launch_add_states(const GridInfo *grids, int G, long long ntot, int nb, const double *x, const double *y,
                              double *out, const int *active, cudaStream_t s);
cudaError_t launch_resid_max(int G, int nb, const double *resid, const int *active, double *rmax,
                             cudaStream_t s);

// Recombination (Sec. 2.2.2): the sparse grid's hierarchical increments lam
// (level multi-indices contained in some grid), block b holding the
// 2^{|lam|_1 - d} surpluses of increment blk_lam[b*d .. b*d+d-1] at
// [blk_off[b], blk_off[b+1]) in C order; list[list_off[b] .. list_off[b+1])
// are the grids that contain lam, ascending; lookup[code(lam)] = b (-1: none),
// code(lam) = ((lam_0 radix + lam_1) radix + ...) + lam_{d-1}.  Device pointers.
struct RecombPlan {
    int n_blk;
    int radix;
    long long n_sparse;
    const int *blk_lam;
    const long long *blk_off;
    const int *list_off;
    const int *list;
    const int *lookup;
};
// out_b = Q u_b on every grid for nb consecutive states b (stride ntot; out
// may alias u); H: nb x n_total, S: nb x n_sparse doubles of scratch.
cudaError_t launch_recombine(const RecombPlan &R, int d, const GridInfo *grids, const double *coef, int G,
                             long long ntot, int nb, const double *u, double *H, double *S, double *out,
                             cudaStream_t s);

}  // namespace pit
