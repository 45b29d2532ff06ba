// Batched multi-step backward-Euler propagator (Sec. 2, Eq. "parabolic_problem_
// time_propagation"): every (batch entry, component grid) item is advanced by
// nsteps backward-Euler steps
//     (I + dt L_l) x_s = x_{s-1} + dt f,   x_s <- x_s + g_s (optional forcing),
// each solved matrix-free with CG (symmetric operators) or BiCGStab (drift
// operator, Sec. 4.1), initial guess x_{s-1}.
//
// Design (grid-resident, multi-step): one CTA owns one item for all its
// steps.  The FP64 state, the Krylov vectors and the neighbour masks live in
// shared memory; dot products are reduced with warp shuffles and one block
// barrier.  A whole F-relaxation interval (m - 1 steps) or a sequential
// coarse sweep is one launch, HBM is touched once to read the start state
// and once per stored output state, and the intermediate F-values never
// leave the SM (the C-point-only storage of Sec. 3.3.2).
//
// Precision forms:
//   PLAIN  Krylov in FP64 until ||b - A x|| <= rtol ||b||.
//   MIXED  FP64 iterative refinement around an FP32 Krylov solve: residual
//          b - A x formed in FP64 from the FP64 state, the correction
//          equation solved in FP32 to inner_rtol, correction added in FP64;
//          same FP64 stopping rule.
// CG is the single-reduction (Chronopoulos-Gear) form: one fused block
// reduction of (r,r) and (Ar,r) per iteration and two barriers.
#include <type_traits>

#include "pit_internal.cuh"

namespace pit {

#define FULL_MASK 0xffffffffu

// ----------------------------------------------------------------------------
// Operator coefficients of node j in FP64: (A p)_j = diag p_j + sum_i cm_i
// p_{j-e_i} + cp_i p_{j+e_i}, zero towards boundary nodes (zero Dirichlet):
//   heat    L p = sum_i (2 p_j - p_- - p_+) / h_i^2
//   varheat L p = sum_i [a_+ (p_j - p_+) + a_- (p_j - p_-)] / h_i^2
//   OU      L p = sum_i (F_+ - F_-) / h_i + (sigma^2/2)(2 p_j - p_- - p_+) / h_i^2,
//           F_+ = max(v_+,0) p_j + min(v_+,0) p_+,  v_+ = -theta (x_i + h_i/2).
__device__ __forceinline__ void op_coef(const OpParams &op, const GridInfo &G, const double *faces, int j,
                                        double dt, double &diag, double *cm, double *cp)
{
    const int d = op.d;
    diag = 1.0;
#pragma unroll
    for (int i = 0; i < PIT_D; ++i) {
        if (i >= d) break;
        const int c = (j / G.S[i]) % G.N[i];
        const double h = G.h[i];
        const double ih2 = 1.0 / (h * h);
        double dd, dm, dp;
        if (op.op == PIT_OP_HEAT) {
            dd = 2.0 * ih2; dm = -ih2; dp = -ih2;
        } else if (op.op == PIT_OP_VARHEAT) {
            const double am = faces[(G.off + j) * (2 * d) + 2 * i];
            const double ap = faces[(G.off + j) * (2 * d) + 2 * i + 1];
            dd = (am + ap) * ih2; dm = -am * ih2; dp = -ap * ih2;
        } else {
            const double x = op.lo[i] + (double)(c + 1) * h;
            const double vp = -op.theta * (x + 0.5 * h);
            const double vm = -op.theta * (x - 0.5 * h);
            const double s2 = 0.5 * op.sigma * op.sigma * ih2;
            dd = (fmax(vp, 0.0) - fmin(vm, 0.0)) / h + 2.0 * s2;
            dm = -fmax(vm, 0.0) / h - s2;
            dp = fmin(vp, 0.0) / h - s2;
        }
        diag += dt * dd;
        cm[i] = (c > 0) ? dt * dm : 0.0;
        cp[i] = (c < G.N[i] - 1) ? dt * dp : 0.0;
    }
}

// Constant-coefficient heat stencil with a per-node neighbour mask
// (bit 2i: interior neighbour at -e_i, bit 2i+1: at +e_i).
template <typename T>
struct HeatSt {
    const uint16_t *mask;
    int d;
    int S[PIT_D];
    T diag;
    T off[PIT_D];
    __device__ __forceinline__ T operator()(const T *p, int j) const
    {
        const unsigned mk = mask[j];
        T s = diag * p[j];
#pragma unroll
        for (int i = 0; i < PIT_D; ++i) {
            if (i >= d) break;
            const T pm = ((mk >> (2 * i)) & 1u) ? p[j - S[i]] : T(0);
            const T pp = ((mk >> (2 * i + 1)) & 1u) ? p[j + S[i]] : T(0);
            s += off[i] * (pm + pp);
        }
        return s;
    }
};

// Variable-coefficient stencil from a per-node table in shared memory
// (structure of arrays: tab[k*ld + j], k = 0 diagonal, 1+2i minus, 2+2i plus;
// zero coefficients towards the boundary).
template <typename T>
struct TabSt {
    const uint16_t *mask;
    const T *tab;
    int ld;
    int d;
    int S[PIT_D];
    __device__ __forceinline__ T operator()(const T *p, int j) const
    {
        const unsigned mk = mask[j];
        T s = tab[j] * p[j];
#pragma unroll
        for (int i = 0; i < PIT_D; ++i) {
            if (i >= d) break;
            const int jm = ((mk >> (2 * i)) & 1u) ? j - S[i] : j;
            const int jp = ((mk >> (2 * i + 1)) & 1u) ? j + S[i] : j;
            s += tab[(1 + 2 * i) * ld + j] * p[jm] + tab[(2 + 2 * i) * ld + j] * p[jp];
        }
        return s;
    }
};

// ----------------------------------------------------------------------------
// Block reductions: warp shuffles, one partial per warp in a 32-slot buffer,
// one barrier, then every warp reduces the partials with the same shuffle
// tree and broadcasts lane 0: all threads hold the bitwise same value,
// independent of scheduling.  Consecutive reductions alternate two buffers,
// so one barrier per reduction suffices (a warp can only reuse a buffer after
// every warp passed the barrier of the reduction in between).
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL_MASK, v, o);
    return v;
}

template <typename T>
struct Reducer {
    T *buf;    // two halves of 4 x 32 slots
    int slot;
    template <int K>
    __device__ __forceinline__ void sum(T *v)
    {
        T *red = buf + (slot & 1) * 128;
        ++slot;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const T x = warp_sum(v[k]);
            if (lane == 0) red[k * 32 + w] = x;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < K; ++k) {
            T x = (lane < nw) ? red[k * 32 + lane] : T(0);
            x = warp_sum(x);
            v[k] = __shfl_sync(FULL_MASK, x, 0);
        }
    }
};

__device__ __forceinline__ bool finite_pos(double v) { return v > 0.0 && v < 1.0e300; }
__device__ __forceinline__ bool finite_pos(float v) { return v > 0.0f && v < 1.0e37f; }

// ----------------------------------------------------------------------------
// Single-reduction CG (Chronopoulos & Gear 1989) on A e = r0: r holds r0 on
// entry (own nodes written by the caller), the iterate is accumulated into X
// (FP64 state or FP32 correction).  Stops when (r,r) <= stop2.
template <typename T, typename TX, class ST>
__device__ int cg_core(const ST &A, int n, TX *X, T *r, T *p, T *s, T *w, Reducer<T> &R, T stop2, int maxit,
                       int &status)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    status = PIT_OK;
    __syncthreads();  // r complete
    T v[2] = {T(0), T(0)};
    for (int j = tid; j < n; j += nt) {
        const T wj = A(r, j);
        w[j] = wj;
        const T rj = r[j];
        v[0] += rj * rj;
        v[1] += wj * rj;
    }
    R.template sum<2>(v);
    T gam = v[0];
    if (!(gam > stop2)) {
        if (gam != gam) status = PIT_ERR_NONFINITE;
        return 0;
    }
    if (!finite_pos(v[1])) {
        status = (v[1] != v[1]) ? PIT_ERR_NONFINITE : PIT_ERR_BREAKDOWN;
        return 0;
    }
    T alpha = gam / v[1], beta = T(0);
    bool first = true;
    int k = 0;
    for (;;) {
        if (k >= maxit) { status = PIT_ERR_NOCONV; break; }
        for (int j = tid; j < n; j += nt) {
            const T pj = first ? r[j] : r[j] + beta * p[j];
            const T sj = first ? w[j] : w[j] + beta * s[j];
            p[j] = pj;
            s[j] = sj;
            X[j] += (TX)(alpha * pj);
            r[j] -= alpha * sj;
        }
        first = false;
        ++k;
        __syncthreads();
        T u[2] = {T(0), T(0)};
        for (int j = tid; j < n; j += nt) {
            const T wj = A(r, j);
            w[j] = wj;
            const T rj = r[j];
            u[0] += rj * rj;
            u[1] += wj * rj;
        }
        R.template sum<2>(u);
        if (!(u[0] > stop2)) {
            if (u[0] != u[0]) status = PIT_ERR_NONFINITE;
            break;
        }
        beta = u[0] / gam;
        const T den = u[1] - beta * u[0] / alpha;
        if (!finite_pos(den)) { status = (den != den) ? PIT_ERR_NONFINITE : PIT_ERR_BREAKDOWN; break; }
        alpha = u[0] / den;
        gam = u[0];
    }
    return k;
}

// BiCGStab (van der Vorst 1992) on A e = r0: r holds r0 on entry; rh, p, v
// are initialised here; s shares r's storage.
template <typename T, typename TX, class ST>
__device__ int bicgstab_core(const ST &A, int n, TX *X, T *r, T *rh, T *p, T *v, T *t, Reducer<T> &R, T stop2,
                             int maxit, int &status)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    T rr[1] = {T(0)};
    for (int j = tid; j < n; j += nt) {
        const T rj = r[j];
        rh[j] = rj;
        p[j] = T(0);
        v[j] = T(0);
        rr[0] += rj * rj;
    }
    R.template sum<1>(rr);
    T rho = T(1), alpha = T(1), omega = T(1), rrv = rr[0];
    int k = 0;
    status = PIT_OK;
    for (;;) {
        if (!(rrv > stop2)) {
            if (rrv != rrv) status = PIT_ERR_NONFINITE;
            break;
        }
        if (k >= maxit) { status = PIT_ERR_NOCONV; break; }
        T rho_n[1] = {T(0)};
        for (int j = tid; j < n; j += nt) rho_n[0] += rh[j] * r[j];
        R.template sum<1>(rho_n);
        if (rho_n[0] == T(0) || omega == T(0) || rho_n[0] != rho_n[0]) {
            status = (rho_n[0] != rho_n[0]) ? PIT_ERR_NONFINITE : PIT_ERR_BREAKDOWN;
            break;
        }
        const T beta = (rho_n[0] / rho) * (alpha / omega);
        for (int j = tid; j < n; j += nt) p[j] = r[j] + beta * (p[j] - omega * v[j]);
        __syncthreads();
        T rhv[1] = {T(0)};
        for (int j = tid; j < n; j += nt) {
            const T vj = A(p, j);
            v[j] = vj;
            rhv[0] += rh[j] * vj;
        }
        R.template sum<1>(rhv);
        if (rhv[0] == T(0) || rhv[0] != rhv[0]) {
            status = (rhv[0] != rhv[0]) ? PIT_ERR_NONFINITE : PIT_ERR_BREAKDOWN;
            break;
        }
        alpha = rho_n[0] / rhv[0];
        for (int j = tid; j < n; j += nt) r[j] = r[j] - alpha * v[j];  // s
        __syncthreads();
        T tt[2] = {T(0), T(0)};
        for (int j = tid; j < n; j += nt) {
            const T tj = A(r, j);
            t[j] = tj;
            tt[0] += tj * tj;
            tt[1] += tj * r[j];
        }
        R.template sum<2>(tt);
        omega = (tt[0] > T(0)) ? tt[1] / tt[0] : T(0);
        T rn[1] = {T(0)};
        for (int j = tid; j < n; j += nt) {
            X[j] += (TX)(alpha * p[j] + omega * r[j]);
            const T rj = r[j] - omega * t[j];
            r[j] = rj;
            rn[0] += rj * rj;
        }
        R.template sum<1>(rn);
        rho = rho_n[0];
        rrv = rn[0];
        ++k;
        if (omega == T(0) && rrv > stop2) { status = PIT_ERR_BREAKDOWN; break; }
    }
    return k;
}

// ----------------------------------------------------------------------------
// Shared-memory layout of one item (ld = n rounded up to 4):
//   FP64 arrays: x, [b (MIXED)], [Krylov vectors (PLAIN)], [table (var. coef.)]
//   FP32 arrays: [Krylov vectors + table (MIXED)]
//   u16 mask
__host__ __device__ inline int krylov_vecs(int op, int prec)
{
    if (op == PIT_OP_OU) return prec == PLAIN ? 5 : 6;  // r rh p v t (+ e)
    return prec == PLAIN ? 4 : 5;                        // r p s w (+ e)
}
__host__ __device__ inline int n_tab(int op, int d) { return op == PIT_OP_HEAT ? 0 : 2 * d + 1; }
__host__ __device__ inline int n_f64(int op, int prec, int d)
{
    return (prec == PLAIN ? 1 + krylov_vecs(op, prec) : 2) + n_tab(op, d);
}
__host__ __device__ inline int n_f32(int op, int prec, int d)
{
    return prec == MIXED ? krylov_vecs(op, prec) + n_tab(op, d) : 0;
}

size_t phi_smem_bytes(int prec, int op, int d, int n)
{
    const size_t ld = (size_t)((n + 3) & ~3);
    return (size_t)n_f64(op, prec, d) * ld * 8 + (size_t)n_f32(op, prec, d) * ld * 4 + ld * 2 + 16;
}

template <int OP, int PREC>
__global__ void __launch_bounds__(512) steps_kernel(StepArgs a)
{
    typedef typename std::conditional<PREC == PLAIN, double, float>::type T;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ GridInfo GI;
    __shared__ double red64[2 * 128];
    __shared__ float red32[2 * 128];

    const int g = a.order[blockIdx.x / a.n_batch];
    const int b = blockIdx.x % a.n_batch;
    if (a.active && !a.active[g]) return;  // uniform over the block
    if (threadIdx.x == 0) GI = a.grids[g];
    __syncthreads();

    const int tid = threadIdx.x, nt = blockDim.x;
    const int n = GI.n, d = a.op.d;
    const int ld = (n + 3) & ~3;
    const double dt = a.dt;
    const int K = n_tab(OP, d);

    double *x = reinterpret_cast<double *>(smem);
    double *bvec = x + ld;  // MIXED only
    double *v64 = x + ld;   // PLAIN Krylov vectors
    double *tab64 = x + (size_t)(n_f64(OP, PREC, d) - K) * ld;
    float *f32 = reinterpret_cast<float *>(x + (size_t)n_f64(OP, PREC, d) * ld);
    float *tab32 = f32 + (size_t)krylov_vecs(OP, PREC) * ld;
    uint16_t *mask = reinterpret_cast<uint16_t *>(f32 + (size_t)n_f32(OP, PREC, d) * ld);

    const double *in = a.in + (long long)b * a.in_stride + GI.off;
    const double *f = a.f ? a.f + (long long)b * a.f_stride + GI.off : nullptr;
    const uint16_t *gmask = a.masks + GI.off;

    for (int j = tid; j < n; j += nt) {
        mask[j] = gmask[j];
        x[j] = in[j];
    }
    if constexpr (OP != PIT_OP_HEAT) {
        for (int j = tid; j < n; j += nt) {
            double diag, cm[PIT_D], cp[PIT_D];
            op_coef(a.op, GI, a.faces, j, dt, diag, cm, cp);
            tab64[j] = diag;
            if constexpr (PREC == MIXED) tab32[j] = (float)diag;
            for (int i = 0; i < d; ++i) {
                tab64[(1 + 2 * i) * ld + j] = cm[i];
                tab64[(2 + 2 * i) * ld + j] = cp[i];
                if constexpr (PREC == MIXED) {
                    tab32[(1 + 2 * i) * ld + j] = (float)cm[i];
                    tab32[(2 + 2 * i) * ld + j] = (float)cp[i];
                }
            }
        }
    }
    // stencils in FP64 and in the working precision
    HeatSt<double> H64;
    HeatSt<T> HT;
    TabSt<double> T64;
    TabSt<float> T32;
    H64.mask = HT.mask = T64.mask = T32.mask = mask;
    H64.d = HT.d = T64.d = T32.d = d;
    T64.tab = tab64;
    T32.tab = tab32;
    T64.ld = T32.ld = ld;
    {
        double diag = 1.0;
        for (int i = 0; i < PIT_D; ++i) {
            const double ih2 = (i < d) ? 1.0 / (GI.h[i] * GI.h[i]) : 0.0;
            const int S = (i < d) ? GI.S[i] : 0;
            H64.S[i] = HT.S[i] = T64.S[i] = T32.S[i] = S;
            H64.off[i] = -dt * ih2;
            HT.off[i] = (T)(-dt * ih2);
            diag += 2.0 * dt * ih2;
        }
        H64.diag = diag;
        HT.diag = (T)diag;
    }

    Reducer<double> R64{red64, 0};
    Reducer<float> R32{red32, 0};
    int status = PIT_OK, iters = 0, passes = 0;

    for (int step = 1; step <= a.nsteps; ++step) {
        __syncthreads();  // state complete
        if constexpr (PREC == PLAIN) {
            double *r = v64, *q1 = v64 + ld, *q2 = v64 + 2 * ld, *q3 = v64 + 3 * ld, *q4 = v64 + 4 * ld;
            double bb[1] = {0.0};
            for (int j = tid; j < n; j += nt) {
                const double bj = x[j] + (f ? dt * f[j] : 0.0);
                double Ax;
                if constexpr (OP == PIT_OP_HEAT) Ax = H64(x, j);
                else Ax = T64(x, j);
                r[j] = bj - Ax;
                bb[0] += bj * bj;
            }
            R64.template sum<1>(bb);  // also orders the residual before x changes
            const double stop2 = a.rtol * a.rtol * bb[0];
            int st, k;
            if constexpr (OP == PIT_OP_OU) k = bicgstab_core<double, double>(T64, n, x, r, q1, q2, q3, q4, R64, stop2, a.maxit, st);
            else if constexpr (OP == PIT_OP_HEAT) k = cg_core<double, double>(H64, n, x, r, q1, q2, q3, R64, stop2, a.maxit, st);
            else k = cg_core<double, double>(T64, n, x, r, q1, q2, q3, R64, stop2, a.maxit, st);
            iters += k;
            ++passes;
            if (st > status) status = st;
        } else {
            float *e = f32, *r = f32 + ld, *q1 = f32 + 2 * ld, *q2 = f32 + 3 * ld, *q3 = f32 + 4 * ld;
            float *q4 = f32 + 5 * ld;
            double bb[1] = {0.0};
            for (int j = tid; j < n; j += nt) {
                const double bj = x[j] + (f ? dt * f[j] : 0.0);
                bvec[j] = bj;
                bb[0] += bj * bj;
            }
            R64.template sum<1>(bb);
            const double stop2 = a.rtol * a.rtol * bb[0];
            int st_step = PIT_OK;
            for (int pass = 0;; ++pass) {
                __syncthreads();  // x complete
                double rn2[1] = {0.0};
                for (int j = tid; j < n; j += nt) {
                    double Ax;
                    if constexpr (OP == PIT_OP_HEAT) Ax = H64(x, j);
                    else Ax = T64(x, j);
                    const double rj = bvec[j] - Ax;
                    r[j] = (float)rj;
                    rn2[0] += rj * rj;
                }
                R64.template sum<1>(rn2);
                ++passes;
                if (!(rn2[0] > stop2)) {
                    if (rn2[0] != rn2[0]) st_step = PIT_ERR_NONFINITE;
                    break;
                }
                if (pass >= a.ir_maxit) { st_step = PIT_ERR_NOCONV; break; }
                const double rnorm = sqrt(rn2[0]);
                const float inv = (float)(1.0 / rnorm);
                for (int j = tid; j < n; j += nt) {
                    r[j] *= inv;
                    e[j] = 0.0f;
                }
                const float stop32 = a.inner_rtol * a.inner_rtol;
                int st, k;
                if constexpr (OP == PIT_OP_OU) k = bicgstab_core<float, float>(T32, n, e, r, q1, q2, q3, q4, R32, stop32, a.maxit, st);
                else if constexpr (OP == PIT_OP_HEAT) k = cg_core<float, float>(HT, n, e, r, q1, q2, q3, R32, stop32, a.maxit, st);
                else k = cg_core<float, float>(T32, n, e, r, q1, q2, q3, R32, stop32, a.maxit, st);
                iters += k;
                if (st == PIT_ERR_NONFINITE) { st_step = st; break; }
                // a stalled or broken-down inner solve still gives a usable
                // correction; the FP64 residual decides
                for (int j = tid; j < n; j += nt) x[j] += (double)e[j] * rnorm;
            }
            if (st_step > status) status = st_step;
        }
        // forcing of this step and the stored outputs (own nodes only)
        const long long sb = (long long)(step - 1);
        if (a.g) {
            const double *gs = a.g + (long long)b * a.g_stride + sb * a.g_step + GI.off;
            for (int j = tid; j < n; j += nt) x[j] += gs[j];
        }
        if (step < a.nsteps) {
            if (a.out_steps) {
                double *os = a.out_steps + (long long)b * a.os_stride + sb * a.os_step + GI.off;
                for (int j = tid; j < n; j += nt) os[j] = x[j];
            }
        } else {
            double *ol = a.out_last + (long long)b * a.ol_stride + GI.off;
            const double *h = a.h ? a.h + (long long)b * a.h_stride + GI.off : nullptr;
            const double *cmp = a.cmp ? a.cmp + (long long)b * a.cmp_stride + GI.off : nullptr;
            double acc[1] = {0.0};
            for (int j = tid; j < n; j += nt) {
                const double xj = x[j];
                if (cmp) {
                    const double dlt = xj - cmp[j];
                    acc[0] += dlt * dlt;
                }
                ol[j] = a.out_scale * xj + (h ? h[j] : 0.0);
            }
            if (cmp) {
                R64.template sum<1>(acc);
                if (tid == 0) a.norms[(long long)b * a.n_grids + g] = sqrt(acc[0]);
            }
        }
    }
    if (tid == 0 && a.stats) {
        atomicAdd(&a.stats->sum_iters, (unsigned long long)iters);
        atomicAdd(&a.stats->items, (unsigned long long)a.nsteps);
        atomicAdd(&a.stats->point_iters, (unsigned long long)iters * (unsigned long long)n);
        atomicAdd(&a.stats->point_passes, (unsigned long long)passes * (unsigned long long)n);
        atomicMax(&a.stats->max_iters, iters);
        atomicMax(&a.stats->max_refine, passes);
        if (status != PIT_OK) {
            atomicAdd(&a.stats->n_failed, 1);
            atomicMax(&a.stats->worst, status);
        }
    }
}

static size_t g_max_smem = 0;

cudaError_t phi_kernels_init(size_t max_smem)
{
    cudaError_t e = cudaSuccess;
    const int bytes = (int)max_smem;
#define PIT_SET(OPV, PV)                                                                                     \
    if (e == cudaSuccess)                                                                                    \
        e = cudaFuncSetAttribute(steps_kernel<OPV, PV>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    PIT_SET(PIT_OP_HEAT, PLAIN) PIT_SET(PIT_OP_HEAT, MIXED)
    PIT_SET(PIT_OP_VARHEAT, PLAIN) PIT_SET(PIT_OP_VARHEAT, MIXED)
    PIT_SET(PIT_OP_OU, PLAIN) PIT_SET(PIT_OP_OU, MIXED)
#undef PIT_SET
    if (e == cudaSuccess) g_max_smem = max_smem;
    return e;
}

cudaError_t launch_steps(int prec, const StepArgs &a, int threads, size_t smem, cudaStream_t s)
{
    const long long blocks = (long long)a.n_batch * a.n_grids;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL || smem > g_max_smem || threads < 32 || threads > 512 || (threads & 31))
        return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)blocks), block(threads);
    switch (a.op.op * 2 + prec) {
    case PIT_OP_HEAT * 2 + PLAIN: steps_kernel<PIT_OP_HEAT, PLAIN><<<grid, block, smem, s>>>(a); break;
    case PIT_OP_HEAT * 2 + MIXED: steps_kernel<PIT_OP_HEAT, MIXED><<<grid, block, smem, s>>>(a); break;
    case PIT_OP_VARHEAT * 2 + PLAIN: steps_kernel<PIT_OP_VARHEAT, PLAIN><<<grid, block, smem, s>>>(a); break;
    case PIT_OP_VARHEAT * 2 + MIXED: steps_kernel<PIT_OP_VARHEAT, MIXED><<<grid, block, smem, s>>>(a); break;
    case PIT_OP_OU * 2 + PLAIN: steps_kernel<PIT_OP_OU, PLAIN><<<grid, block, smem, s>>>(a); break;
    case PIT_OP_OU * 2 + MIXED: steps_kernel<PIT_OP_OU, MIXED><<<grid, block, smem, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pit
