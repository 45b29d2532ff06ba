// Batched backward-Euler propagator Phi (Sec. 2, Eq. "parabolic_problem_time_
// propagation"): for every (batch entry, component grid) item solve
//     (I + dt L_l) x = u_prev + dt f,   initial guess u_prev,
// matrix-free, with CG for the symmetric operators and BiCGStab for the
// drift operator (Sec. 4.1).
//
// Design (grid-resident): one CTA owns one item for the whole solve.  The
// Krylov vectors live in shared memory, the dot products are reduced by warp
// shuffles and one block barrier, and the iterate x is accumulated in the
// output buffer.  HBM is touched once to read u_prev (and f) and once to
// write x, instead of once per Krylov iteration; every grid of the
// workloads (at most 9261 nodes) fits on one SM.
//
// Two precision forms:
//   PLAIN  Krylov in FP64 until ||b - A x|| <= rtol ||b||.
//   MIXED  FP64 iterative refinement around an FP32 Krylov solve: the
//          residual b - A x is formed in FP64 from the FP64 iterate, the
//          correction equation is solved in FP32 to inner_rtol, and the
//          correction is added in FP64; same FP64 stopping rule.
#include <type_traits>

#include "pit_internal.cuh"

namespace pit {

#define FULL_MASK 0xffffffffu

// ----------------------------------------------------------------------------
// Operator coefficients of node j in FP64: q_j = diag p_j + sum_i cm_i p_{j-e_i}
// + cp_i p_{j+e_i}, with zero coefficients towards boundary nodes (zero
// Dirichlet values).  Matches the oracle's operator definitions:
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
// (bit 2i: node has an interior neighbour at -e_i, bit 2i+1: at +e_i).
template <typename T>
struct HeatSt {
    const uint16_t *mask;
    int d;
    int S[PIT_D];
    T diag;
    T off[PIT_D];
    template <typename P>
    __device__ __forceinline__ T operator()(const P *p, int j) const
    {
        const unsigned mk = mask[j];
        T s = diag * (T)p[j];
#pragma unroll
        for (int i = 0; i < PIT_D; ++i) {
            if (i >= d) break;
            const T pm = ((mk >> (2 * i)) & 1u) ? (T)p[j - S[i]] : T(0);
            const T pp = ((mk >> (2 * i + 1)) & 1u) ? (T)p[j + S[i]] : T(0);
            s += off[i] * (pm + pp);
        }
        return s;
    }
};

// Variable-coefficient stencil from a per-node table in shared memory
// (structure of arrays: tab[k*ld + j], k = 0 diagonal, 1+2i minus, 2+2i plus).
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

// FP64 stencil with coefficients evaluated on the fly (refinement residual of
// the variable-coefficient operators; a few evaluations per solve).
struct Op64St {
    const GridInfo *G;
    const OpParams *op;
    const double *faces;
    const uint16_t *mask;
    double dt;
    __device__ __forceinline__ double operator()(const double *p, int j) const
    {
        double diag, cm[PIT_D], cp[PIT_D];
        op_coef(*op, *G, faces, j, dt, diag, cm, cp);
        const unsigned mk = mask[j];
        double s = diag * p[j];
#pragma unroll
        for (int i = 0; i < PIT_D; ++i) {
            if (i >= op->d) break;
            const double pm = ((mk >> (2 * i)) & 1u) ? p[j - G->S[i]] : 0.0;
            const double pp = ((mk >> (2 * i + 1)) & 1u) ? p[j + G->S[i]] : 0.0;
            s += cm[i] * pm + cp[i] * pp;
        }
        return s;
    }
};

// ----------------------------------------------------------------------------
// Block reductions.  Each warp reduces with shuffles, lane 0 stores its
// partial in a 32-slot buffer, one barrier, and every thread adds the
// partials in the same order: all threads hold the bitwise same sum and the
// result does not depend on scheduling.  Callers alternate two buffers, so
// one barrier per reduction is enough: a warp can only overwrite a buffer
// after every warp has passed the barrier of the reduction in between.
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL_MASK, v, o);
    return v;
}

template <typename T>
struct Reducer {
    T *buf;    // two halves of 2 x 32 slots
    int slot;  // reductions done so far; selects the half
    template <int K>
    __device__ __forceinline__ void sum(T *v)
    {
        T *red = buf + (slot & 1) * 64;
        ++slot;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            T x = warp_sum(v[k]);
            if (lane == 0) red[k * 32 + w] = x;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < K; ++k) {
            T s = T(0);
            for (int q = 0; q < nw; ++q) s += red[k * 32 + q];
            v[k] = s;
        }
    }
};

__device__ __forceinline__ bool finite_pos(double v) { return v > 0.0 && v < 1.0e300; }
__device__ __forceinline__ bool finite_pos(float v) { return v > 0.0f && v < 1.0e37f; }

// ----------------------------------------------------------------------------
// Conjugate gradients on A e = r0 (r holds r0, p = r0, rr = r0.r0 on entry),
// accumulating the iterate into X (X may be global FP64 or shared FP32).
template <typename T, typename TX, class ST>
__device__ int cg_core(const ST &A, int n, TX *X, T *r, T *p, T *q, Reducer<T> &R, T rr, T stop2,
                       int maxit, int &status)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    int k = 0;
    status = PIT_OK;
    for (;;) {
        if (!(rr > stop2)) {
            if (rr != rr) status = PIT_ERR_NONFINITE;
            break;
        }
        if (k >= maxit) { status = PIT_ERR_NOCONV; break; }
        __syncthreads();  // p complete
        T pq[1] = {T(0)};
        for (int j = tid; j < n; j += nt) {
            const T qj = A(p, j);
            q[j] = qj;
            pq[0] += p[j] * qj;
        }
        R.template sum<1>(pq);
        if (!finite_pos(pq[0])) { status = (pq[0] != pq[0]) ? PIT_ERR_NONFINITE : PIT_ERR_BREAKDOWN; break; }
        const T alpha = rr / pq[0];
        T rn[1] = {T(0)};
        for (int j = tid; j < n; j += nt) {
            X[j] += (TX)(alpha * p[j]);
            const T rj = r[j] - alpha * q[j];
            r[j] = rj;
            rn[0] += rj * rj;
        }
        R.template sum<1>(rn);
        const T beta = rn[0] / rr;
        for (int j = tid; j < n; j += nt) p[j] = r[j] + beta * p[j];
        rr = rn[0];
        ++k;
    }
    return k;
}

// BiCGStab (van der Vorst 1992) on A e = r0 (r holds r0, rh = r0, p = v = 0
// on entry).  The vector s shares r's storage.
template <typename T, typename TX, class ST>
__device__ int bicgstab_core(const ST &A, int n, TX *X, T *r, T *rh, T *p, T *v, T *t, Reducer<T> &R,
                             T rr, T stop2, int maxit, int &status)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    T rho = T(1), alpha = T(1), omega = T(1);
    int k = 0;
    status = PIT_OK;
    for (;;) {
        if (!(rr > stop2)) {
            if (rr != rr) status = PIT_ERR_NONFINITE;
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
        rr = rn[0];
        ++k;
        if (omega == T(0) && rr > stop2) { status = PIT_ERR_BREAKDOWN; break; }
    }
    return k;
}

// ----------------------------------------------------------------------------
// Shared-memory layout of one item (n nodes, rounded up to ld = n rounded to 4):
//   vectors (nvec * ld of T), coefficient table (ntab * ld of T), mask (ld u16).
__host__ __device__ inline int phi_nvec(int prec, int op)
{
    if (op == PIT_OP_OU) return prec == PLAIN ? 5 : 6;
    return prec == PLAIN ? 3 : 4;
}

__host__ __device__ inline int phi_ntab(int op, int d) { return op == PIT_OP_HEAT ? 0 : 2 * d + 1; }

size_t phi_smem_bytes(int prec, int op, int d, int n)
{
    const size_t ld = (size_t)((n + 3) & ~3);
    const size_t esz = prec == PLAIN ? 8 : 4;
    return (size_t)(phi_nvec(prec, op) + phi_ntab(op, d)) * ld * esz + ld * 2 + 16;
}

template <int OP, int PREC>
__global__ void __launch_bounds__(512) phi_kernel(PhiArgs a)
{
    typedef typename std::conditional<PREC == PLAIN, double, float>::type T;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ GridInfo GI;
    __shared__ double red64[2 * 2 * 32];
    __shared__ float red32[2 * 2 * 32];

    const int gi = blockIdx.x % a.n_bucket;
    const int b = blockIdx.x / a.n_bucket;
    const int g = a.bucket_grids[gi];
    if (a.active && !a.active[g]) return;  // uniform over the block
    if (threadIdx.x == 0) GI = a.grids[g];
    __syncthreads();

    const int tid = threadIdx.x, nt = blockDim.x;
    const int n = GI.n, d = a.op.d;
    const int ld = (n + 3) & ~3;
    const double dt = a.dt;
    const double *in = a.in + (long long)b * a.in_stride + GI.off;
    const double *f = a.f ? a.f + (long long)b * a.f_stride + GI.off : nullptr;
    double *out = a.out + (long long)b * a.out_stride + GI.off;

    T *vec = reinterpret_cast<T *>(smem);
    const int nvec = phi_nvec(PREC, OP);
    T *tab = vec + (size_t)nvec * ld;
    uint16_t *mask = reinterpret_cast<uint16_t *>(tab + (size_t)phi_ntab(OP, d) * ld);

    // neighbour masks and (variable-coefficient operators) the coefficient table
    for (int j = tid; j < n; j += nt) {
        unsigned mk = 0;
#pragma unroll
        for (int i = 0; i < PIT_D; ++i) {
            if (i >= d) break;
            const int c = (j / GI.S[i]) % GI.N[i];
            if (c > 0) mk |= 1u << (2 * i);
            if (c < GI.N[i] - 1) mk |= 1u << (2 * i + 1);
        }
        mask[j] = (uint16_t)mk;
        if constexpr (OP != PIT_OP_HEAT) {
            double diag, cm[PIT_D], cp[PIT_D];
            op_coef(a.op, GI, a.faces, j, dt, diag, cm, cp);
            tab[j] = (T)diag;
            for (int i = 0; i < d; ++i) {
                tab[(1 + 2 * i) * ld + j] = (T)cm[i];
                tab[(2 + 2 * i) * ld + j] = (T)cp[i];
            }
        }
    }
    // constant heat coefficients (FP64 and working precision)
    HeatSt<double> H64;
    HeatSt<T> HT;
    H64.mask = HT.mask = mask;
    H64.d = HT.d = d;
    {
        double diag = 1.0;
        for (int i = 0; i < PIT_D; ++i) {
            const double ih2 = (i < d) ? 1.0 / (GI.h[i] * GI.h[i]) : 0.0;
            H64.S[i] = HT.S[i] = (i < d) ? GI.S[i] : 0;
            H64.off[i] = -dt * ih2;
            HT.off[i] = (T)(-dt * ih2);
            diag += 2.0 * dt * ih2;
        }
        H64.diag = diag;
        HT.diag = (T)diag;
    }
    TabSt<T> TT;
    TT.mask = mask;
    TT.tab = tab;
    TT.ld = ld;
    TT.d = d;
    for (int i = 0; i < PIT_D; ++i) TT.S[i] = (i < d) ? GI.S[i] : 0;
    Op64St O64{&GI, &a.op, a.faces, mask, dt};
    __syncthreads();

    Reducer<double> R64{red64, 0};
    Reducer<float> R32{red32, 0};
    int status = PIT_OK, iters = 0, passes = 0;

    if constexpr (PREC == PLAIN) {
        T *r = vec, *p = vec + ld, *q = vec + 2 * ld;
        T *rh = vec + 2 * ld, *v = vec + 3 * ld, *t = vec + 4 * ld;  // BiCGStab uses r, rh, p, v, t
        double acc[2] = {0.0, 0.0};
        for (int j = tid; j < n; j += nt) {
            const double bj = in[j] + (f ? dt * f[j] : 0.0);
            double Ax;
            if constexpr (OP == PIT_OP_HEAT) Ax = H64(in, j);
            else Ax = O64(in, j);
            const double rj = bj - Ax;
            r[j] = rj;
            out[j] = in[j];
            if constexpr (OP == PIT_OP_OU) { rh[j] = rj; p[j] = 0.0; v[j] = 0.0; }
            else p[j] = rj;
            acc[0] += bj * bj;
            acc[1] += rj * rj;
        }
        R64.template sum<2>(acc);
        const double stop2 = a.rtol * a.rtol * acc[0];
        Reducer<double> &R = R64;
        if constexpr (OP == PIT_OP_OU) {
            iters = bicgstab_core<double, double>(TT, n, out, (double *)r, (double *)rh, (double *)p,
                                                  (double *)v, (double *)t, R, acc[1], stop2, a.maxit, status);
        } else if constexpr (OP == PIT_OP_HEAT) {
            iters = cg_core<double, double>(H64, n, out, (double *)r, (double *)p, (double *)q, R, acc[1], stop2,
                                            a.maxit, status);
        } else {
            iters = cg_core<double, double>(TT, n, out, (double *)r, (double *)p, (double *)q, R, acc[1], stop2,
                                            a.maxit, status);
        }
        passes = 1;
    } else {
        float *e = (float *)vec, *r = (float *)vec + ld, *p = (float *)vec + 2 * ld, *q = (float *)vec + 3 * ld;
        float *rh = (float *)vec + 3 * ld, *v = (float *)vec + 4 * ld, *t = (float *)vec + 5 * ld;
        double bb[1] = {0.0};
        for (int j = tid; j < n; j += nt) {
            const double bj = in[j] + (f ? dt * f[j] : 0.0);
            out[j] = in[j];
            bb[0] += bj * bj;
        }
        R64.template sum<1>(bb);
        const double stop2 = a.rtol * a.rtol * bb[0];
        for (;;) {
            __syncthreads();  // iterate visible to the whole block
            double rn2[1] = {0.0};
            for (int j = tid; j < n; j += nt) {
                const double bj = in[j] + (f ? dt * f[j] : 0.0);
                double Ax;
                if constexpr (OP == PIT_OP_HEAT) Ax = H64(out, j);
                else Ax = O64(out, j);
                const double rj = bj - Ax;
                r[j] = (float)rj;
                rn2[0] += rj * rj;
            }
            R64.template sum<1>(rn2);
            if (!(rn2[0] > stop2)) {
                if (rn2[0] != rn2[0]) status = PIT_ERR_NONFINITE;
                break;
            }
            if (passes >= a.ir_maxit) { status = PIT_ERR_NOCONV; break; }
            const double rnorm = sqrt(rn2[0]);
            const float inv = (float)(1.0 / rnorm);
            float rr[1] = {0.0f};
            for (int j = tid; j < n; j += nt) {
                const float rj = r[j] * inv;
                r[j] = rj;
                e[j] = 0.0f;
                if constexpr (OP == PIT_OP_OU) { rh[j] = rj; p[j] = 0.0f; v[j] = 0.0f; }
                else p[j] = rj;
                rr[0] += rj * rj;
            }
            R32.template sum<1>(rr);
            const float stop32 = a.inner_rtol * a.inner_rtol * rr[0];
            int st = PIT_OK, k;
            if constexpr (OP == PIT_OP_OU)
                k = bicgstab_core<float, float>(TT, n, e, r, rh, p, v, t, R32, rr[0], stop32, a.maxit, st);
            else if constexpr (OP == PIT_OP_HEAT)
                k = cg_core<float, float>(HT, n, e, r, p, q, R32, rr[0], stop32, a.maxit, st);
            else
                k = cg_core<float, float>(TT, n, e, r, p, q, R32, rr[0], stop32, a.maxit, st);
            iters += k;
            ++passes;
            if (st == PIT_ERR_NONFINITE) { status = st; break; }
            // an inner solve that stalls (FP32 floor) or breaks down still
            // yields a usable correction; the FP64 residual decides.
            for (int j = tid; j < n; j += nt) out[j] += (double)e[j] * rnorm;
        }
    }
    // out = post_scale * x + gpost: each thread its own nodes, after a barrier
    // that ended every neighbour read of x.
    __syncthreads();
    const double *gp = a.gpost ? a.gpost + (long long)b * a.g_stride + GI.off : nullptr;
    if (a.post_scale != 1.0 || gp) {
        for (int j = tid; j < n; j += nt) out[j] = a.post_scale * out[j] + (gp ? gp[j] : 0.0);
    }
    if (tid == 0 && a.stats) {
        atomicAdd(&a.stats->sum_iters, (unsigned long long)iters);
        atomicAdd(&a.stats->items, 1ull);
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
#define PIT_SET(OPV, PV)                                                                                  \
    if (e == cudaSuccess)                                                                                 \
        e = cudaFuncSetAttribute(phi_kernel<OPV, PV>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    PIT_SET(PIT_OP_HEAT, PLAIN) PIT_SET(PIT_OP_HEAT, MIXED)
    PIT_SET(PIT_OP_VARHEAT, PLAIN) PIT_SET(PIT_OP_VARHEAT, MIXED)
    PIT_SET(PIT_OP_OU, PLAIN) PIT_SET(PIT_OP_OU, MIXED)
#undef PIT_SET
    if (e == cudaSuccess) g_max_smem = max_smem;
    return e;
}

cudaError_t launch_phi_bucket(int prec, const PhiArgs &a, int threads, size_t smem, cudaStream_t s)
{
    const long long blocks = (long long)a.n_batch * a.n_bucket;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL || smem > g_max_smem) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)blocks), block(threads);
    switch (a.op.op * 2 + prec) {
    case PIT_OP_HEAT * 2 + PLAIN: phi_kernel<PIT_OP_HEAT, PLAIN><<<grid, block, smem, s>>>(a); break;
    case PIT_OP_HEAT * 2 + MIXED: phi_kernel<PIT_OP_HEAT, MIXED><<<grid, block, smem, s>>>(a); break;
    case PIT_OP_VARHEAT * 2 + PLAIN: phi_kernel<PIT_OP_VARHEAT, PLAIN><<<grid, block, smem, s>>>(a); break;
    case PIT_OP_VARHEAT * 2 + MIXED: phi_kernel<PIT_OP_VARHEAT, MIXED><<<grid, block, smem, s>>>(a); break;
    case PIT_OP_OU * 2 + PLAIN: phi_kernel<PIT_OP_OU, PLAIN><<<grid, block, smem, s>>>(a); break;
    case PIT_OP_OU * 2 + MIXED: phi_kernel<PIT_OP_OU, MIXED><<<grid, block, smem, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pit
