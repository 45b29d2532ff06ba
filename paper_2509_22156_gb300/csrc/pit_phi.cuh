// Device code of the batched multi-step backward-Euler propagator
// (Sec. 2, Eq. "parabolic_problem_time_propagation"): every (batch entry,
// component grid) item is advanced by nsteps backward-Euler steps
//     (I + dt L_l) x_s = x_{s-1} + dt f,   x_s <- x_s + g_s (optional forcing),
// each solved matrix-free with CG (symmetric operators) or BiCGStab (drift
// operator, Sec. 4.1), initial guess x_{s-1}.
//
// Design (grid-resident, multi-step): one CTA owns one item for all its
// steps.  The FP64 state, the Krylov vectors and the neighbour masks live in
// shared memory; dot products are reduced with warp shuffles and one block
// barrier.  A whole F-relaxation interval or a sequential coarse sweep is one
// launch; HBM is touched once to read the start state and once per stored
// output state; the intermediate F-values never leave the SM (the C-point-only
// storage of Sec. 3.3.2).  Kernels are instantiated per dimension D so that
// every per-axis loop is unrolled and per-axis constants stay in registers.
//
// Precision forms:
//   PLAIN  Krylov in FP64 until ||b - A x|| <= rtol ||b||.
//   MIXED  FP64 iterative refinement around an FP32 Krylov solve: residual
//          b - A x formed in FP64 from the FP64 state, the correction equation
//          solved in FP32, the correction added in FP64; same FP64 stopping
//          rule.  The FP32 target of each correction solve is the looser of
//          inner_rtol and half of what the FP64 tolerance still asks for.  On
//          GB300 FP64 arithmetic (and the hardware FP64<->FP32 conversion)
//          runs at 1/58 of the FP32 rate, so the FP64 stencil passes bound the
//          kernel and are kept lean: when a step has no forcing, the FP64 pass
//          that verifies step s gives r_s = b_s - A x_s, hence
//          c_s = x_s - A x_s = r_s + (x_s - x_{s-1}), the initial residual of
//          step s+1 for the guess x_s, without a stencil pass; and with
//          c_{s-1} kept in FP64 the residual of the extrapolated guess
//          2 x_s - x_{s-1} is c_s - c_{s-1} + r_s, also without one (the
//          extrapolation starts a smooth solution's step about (dt lambda)^2
//          instead of dt lambda from its solution, so one FP32 correction
//          mostly suffices).  Each step then costs one FP64 stencil pass per
//          correction.  The FP64 pipe does only what needs FP64 (the stencil on
//          the FP64 state, b - A x, the carried residuals): conversions run on
//          the integer pipes with an exact power-of-two scale, and the squared
//          norms that feed the stopping test and the tolerances are summed from
//          the FP32 copies (relative accuracy about 1e-7, far below what a
//          stopping test resolves).
//   PAIR   the MIXED refinement with the state and right-hand side held as
//          pairs of FP32 numbers (about 48 significant bits, scaled by a power
//          of two) and b - A x formed from them by error-free FP32
//          transformations (PairHeat, PairTab): no FP64 arithmetic per step
//          (heat and variable-coefficient operators).
//   SINGLE FP32 Krylov on an FP32 copy of the state scaled by a power of two,
//          for loose tolerances (the coarse correction solves).
// CG uses the Chronopoulos-Gear recurrences: the update pass sums (r,r) of
// the new residual, whose reduction (one barrier) decides convergence before
// the stencil pass forms A r and (Ar,r) (a second reduction): the last,
// converged iteration of every solve skips its stencil pass.
#pragma once

#include <type_traits>

#include "pit_internal.cuh"

namespace pit {

#define PIT_FULL_MASK 0xffffffffu

// ----------------------------------------------------------------------------
// Operator coefficients of node j in FP64: (A p)_j = diag p_j + sum_i cm_i
// p_{j-e_i} + cp_i p_{j+e_i}, zero towards boundary nodes (zero Dirichlet):
//   heat    L p = sum_i (2 p_j - p_- - p_+) / h_i^2
//   varheat L p = sum_i [a_+ (p_j - p_+) + a_- (p_j - p_-)] / h_i^2
//   OU      L p = sum_i (F_+ - F_-) / h_i + (sigma^2/2)(2 p_j - p_- - p_+) / h_i^2,
//           F_+ = max(v_+,0) p_j + min(v_+,0) p_+,  v_+ = -theta (x_i + h_i/2).
//   LSDE    the donor-cell (or central) flux with the face velocity (A x)_i of the
//           linear SDE dX = A X dt + sigma dW (Sec. 4.4) and diffusion
//           (H_ii/2)(2 p_j - p_- - p_+) / h_i^2; its mixed-derivative terms
//           (i != k) are constant per grid and applied by TabSt<.., true>.
//   CME     toggle-switch chemical master equation (Sec. 4.3): the same
//           flux with face velocity a_i - g_i x_i (production a_i, degradation
//           g_i x_i) and the second difference of (a_i + g_i x_i) p / 2.
template <int D>
__device__ __forceinline__ void op_coef(const OpParams &op, const GridInfo &G, const double *faces, int j,
                                        double dt, double &diag, double *cm, double *cp)
{
    diag = 1.0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        const int c = (j / G.S[i]) % G.N[i];
        const double h = G.h[i];
        const double ih2 = 1.0 / (h * h);
        double dd, dm, dp;
        if (op.op == PIT_OP_HEAT) {
            dd = 2.0 * ih2; dm = -ih2; dp = -ih2;
        } else if (op.op == PIT_OP_VARHEAT) {
            const double am = faces[(G.off + j) * (2 * D) + 2 * i];
            const double ap = faces[(G.off + j) * (2 * D) + 2 * i + 1];
            dd = (am + ap) * ih2; dm = -am * ih2; dp = -ap * ih2;
        } else if (op.op == PIT_OP_OU) {
            const double x = op.lo[i] + (double)(c + 1) * h;
            const double vp = -op.theta * (x + 0.5 * h);
            const double vm = -op.theta * (x - 0.5 * h);
            const double s2 = 0.5 * op.sigma * op.sigma * ih2;
            drift_coef(vp, vm, h, false, dd, dm, dp);
            dd += 2.0 * s2;
            dm -= s2;
            dp -= s2;
        } else if (op.op == PIT_OP_CME) {
            double xc[D];
#pragma unroll
            for (int k = 0; k < D; ++k) xc[k] = op.lo[k] + (double)((j / G.S[k]) % G.N[k] + 1) * G.h[k];
            cme_coef(cme_production(op, i, xc, D), op.cg[i], xc[i], h, op.central != 0, dd, dm, dp);
        } else {
            // face velocities (A x)_i at x -+ h/2 e_i
            double ax = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) ax += op.A[i * D + k] * (op.lo[k] + (double)((j / G.S[k]) % G.N[k] + 1) * G.h[k]);
            const double vp = ax + 0.5 * h * op.A[i * D + i];
            const double vm = ax - 0.5 * h * op.A[i * D + i];
            const double s2 = 0.5 * op.H[i * D + i] * ih2;
            drift_coef(vp, vm, h, op.central != 0, dd, dm, dp);
            dd += 2.0 * s2;
            dm -= s2;
            dp -= s2;
        }
        diag += dt * dd;
        cm[i] = (c > 0) ? dt * dm : 0.0;
        cp[i] = (c < G.N[i] - 1) ? dt * dp : 0.0;
    }
}

// Constant-coefficient heat stencil with a per-node neighbour mask
// (bit 2i: interior neighbour at -e_i, bit 2i+1: at +e_i).
template <typename T, int D>
struct HeatSt {
    const uint16_t *mask;
    int S[D];
    T diag;
    T off[D];
    __device__ __forceinline__ T operator()(const T *p, int j) const
    {
        const unsigned mk = mask[j];
        T s = diag * p[j];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const T pm = ((mk >> (2 * i)) & 1u) ? p[j - S[i]] : T(0);
            const T pp = ((mk >> (2 * i + 1)) & 1u) ? p[j + S[i]] : T(0);
            s += off[i] * (pm + pp);
        }
        return s;
    }
    // b_j - (A p)_j as one chain of fused multiply-adds (one instruction fewer
    // than the product followed by a subtraction)
    __device__ __forceinline__ T resid(T bj, const T *p, int j) const
    {
        const unsigned mk = mask[j];
        T s = fma(-diag, p[j], bj);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const T pm = ((mk >> (2 * i)) & 1u) ? p[j - S[i]] : T(0);
            const T pp = ((mk >> (2 * i + 1)) & 1u) ? p[j + S[i]] : T(0);
            s = fma(-off[i], pm + pp, s);
        }
        return s;
    }
};

// Variable-coefficient stencil from a per-node table in shared memory
// (structure of arrays: tab[k*ld + j], k = 0 diagonal, 1+2i minus, 2+2i plus;
// zero coefficients towards the boundary).  CROSS adds the mixed-derivative
// terms of the linear-SDE operator, constant per grid: for every axis pair
// i < k, cr[q] (p_{++} - p_{+-} - p_{-+} + p_{--}) over the four diagonal
// neighbours j +- e_i +- e_k, a corner outside the grid reading zero.
template <typename T, int D, bool CROSS = false>
struct TabSt {
    static constexpr int NP = D * (D - 1) / 2;
    const uint16_t *mask;
    const T *tab;
    int ld;
    int S[D];
    T cr[NP > 0 ? NP : 1];
    bool unit = false;  // Jacobi-scaled table: unit diagonal, the diagonal slot holds D^{-1/2}
    __device__ __forceinline__ T operator()(const T *p, int j) const
    {
        const unsigned mk = mask[j];
        T s = unit ? p[j] : tab[j] * p[j];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const int jm = ((mk >> (2 * i)) & 1u) ? j - S[i] : j;
            const int jp = ((mk >> (2 * i + 1)) & 1u) ? j + S[i] : j;
            s += tab[(1 + 2 * i) * ld + j] * p[jm] + tab[(2 + 2 * i) * ld + j] * p[jp];
        }
        if constexpr (CROSS && NP > 0) s += cross(p, j, mk);
        return s;
    }
    __device__ __forceinline__ T cross(const T *p, int j, unsigned mk) const
    {
        T s = T(0);
        int q = 0;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const bool im = (mk >> (2 * i)) & 1u, ip = (mk >> (2 * i + 1)) & 1u;
#pragma unroll
            for (int k = i + 1; k < D; ++k, ++q) {
                const bool km = (mk >> (2 * k)) & 1u, kp = (mk >> (2 * k + 1)) & 1u;
                T c = T(0);
                if (ip && kp) c += p[j + S[i] + S[k]];
                if (ip && km) c -= p[j + S[i] - S[k]];
                if (im && kp) c -= p[j - S[i] + S[k]];
                if (im && km) c += p[j - S[i] - S[k]];
                s += cr[q] * c;
            }
        }
        return s;
    }
    // b_j - (A p)_j as one chain of fused multiply-adds (unscaled table)
    __device__ __forceinline__ T resid(T bj, const T *p, int j) const
    {
        const unsigned mk = mask[j];
        T s = fma(-tab[j], p[j], bj);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const int jm = ((mk >> (2 * i)) & 1u) ? j - S[i] : j;
            const int jp = ((mk >> (2 * i + 1)) & 1u) ? j + S[i] : j;
            s = fma(-tab[(1 + 2 * i) * ld + j], p[jm], s);
            s = fma(-tab[(2 + 2 * i) * ld + j], p[jp], s);
        }
        if constexpr (CROSS && NP > 0) s -= cross(p, j, mk);
        return s;
    }
};

// ----------------------------------------------------------------------------
// Block reductions: warp shuffles, one partial per warp in a 32-slot buffer,
// one barrier, then every warp reduces the nw partials with the same shuffle
// tree (log2 nw levels) and broadcasts lane 0: all threads hold the bitwise
// same value, independent of scheduling.  Consecutive reductions alternate two
// buffers, so one barrier per reduction suffices (a warp can only reuse a
// buffer after every warp passed the barrier of the reduction in between).
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(PIT_FULL_MASK, v, o);
    return v;
}

template <typename T>
struct Reducer {
    T *buf;    // two halves of 4 x 32 slots
    int slot;
    // first stage: warp sums into the current half; returns that half
    template <int K>
    __device__ __forceinline__ T *stage1(const T *v)
    {
        static_assert(K <= 4, "at most four values per reduction");
        T *red = buf + (slot & 1) * 128;
        ++slot;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const T x = warp_sum(v[k]);
            if (lane == 0) red[k * 32 + w] = x;
        }
        return red;
    }
    // second stage, after the barrier: sum of the nw warp partials
    template <int K>
    __device__ __forceinline__ void stage2(const T *red, T *v)
    {
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        const int top = 1 << (32 - __clz(nw - 1));  // nw rounded up to a power of two
#pragma unroll
        for (int k = 0; k < K; ++k) {
            T x = (lane < nw) ? red[k * 32 + lane] : T(0);
            for (int o = top >> 1; o > 0; o >>= 1) x += __shfl_down_sync(PIT_FULL_MASK, x, o);
            v[k] = __shfl_sync(PIT_FULL_MASK, x, 0);
        }
    }
    template <int K>
    __device__ __forceinline__ void sum(T *v)
    {
        const T *red = stage1<K>(v);
        __syncthreads();
        stage2<K>(red, v);
    }
};

// KD FP64 and KF FP32 sums behind one barrier.
template <int KD, int KF>
__device__ __forceinline__ void sum_mixed(Reducer<double> &Rd, double *vd, Reducer<float> &Rf, float *vf)
{
    const double *rd = Rd.template stage1<KD>(vd);
    const float *rf = Rf.template stage1<KF>(vf);
    __syncthreads();
    Rd.template stage2<KD>(rd, vd);
    Rf.template stage2<KF>(rf, vf);
}

// ----------------------------------------------------------------------------
// Conversions between FP64 and FP32 by IEEE-754 bit-field arithmetic on the
// integer pipes, with an exact power-of-two scale folded into the exponent.
// GB300 executes the hardware conversion instructions on its FP64 pipe at the
// FP64 rate; these keep that pipe for the residual arithmetic.
//   to_f32(v, k): v 2^k with the mantissa truncated to 24 bits (error below
//     one FP32 ulp); zero when v 2^k is below the normal FP32 range, infinity
//     or NaN when it is above it or v is not finite.
//   to_f64(f, k): f 2^k exactly for normal f; zero for zero or subnormal f or
//     when the result would be below the normal FP64 range.
__device__ __forceinline__ float to_f32(double v, int k)
{
    const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
    const int ex = (int)((hi >> 20) & 0x7ffu) - (1023 - 127) + k;  // FP32 biased exponent
    const unsigned sign = hi & 0x80000000u;
    const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned bits = sign | ((unsigned)min(ex, 255) << 23) | mant;
    return __uint_as_float(ex > 0 ? bits : sign);
}
// to_f32_rn: the same with the mantissa rounded to nearest (ties away from
//   zero): for residuals that a single correction solves for, where
//   truncation's bias toward zero would leave the same sign of error in
//   every step.
__device__ __forceinline__ float to_f32_rn(double v, int k)
{
    const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
    const int ex = (int)((hi >> 20) & 0x7ffu) - (1023 - 127) + k;
    const unsigned sign = hi & 0x80000000u;
    const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned mag = ((unsigned)min(ex, 255) << 23) | mant;
    // first dropped bit: add one unit in the last place of the magnitude (a
    // carry out of the mantissa moves into the exponent, up to infinity)
    const unsigned rmag = ex < 255 ? mag + ((lo >> 28) & 1u) : mag;
    return __uint_as_float(ex > 0 ? (sign | rmag) : sign);
}
__device__ __forceinline__ double to_f64(float f, int k)
{
    const unsigned u = __float_as_uint(f);
    const unsigned sign = u & 0x80000000u;
    const int ef = (int)((u >> 23) & 0xffu);
    const unsigned m = u & 0x7fffffu;
    const int ex = min(ef == 255 ? 2047 : ef + (1023 - 127) + k, 2047);
    const bool zero = (ef == 0) || (ex <= 0);
    const unsigned hi = zero ? sign : (sign | ((unsigned)ex << 20) | (m >> 3));
    const unsigned lo = zero ? 0u : (m << 29);
    return __hiloint2double((int)hi, (int)lo);
}
// 2^k as FP64 for |k| <= 1022
__device__ __forceinline__ double pow2d(int k) { return __hiloint2double((1023 + k) << 20, 0); }
// k with ||b|| 2^k in [1, 2) from bb = ||b||^2 (0 for bb = 0 or not finite)
__device__ __forceinline__ int scale_exp(double bb)
{
    const int eb = (int)(((unsigned)__double2hiint(bb) >> 20) & 0x7ffu);
    if (eb == 0 || eb == 2047) return eb == 0 && bb != 0.0 ? 540 : 0;
    const int e = eb - 1023;
    const int half = (e >= 0) ? e / 2 : -((1 - e) / 2);  // floor(e / 2)
    return -half;
}

// ----------------------------------------------------------------------------
// FP32 pairs: a value held as hi + lo with |lo| <= ulp(hi) / 2 carries about 48
// significant bits (Dekker 1971).  two_sum is Knuth's error-free addition
// (s + e = a + b exactly, no ordering of |a| and |b| needed); the error of a
// product comes from one FMA (p = fl(a b), e = a b - p exactly).  The
// round-to-nearest intrinsics keep the compiler from contracting these
// operations into FMAs, which would break the exactness.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}
// v 2^k as a pair: hi = v 2^k truncated to 24 bits; lo = the next 24 bits of
// the remainder v - hi 2^-k (exact in FP64: the low bits of v).  One FP64
// subtraction; the scale is exact.
__device__ __forceinline__ float2 split_pair(double v, int k)
{
    const float hi = to_f32(v, k);
    return make_float2(hi, to_f32(v - to_f64(hi, -k), k));
}
// (hi + lo) 2^-k in FP64: both parts convert exactly, one FP64 addition rounds
__device__ __forceinline__ double pair_to_f64(float2 p, int k) { return to_f64(p.x, -k) + to_f64(p.y, -k); }
// pair + FP32 value, renormalised
__device__ __forceinline__ float2 pair_add(float2 x, float v)
{
    float s, e, h, l;
    two_sum(x.x, v, s, e);
    two_sum(s, __fadd_rn(e, x.y), h, l);
    return make_float2(h, l);
}
// pair + pair, renormalised (relative error about 2^-47 of the larger operand)
__device__ __forceinline__ float2 pair_add(float2 x, float2 y)
{
    float s, e, h, l;
    two_sum(x.x, y.x, s, e);
    two_sum(s, __fadd_rn(e, __fadd_rn(x.y, y.y)), h, l);
    return make_float2(h, l);
}

// b_j - (A x)_j of the constant-coefficient heat stencil on pairs (state and
// right-hand side scaled by the same power of two), rounded once to FP32:
//     A x = x + sum_i c_i (2 x_j - x_{j-e_i} - x_{j+e_i}),  c_i = dt / h_i^2,
// with zero neighbours towards the boundary (the same operator as HeatSt).
// The hi parts of b - x and of the neighbour differences are formed with
// two_sum, c_i (a pair) times the difference with the FMA product error, and
// the big terms are summed with two_sum; every rounding error, the lo parts
// and the small cross products go to one FP32 compensation term.  The lo
// parts of the differences are combined in FP32, so the residual is lost
// below about 2^-48 (|x_j| + sum_i c_i (2 |x_j| + |x_m| + |x_p|)) (the FP64
// residual's bound with 2^-48 for 2^-53): far below the 1e-11 relative
// residuals the refinement asks for unless dt / h^2 reaches the hundreds.
// Also yields x_j - b_j rounded to FP32.
template <int D>
struct PairHeat {
    const uint16_t *mask;
    int S[D];
    float ch[D], cl[D];
    __device__ __forceinline__ float operator()(const float2 *x, const float2 *bv, int j, float &xmb) const
    {
        const unsigned mk = mask[j];
        const float2 xj = x[j], bj = bv[j];
        float s, comp;
        two_sum(bj.x, -xj.x, s, comp);
        comp = __fadd_rn(comp, __fsub_rn(bj.y, xj.y));
        xmb = -__fadd_rn(s, comp);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const float2 xm = ((mk >> (2 * i)) & 1u) ? x[j - S[i]] : make_float2(0.0f, 0.0f);
            const float2 xq = ((mk >> (2 * i + 1)) & 1u) ? x[j + S[i]] : make_float2(0.0f, 0.0f);
            float a1, e1, a2, e2, t, e3, e4;
            two_sum(xj.x, -xm.x, a1, e1);
            two_sum(xj.x, -xq.x, a2, e2);
            two_sum(a1, a2, t, e3);
            const float tl = ((e1 + e2) + e3) + ((2.0f * xj.y - xm.y) - xq.y);
            const float p = __fmul_rn(ch[i], t);
            const float q = __fmaf_rn(ch[i], t, -p) + (ch[i] * tl + cl[i] * t);
            two_sum(s, -p, s, e4);
            comp = comp + (e4 - q);
        }
        return __fadd_rn(s, comp);
    }
};

// The same for the variable-coefficient operator, from the face
// coefficients c = dt a / h_i^2 of every node held as pairs (zero neighbours
// towards the boundary, whose face coefficient still counts):
//     A x = x + sum_i c_{j-e_i/2} (x_j - x_{j-e_i}) + c_{j+e_i/2} (x_j - x_{j+e_i}).
// Table layout: c[(2 i) ld + j] towards -e_i, c[(2 i + 1) ld + j] towards +e_i.
template <int D>
struct PairTab {
    const uint16_t *mask;
    const float2 *c;
    int ld;
    int S[D];
    __device__ __forceinline__ float operator()(const float2 *x, const float2 *bv, int j, float &xmb) const
    {
        const unsigned mk = mask[j];
        const float2 xj = x[j], bj = bv[j];
        float s, comp;
        two_sum(bj.x, -xj.x, s, comp);
        comp = __fadd_rn(comp, __fsub_rn(bj.y, xj.y));
        xmb = -__fadd_rn(s, comp);
#pragma unroll
        for (int i = 0; i < D; ++i) {
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const bool inner = (mk >> (2 * i + side)) & 1u;
                const float2 xn = inner ? x[side ? j + S[i] : j - S[i]] : make_float2(0.0f, 0.0f);
                const float2 cf = c[(2 * i + side) * ld + j];
                float dh, e1, e2;
                two_sum(xj.x, -xn.x, dh, e1);
                const float dl = e1 + (xj.y - xn.y);
                const float p = __fmul_rn(cf.x, dh);
                const float q = __fmaf_rn(cf.x, dh, -p) + (cf.x * dl + cf.y * dh);
                two_sum(s, -p, s, e2);
                comp = comp + (e2 - q);
            }
        }
        return __fadd_rn(s, comp);
    }
};

__device__ __forceinline__ bool finite_pos(double v) { return v > 0.0 && v < 1.0e300; }
__device__ __forceinline__ bool finite_pos(float v) { return v > 0.0f && v < 1.0e37f; }

// ----------------------------------------------------------------------------
// CG with the Chronopoulos & Gear (1989) recurrences on A e = r0: r holds r0
// on entry (own nodes written by the caller), the iterate is accumulated into
// X (FP64 state or FP32 correction).  Stops when (r,r) <= stop2, tested on
// the sum of the update pass before the stencil pass of the next iteration.
template <typename T, typename TX, class ST>
__device__ int cg_core(const ST &A, int n, TX *X, T *r, T *p, T *s, T *w, Reducer<T> &R, T stop2, int maxit,
                       int &status)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    status = PIT_OK;
    __syncthreads();  // r complete
    T v[2] = {T(0), T(0)};
#pragma unroll 4
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
        // (r, r) of the new residual is summed in the update pass and tested
        // before the stencil: the converged last iteration skips A r
        T rr[1] = {T(0)};
#pragma unroll 4
        for (int j = tid; j < n; j += nt) {
            const T pj = first ? r[j] : r[j] + beta * p[j];
            const T sj = first ? w[j] : w[j] + beta * s[j];
            p[j] = pj;
            s[j] = sj;
            X[j] += (TX)(alpha * pj);
            const T rj = r[j] - alpha * sj;
            r[j] = rj;
            rr[0] += rj * rj;
        }
        first = false;
        ++k;
        R.template sum<1>(rr);  // also: r complete
        if (!(rr[0] > stop2)) {
            if (rr[0] != rr[0]) status = PIT_ERR_NONFINITE;
            break;
        }
        T wr[1] = {T(0)};
#pragma unroll 4
        for (int j = tid; j < n; j += nt) {
            const T wj = A(r, j);
            w[j] = wj;
            wr[0] += wj * r[j];
        }
        R.template sum<1>(wr);
        beta = rr[0] / gam;
        const T den = wr[0] - beta * rr[0] / alpha;
        if (!finite_pos(den)) { status = (den != den) ? PIT_ERR_NONFINITE : PIT_ERR_BREAKDOWN; break; }
        alpha = rr[0] / den;
        gam = rr[0];
    }
    return k;
}

// Line preconditioner of the constant-coefficient heat operator: M keeps the
// full diagonal dg of A = I + dt L and the couplings o along one axis a (the
// finest), so M is the tridiagonal Toeplitz matrix tridiag(o, dg, o) on every
// grid line along a (zero Dirichlet values).  For a grid whose axis a is much
// finer than the others, M captures the stiff part of A and the preconditioned
// CG needs a few iterations where the plain one needs tens.
//
// M^{-1} r is a partitioned tridiagonal solve, so that one long line (the
// 1-D-like grids of the combination technique) still keeps many threads busy:
// every line is cut into P chunks (P - 1 of length L, the last of length Lz).
// On a chunk with left and right outside neighbours xl, xr,
//     x = g - xl alpha - xr beta,  T g = r_chunk, T alpha = o e_first, T beta = o e_last
// (T the chunk's own tridiag(o, dg, o)).  The chunk ends give a small system
// in the boundary values, solved per line by one forward and one backward
// sweep over the chunks (phase 2), after which every interior node is updated
// (phase 3).  Everything that depends on the matrix only (the LU factors of
// both chunk lengths, alpha, beta, and the reduced-system coefficients) is the
// same on every line and is computed once per launch (setup).
// Line l = hi S_a + lo, node k of the line at hi S_a N_a + lo + k S_a.
template <typename T>
struct LineM {
    const T *f;  // factors: see setup()
    T off;
    int Na, Sa, nlines, P, L, Lz;
    // shared-memory floats the factors need for a line of n nodes (upper bound)
    __host__ __device__ static int floats(int n) { return 6 * n + 3 * 33 + 8; }
    __device__ __forceinline__ const T *cz() const { return f; }
    __device__ __forceinline__ const T *pz() const { return f + Lz; }
    __device__ __forceinline__ const T *az() const { return f + 2 * Lz; }
    __device__ __forceinline__ const T *bz() const { return f + 3 * Lz; }
    __device__ __forceinline__ const T *cf() const { return f + 4 * Lz; }
    __device__ __forceinline__ const T *pf() const { return f + 4 * Lz + L; }
    __device__ __forceinline__ const T *af() const { return f + 4 * Lz + 2 * L; }
    __device__ __forceinline__ const T *bf() const { return f + 4 * Lz + 3 * L; }
    __device__ __forceinline__ const T *psi() const { return f + 4 * Lz + 4 * L; }
    __device__ __forceinline__ const T *nu() const { return f + 4 * Lz + 4 * L + P; }
    __device__ __forceinline__ const T *den() const { return f + 4 * Lz + 4 * L + 2 * P; }

    // chunk layout for nt threads: about nt / nlines chunks per line (at most
    // 32), every chunk at least 2 nodes long
    __device__ void layout(int na, int sa, int n, int nt)
    {
        Na = na;
        Sa = sa;
        nlines = n / na;
        int p = nt / nlines;
        p = p < 1 ? 1 : (p > 32 ? 32 : p);
        if (p > na / 2) p = na / 2 > 1 ? na / 2 : 1;
        L = (na + p - 1) / p;
        L |= 1;  // odd chunk length: the chunks of one line start in distinct banks
        p = (na + L - 1) / L;
        Lz = na - (p - 1) * L;
        if (p > 1 && Lz < 2) {
            --p;
            Lz += L;
        }
        P = p;
        if (P == 1) L = 0;
    }
    // LU factors (c: super-diagonal of U scaled, piv: 1 / pivot) and the
    // responses alpha, beta of tridiag(o, dg, o) of length m
    __device__ static void chunk_factors(T o, T dg, int m, T *c, T *piv, T *al, T *be)
    {
        T cprev = T(0);
        for (int k = 0; k < m; ++k) {
            piv[k] = T(1) / (dg - o * cprev);
            cprev = o * piv[k];
            c[k] = cprev;
        }
        // alpha: right-hand side o e_first; beta: o e_last
        T y = o * piv[0];
        al[0] = y;
        for (int k = 1; k < m; ++k) {
            y = (-o * y) * piv[k];
            al[k] = y;
        }
        for (int k = m - 2; k >= 0; --k) al[k] -= c[k] * al[k + 1];
        T z = o * piv[m - 1];
        be[m - 1] = z;
        for (int k = m - 2; k >= 0; --k) {
            z = -c[k] * z;
            be[k] = z;
        }
    }
    // one thread: every factor (the caller orders it with a barrier)
    __device__ void setup(T *buf, T o, T dg)
    {
        f = buf;
        off = o;
        T *F = buf;
        chunk_factors(o, dg, Lz, F, F + Lz, F + 2 * Lz, F + 3 * Lz);
        if (P > 1) {
            chunk_factors(o, dg, L, F + 4 * Lz, F + 4 * Lz + L, F + 4 * Lz + 2 * L, F + 4 * Lz + 3 * L);
            T *ps = F + 4 * Lz + 4 * L, *nv = ps + P, *dn = nv + P;
            T nu_prev = T(0);
            for (int q = 0; q < P; ++q) {
                const bool last = q == P - 1;
                const int m = last ? Lz : L;
                const T *al = last ? F + 2 * Lz : F + 4 * Lz + 2 * L;
                const T *be = last ? F + 3 * Lz : F + 4 * Lz + 3 * L;
                const T d = T(1) / (T(1) - al[0] * nu_prev);
                dn[q] = d;
                ps[q] = be[0] * d;
                nv[q] = be[m - 1] + al[m - 1] * nu_prev * ps[q];
                nu_prev = nv[q];
            }
        }
    }
    __device__ __forceinline__ int node(int l, int k) const
    {
        const int hi = l / Sa, lo = l - hi * Sa;
        return hi * Sa * Na + lo + k * Sa;
    }
    // all threads of the block; u complete after the caller's next barrier
    __device__ void operator()(const T *r, T *u) const
    {
        const int tid = threadIdx.x, nt = blockDim.x;
        // phase 1: chunk solves g (into u)
        for (int t = tid; t < nlines * P; t += nt) {
            const int q = t / nlines, l = t - q * nlines;  // neighbouring threads: neighbouring lines
            const bool last = q == P - 1;
            const int m = last ? Lz : L, k0 = q * L;
            const T *c = last ? cz() : cf(), *pv = last ? pz() : pf();
            const int j0 = node(l, k0);
            T y = r[j0] * pv[0];
            u[j0] = y;
            for (int k = 1; k < m; ++k) {
                const int j = j0 + k * Sa;
                y = (r[j] - off * y) * pv[k];
                u[j] = y;
            }
            for (int k = m - 2; k >= 0; --k) {
                const int j = j0 + k * Sa;
                y = u[j] - c[k] * y;
                u[j] = y;
            }
        }
        if (P == 1) return;
        __syncthreads();
        // phase 2: chunk boundary values, one thread per line
        for (int l = tid; l < nlines; l += nt) {
            const T *ps = psi(), *nv = nu(), *dn = den();
            T mu = T(0), nu_prev = T(0);
            for (int q = 0; q < P; ++q) {
                const bool last = q == P - 1;
                const int m = last ? Lz : L;
                const T *al = last ? az() : af();
                const int js = node(l, q * L), je = js + (m - 1) * Sa;
                const T phi = (u[js] - al[0] * mu) * dn[q];
                mu = u[je] - al[m - 1] * (mu - nu_prev * phi);
                u[js] = phi;
                u[je] = mu;
                nu_prev = nv[q];
            }
            T F = T(0);  // first value of chunk q + 1
            for (int q = P - 1; q >= 0; --q) {
                const int m = q == P - 1 ? Lz : L;
                const int js = node(l, q * L), je = js + (m - 1) * Sa;
                const T E = u[je] - nv[q] * F;
                F = u[js] - ps[q] * F;
                u[je] = E;
                u[js] = F;
            }
        }
        __syncthreads();
        // phase 3: interior nodes from the neighbouring chunks' boundary values
        for (int t = tid; t < nlines * P; t += nt) {
            const int q = t / nlines, l = t - q * nlines;  // neighbouring threads: neighbouring lines
            const bool last = q == P - 1;
            const int m = last ? Lz : L;
            const T *al = last ? az() : af(), *be = last ? bz() : bf();
            const int j0 = node(l, q * L);
            const T xl = q > 0 ? u[j0 - Sa] : T(0);
            const T xr = last ? T(0) : u[j0 + m * Sa];
            for (int k = 1; k < m - 1; ++k) {
                const int j = j0 + k * Sa;
                u[j] -= al[k] * xl + be[k] * xr;
            }
        }
    }
};

// Preconditioned CG (the Chronopoulos-Gear recurrences with u = M^{-1} r):
// per iteration the update pass sums (r,r) (reduction, convergence test),
// then M, then the stencil pass sums (r,u) and (Au,u) (second reduction); a
// converged iteration skips M and the stencil.  Stops when (r,r) <= stop2
// (unpreconditioned norm, the same test as cg_core).
template <typename T, typename TX, class ST, class PC>
__device__ int pcg_core(const ST &A, const PC &M, int n, TX *X, T *r, T *u, T *p, T *s, T *w, Reducer<T> &R,
                        T stop2, int maxit, int &status)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    status = PIT_OK;
    __syncthreads();  // r complete
    M(r, u);
    __syncthreads();  // u complete
    T v[3] = {T(0), T(0), T(0)};
#pragma unroll 4
    for (int j = tid; j < n; j += nt) {
        const T wj = A(u, j);
        w[j] = wj;
        const T rj = r[j], uj = u[j];
        v[0] += rj * rj;
        v[1] += rj * uj;
        v[2] += wj * uj;
    }
    R.template sum<3>(v);
    if (!(v[0] > stop2)) {
        if (v[0] != v[0]) status = PIT_ERR_NONFINITE;
        return 0;
    }
    if (!finite_pos(v[1]) || !finite_pos(v[2])) {
        status = (v[1] != v[1] || v[2] != v[2]) ? PIT_ERR_NONFINITE : PIT_ERR_BREAKDOWN;
        return 0;
    }
    T gam = v[1], alpha = v[1] / v[2], beta = T(0);
    bool first = true;
    int k = 0;
    for (;;) {
        if (k >= maxit) { status = PIT_ERR_NOCONV; break; }
        // (r, r) of the new residual is summed in the update pass and tested
        // before the preconditioner: the converged last iteration skips M and A
        T rr[1] = {T(0)};
#pragma unroll 4
        for (int j = tid; j < n; j += nt) {
            const T pj = first ? u[j] : u[j] + beta * p[j];
            const T sj = first ? w[j] : w[j] + beta * s[j];
            p[j] = pj;
            s[j] = sj;
            X[j] += (TX)(alpha * pj);
            const T rj = r[j] - alpha * sj;
            r[j] = rj;
            rr[0] += rj * rj;
        }
        first = false;
        ++k;
        R.template sum<1>(rr);  // also: r complete
        if (!(rr[0] > stop2)) {
            if (rr[0] != rr[0]) status = PIT_ERR_NONFINITE;
            break;
        }
        M(r, u);
        __syncthreads();  // u complete
        T q[2] = {T(0), T(0)};
#pragma unroll 4
        for (int j = tid; j < n; j += nt) {
            const T wj = A(u, j);
            w[j] = wj;
            const T uj = u[j];
            q[0] += r[j] * uj;
            q[1] += wj * uj;
        }
        R.template sum<2>(q);
        if (!finite_pos(q[0])) { status = (q[0] != q[0]) ? PIT_ERR_NONFINITE : PIT_ERR_BREAKDOWN; break; }
        beta = q[0] / gam;
        const T den = q[1] - beta * q[0] / alpha;
        if (!finite_pos(den)) { status = (den != den) ? PIT_ERR_NONFINITE : PIT_ERR_BREAKDOWN; break; }
        alpha = q[0] / den;
        gam = q[0];
    }
    return k;
}

// BiCGStab (van der Vorst 1992) on A e = r0: r holds r0 on entry; rh, p, v
// are initialised here; s shares r's storage.  A (near-)breakdown (the shadow
// residual rh almost orthogonal to r, (rh, A p) = 0, omega = 0, or a step
// coefficient beyond 1e30) restarts the method from the current iterate with
// rh = r, provided an iteration has completed since the last restart (so the
// solve still ends within maxit iterations); a second breakdown without
// progress is reported.  Strongly non-normal systems (the central drift flux
// at large dt |v| / h) lose the shadow residual's orthogonality every few
// tens of iterations and need this.
template <typename T, typename TX, class ST>
__device__ int bicgstab_core(const ST &A, int n, TX *X, T *r, T *rh, T *p, T *v, T *t, Reducer<T> &R, T stop2,
                             int maxit, int &status)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    // cosine below which (rh, r) counts as a breakdown
    const T near0 = sizeof(T) == 8 ? T(1e-12) : T(1e-6);
    T rr[1] = {T(0)};
#pragma unroll 4
    for (int j = tid; j < n; j += nt) {
        const T rj = r[j];
        rh[j] = rj;
        p[j] = T(0);
        v[j] = T(0);
        rr[0] += rj * rj;
    }
    R.template sum<1>(rr);
    T rho = T(1), alpha = T(1), omega = T(1), rrv = rr[0], rhh = rr[0];
    int k = 0, k_restart = -1;
    status = PIT_OK;
    // restart from the current residual (every thread reads and writes only
    // its own nodes here; the next use of p behind a barrier is A(p, j))
    auto restart = [&]() -> bool {
        if (k == k_restart) return false;
        k_restart = k;
        for (int j = tid; j < n; j += nt) {
            rh[j] = r[j];
            p[j] = T(0);
            v[j] = T(0);
        }
        rho = alpha = omega = T(1);
        rhh = rrv;
        return true;
    };
    for (;;) {
        if (!(rrv > stop2)) {
            if (rrv != rrv) status = PIT_ERR_NONFINITE;
            break;
        }
        if (k >= maxit) { status = PIT_ERR_NOCONV; break; }
        T rho_n[1] = {T(0)};
#pragma unroll 4
        for (int j = tid; j < n; j += nt) rho_n[0] += rh[j] * r[j];
        R.template sum<1>(rho_n);
        if (rho_n[0] != rho_n[0]) { status = PIT_ERR_NONFINITE; break; }
        if (!(fabs(rho_n[0]) > near0 * sqrt(rrv) * sqrt(rhh))) {
            if (restart()) continue;
            status = PIT_ERR_BREAKDOWN;
            break;
        }
        const T beta = (rho_n[0] / rho) * (alpha / omega);
        if (beta != beta) { status = PIT_ERR_NONFINITE; break; }
        if (!(fabs(beta) < (T)1e30)) {
            if (restart()) continue;
            status = PIT_ERR_BREAKDOWN;
            break;
        }
#pragma unroll 4
        for (int j = tid; j < n; j += nt) p[j] = r[j] + beta * (p[j] - omega * v[j]);
        __syncthreads();
        T rhv[1] = {T(0)};
#pragma unroll 4
        for (int j = tid; j < n; j += nt) {
            const T vj = A(p, j);
            v[j] = vj;
            rhv[0] += rh[j] * vj;
        }
        R.template sum<1>(rhv);
        if (rhv[0] != rhv[0]) { status = PIT_ERR_NONFINITE; break; }
        alpha = rho_n[0] / rhv[0];
        if (!(fabs(alpha) < (T)1e30)) {
            if (restart()) continue;
            status = PIT_ERR_BREAKDOWN;
            break;
        }
#pragma unroll 4
        for (int j = tid; j < n; j += nt) r[j] = r[j] - alpha * v[j];  // s
        __syncthreads();
        T tt[2] = {T(0), T(0)};
#pragma unroll 4
        for (int j = tid; j < n; j += nt) {
            const T tj = A(r, j);
            t[j] = tj;
            tt[0] += tj * tj;
            tt[1] += tj * r[j];
        }
        R.template sum<2>(tt);
        omega = (tt[0] > T(0)) ? tt[1] / tt[0] : T(0);
        if (omega != omega) { status = PIT_ERR_NONFINITE; break; }
        if (!(fabs(omega) < (T)1e30)) omega = T(0);  // take the BiCG half step only
        T rn[1] = {T(0)};
#pragma unroll 4
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
        if (omega == T(0) && rrv > stop2) {
            if (rrv != rrv) { status = PIT_ERR_NONFINITE; break; }
            if (restart()) continue;
            status = PIT_ERR_BREAKDOWN;
            break;
        }
    }
    return k;
}

// ----------------------------------------------------------------------------
// Shared-memory layout of one item (ld = n rounded up to 4):
//   FP64 arrays: x, [b (MIXED)], [Krylov vectors (PLAIN)], [table (var. coef.,
//                PLAIN and MIXED)]
//   FP32 arrays: [e (MIXED) or x (SINGLE), Krylov vectors, table (var. coef.)]
//   u16 mask
__host__ __device__ inline bool line_pc_form(int op, int prec, bool xg)
{
    return op == PIT_OP_HEAT && prec != PLAIN && !xg;
}
__host__ __device__ inline int krylov_vecs(int op, int prec, bool xg = false)
{
    if (op == PIT_OP_OU || op == PIT_OP_LSDE || op == PIT_OP_CME) return prec == PLAIN ? 5 : 6;  // r rh p v t (+ e or x)
    if (line_pc_form(op, prec, xg)) return 6;           // r p s w u (+ e or x): u for the line preconditioner
    return prec == PLAIN ? 4 : 5;                        // r p s w (+ e or x)
}
// bytes after the mask: the line preconditioner's factors, 2 N_a floats
// (N_a = nodes of the grid's longest axis, an upper bound for the finest one)
__host__ __device__ inline int line_pc_bytes(int op, int prec, bool xg, int na)
{
    return line_pc_form(op, prec, xg) ? 4 * (6 * na + 3 * 33 + 8) + 16 : 0;
}

__host__ __device__ inline int n_tab(int op, int d) { return op == PIT_OP_HEAT ? 0 : 2 * d + 1; }
// (MIXED keeps a third FP64 array, the carried x - A x of the last step;
// its global-state variant keeps it in global memory with x and b)
__host__ __device__ inline int n_f64(int op, int prec, int d)
{
    if (prec == SINGLE) return 0;
    return (prec == PLAIN ? 1 + krylov_vecs(op, prec) : prec == MIXED ? 3 : 2) + n_tab(op, d);
}
__host__ __device__ inline int n_f32(int op, int prec, int d, bool xg = false)
{
    if (prec == PLAIN) return 0;
    return krylov_vecs(op, prec, xg) + n_tab(op, d);
}

template <int OP, int PREC, int D, bool XG = false>
__global__ void __launch_bounds__(512, 1) steps_kernel(StepArgs a)
{
    typedef typename std::conditional<PREC == PLAIN, double, float>::type T;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ GridInfo GI;
    __shared__ double red64[2 * 128];
    __shared__ float red32[2 * 128];

    static_assert(!XG || PREC != SINGLE, "no global-state variant of the FP32 form");
    static_assert(PREC == PLAIN || PREC == MIXED || PREC == SINGLE || PREC == PAIR, "unknown precision form");
    static_assert(PREC != PAIR || (OP != PIT_OP_OU && OP != PIT_OP_LSDE && OP != PIT_OP_CME),
                  "the pair form is for the symmetric operators");
    constexpr bool DRIFT = (OP == PIT_OP_OU || OP == PIT_OP_LSDE || OP == PIT_OP_CME);  // non-symmetric: BiCGStab
    constexpr bool CROSS = (OP == PIT_OP_LSDE);                      // mixed-derivative terms
    const int item = a.item0 + (int)blockIdx.x;
    const int g = a.order[item / a.n_batch];
    const int b = item % a.n_batch;
    if (a.active && !a.active[g]) return;  // uniform over the block
    if (threadIdx.x == 0) GI = a.grids[g];
    __syncthreads();

    const int tid = threadIdx.x, nt = blockDim.x;
    const int n = GI.n;
    const int ld = (n + 3) & ~3;
    const double dt = a.dt;
    constexpr int K = (OP == PIT_OP_HEAT) ? 0 : 2 * D + 1;
    // the FP64 global-state variant keeps the coefficient table in global
    // memory too (grids of any size); the others keep it on chip
    constexpr bool GTAB = XG && PREC == PLAIN && K > 0;
    constexpr int NF64 = PREC == SINGLE ? 0 : (XG ? 0 : PREC == PLAIN ? 1 + (DRIFT ? 5 : 4) : PREC == MIXED ? 3 : 2) + (GTAB ? 0 : K);
    constexpr int NKV = DRIFT ? (PREC == PLAIN ? 5 : 6)
                                          : (PREC == PLAIN ? 4 : (OP == PIT_OP_HEAT && !XG ? 6 : 5));
    constexpr int NF32 = (PREC != PLAIN) ? NKV + K : 0;

    double *s64 = reinterpret_cast<double *>(smem);
    double *x = XG ? a.xg + (long long)b * a.n_total + GI.off : s64;
    double *bvec = XG ? a.bg + (long long)b * a.n_total + GI.off : s64 + ld;  // MIXED: right-hand side
    // PAIR: the state and the right-hand side as FP32 pairs, in the places of x and bvec
    float2 *xp = reinterpret_cast<float2 *>(x), *bp = reinterpret_cast<float2 *>(bvec);
    // PLAIN: Krylov vectors, in shared memory (stride ld) or, for the
    // global-state variant, in per-vector slabs of n_batch x n_total after x
    double *v64 = XG ? a.xg + ((long long)a.n_batch + b) * a.n_total + GI.off : s64 + ld;
    const long long vs = XG ? (long long)a.n_batch * a.n_total : (long long)ld;
    // GTAB: table entry k of the item in slab (1 + NKV + k) n_batch + b after
    // the Krylov vectors, at the grid's offset (every array of the global
    // workspace is partitioned by grid, so launches of different lanes and
    // batch widths that run concurrently on disjoint grids never overlap)
    double *tab64 = PREC == SINGLE ? nullptr
                    : GTAB ? a.xg + ((long long)(1 + NKV) * a.n_batch + b) * a.n_total + GI.off
                           : s64 + (size_t)(NF64 - (GTAB ? 0 : K)) * ld;
    // stride between the table's entries (the host keeps n_batch n_total below 2^31 here)
    const int tld = GTAB ? (int)((long long)a.n_batch * a.n_total) : ld;
    float *f32 = reinterpret_cast<float *>(s64 + (size_t)NF64 * ld);
    float *tab32 = f32 + (size_t)NKV * ld;
    uint16_t *mask = reinterpret_cast<uint16_t *>(f32 + (size_t)NF32 * ld);

    const double *in = a.in + (long long)b * a.in_stride + GI.off;
    const double *f0 = a.f ? a.f + (long long)b * a.f_stride + GI.off : nullptr;
    const uint16_t *gmask = a.masks + GI.off;

    Reducer<double> R64{red64, 0};
    Reducer<float> R32{red32, 0};
    // SINGLE: the state is held as x 2^ks in FP32 (PAIR: as FP32 pairs), ks
    // from the input state and the first forcing term (the correction sweep of
    // MGRIT starts from zero)
    int ks = 0;
    if constexpr (PREC == SINGLE || PREC == PAIR) {
        const double *g0 = a.g ? a.g + (long long)b * a.g_stride + GI.off : nullptr;
        double acc[1] = {0.0};
        for (int j = tid; j < n; j += nt) {
            const double v = in[j];
            acc[0] += v * v;
            if (g0) acc[0] += g0[j] * g0[j];
        }
        R64.template sum<1>(acc);
        ks = scale_exp(acc[0]);
    }
    for (int j = tid; j < n; j += nt) {
        mask[j] = gmask[j];
        if constexpr (PREC == SINGLE) f32[j] = to_f32(in[j], ks);
        else if constexpr (PREC == PAIR) xp[j] = split_pair(in[j], ks);
        else x[j] = in[j];
    }
    if constexpr (OP != PIT_OP_HEAT) {
        for (int j = tid; j < n; j += nt) {
            double diag, cm[D], cp[D];
            op_coef<D>(a.op, GI, a.faces, j, dt, diag, cm, cp);
            if constexpr (PREC != SINGLE && PREC != PAIR) tab64[j] = diag;
            if constexpr (PREC != PLAIN) tab32[j] = (float)diag;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                if constexpr (PREC != SINGLE && PREC != PAIR) {
                    tab64[(1 + 2 * i) * tld + j] = cm[i];
                    tab64[(2 + 2 * i) * tld + j] = cp[i];
                }
                if constexpr (PREC == PAIR) {
                    // face coefficients dt a / h^2 as pairs, in the FP64 table's place
                    float2 *cpair = reinterpret_cast<float2 *>(tab64);
                    const double ih2 = 1.0 / (GI.h[i] * GI.h[i]);
                    const double am = a.faces[(GI.off + j) * (2 * D) + 2 * i];
                    const double ap = a.faces[(GI.off + j) * (2 * D) + 2 * i + 1];
                    cpair[(2 * i) * ld + j] = split_pair(dt * am * ih2, 0);
                    cpair[(2 * i + 1) * ld + j] = split_pair(dt * ap * ih2, 0);
                }
                if constexpr (PREC != PLAIN) {
                    tab32[(1 + 2 * i) * ld + j] = (float)cm[i];
                    tab32[(2 + 2 * i) * ld + j] = (float)cp[i];
                }
            }
        }
    }
    // stencils in FP64 and in the working precision
    HeatSt<double, D> H64;
    HeatSt<T, D> HT;
    TabSt<double, D, CROSS> T64;
    TabSt<float, D, CROSS> T32;
    H64.mask = HT.mask = T64.mask = T32.mask = mask;
    T64.tab = tab64;
    T32.tab = tab32;
    T64.ld = tld;
    T32.ld = ld;
    if constexpr (CROSS) {
        int q = 0;
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int k = i + 1; k < D; ++k, ++q) {
                const double c = -dt * 0.5 * (a.op.H[i * D + k] + a.op.H[k * D + i]) / (4.0 * GI.h[i] * GI.h[k]);
                T64.cr[q] = c;
                T32.cr[q] = (float)c;
            }
    }
    {
        double diag = 1.0;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const double ih2 = 1.0 / (GI.h[i] * GI.h[i]);
            H64.S[i] = HT.S[i] = T64.S[i] = T32.S[i] = GI.S[i];
            H64.off[i] = -dt * ih2;
            HT.off[i] = (T)(-dt * ih2);
            diag += 2.0 * dt * ih2;
        }
        H64.diag = diag;
        HT.diag = (T)diag;
    }
    // Jacobi preconditioning of the FP32 correction solves (table operators
    // without mixed-derivative terms, refinement forms): the FP32 system is
    // scaled symmetrically, D^{-1/2} A D^{-1/2} y = D^{-1/2} r, e = D^{-1/2} y,
    // D = diag(A): its off-diagonal entries become a_jk / sqrt(d_j d_k) and
    // its diagonal one, whose slot then keeps D^{-1/2} (T32.unit)
    bool jac = false;
    if constexpr ((PREC == MIXED || PREC == PAIR) && (OP == PIT_OP_VARHEAT || OP == PIT_OP_OU)) {
        if (a.precond == PIT_PRECOND_JACOBI && !a.ext) {  // (the extrapolated steps rescale the table)
            jac = true;
            __syncthreads();  // table complete
            for (int j = tid; j < n; j += nt) {
                const unsigned mk = mask[j];
                const float dj = tab32[j];
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    if ((mk >> (2 * i)) & 1u) tab32[(1 + 2 * i) * ld + j] *= rsqrtf(dj * tab32[j - GI.S[i]]);
                    if ((mk >> (2 * i + 1)) & 1u) tab32[(2 + 2 * i) * ld + j] *= rsqrtf(dj * tab32[j + GI.S[i]]);
                }
            }
            __syncthreads();  // every off-diagonal scaled with the old diagonals
            for (int j = tid; j < n; j += nt) tab32[j] = rsqrtf(tab32[j]);
            T32.unit = true;
        }
    }
    PairTab<D> PT;
    if constexpr (PREC == PAIR && OP != PIT_OP_HEAT) {
        PT.mask = mask;
        PT.c = reinterpret_cast<const float2 *>(tab64);
        PT.ld = ld;
#pragma unroll
        for (int i = 0; i < D; ++i) PT.S[i] = GI.S[i];
    }
    PairHeat<D> PH;
    if constexpr (PREC == PAIR && OP == PIT_OP_HEAT) {
        PH.mask = mask;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const double c = dt / (GI.h[i] * GI.h[i]);
            PH.S[i] = GI.S[i];
            PH.ch[i] = to_f32(c, 0);
            PH.cl[i] = to_f32(c - to_f64(PH.ch[i], 0), 0);
        }
    }
    // Line preconditioner (heat, FP32 Krylov, state on chip) along the finest
    // axis a, used when a is at least twice as fine as every other axis and
    // stiff at this step size (4 dt / h_a^2 >= 2); measured faster on the
    // heat workloads than a stricter rule (condition-number ratio >= 16).
    // Its factors are computed once per launch; the barrier at the top of the
    // step loop orders them.  (With the variable coefficient, the constant-
    // coefficient line matrix as preconditioner measured slower than plain CG.)
    bool use_pc = false;
    LineM<float> LM{};
    if constexpr (OP == PIT_OP_HEAT && PREC != PLAIN && !XG) {
        // (every per-axis value is read with a compile-time index, so that
        // the grid description and the stencil stay in registers)
        int ax = 0, Na = 0, Sa = 0;
        double ha = 1e300;
        float offa = 0.0f;
#pragma unroll
        for (int i = 0; i < D; ++i)
            if (GI.h[i] < ha) {
                ax = i;
                ha = GI.h[i];
                Na = GI.N[i];
                Sa = GI.S[i];
                offa = HT.off[i];
            }
        double h2 = 1e300;
#pragma unroll
        for (int i = 0; i < D; ++i)
            if (i != ax && GI.h[i] < h2) h2 = GI.h[i];
        use_pc = a.precond != PIT_PRECOND_NONE && Na >= 3 && 2.0 * ha <= h2 * (1.0 + 1e-12) &&
                 4.0 * dt / (ha * ha) >= 2.0;
        if (use_pc) {
            float *lf = reinterpret_cast<float *>(mask + ld);
            LM.layout(Na, Sa, n, nt);
            LM.f = lf;
            LM.off = offa;
            if (tid == 0) LM.setup(lf, offa, HT.diag);
        }
    }
    auto A64 = [&](const double *v, int j) -> double {
        if constexpr (OP == PIT_OP_HEAT) return H64(v, j);
        else return T64(v, j);
    };
    auto RES64 = [&](double bj, const double *v, int j) -> double {  // b_j - (A v)_j
        if constexpr (OP == PIT_OP_HEAT) return H64.resid(bj, v, j);
        else return T64.resid(bj, v, j);
    };

    // Full step of an extrapolated backward-Euler step for the table-driven
    // variable-coefficient operator: the table of I + dt L becomes that of
    // I + 2 dt L in place (off-diagonal entries doubled, diagonal 2 d - 1,
    // both exact in binary floating point for d >= 1) and back (halved,
    // (d + 1) / 2, exact again); barriers on both sides, since every thread's
    // stencil reads its neighbours' entries.
    auto table_full_step = [&](bool full) {
        if constexpr (OP == PIT_OP_VARHEAT && PREC != PAIR) {
            __syncthreads();
            for (int j = tid; j < n; j += nt) {
                if constexpr (PREC != SINGLE) {
                    tab64[j] = full ? 2.0 * tab64[j] - 1.0 : 0.5 * (tab64[j] + 1.0);
#pragma unroll
                    for (int k = 1; k <= 2 * D; ++k) tab64[k * tld + j] *= full ? 2.0 : 0.5;
                }
                if constexpr (PREC != PLAIN) {
                    tab32[j] = full ? 2.0f * tab32[j] - 1.0f : 0.5f * (tab32[j] + 1.0f);
#pragma unroll
                    for (int k = 1; k <= 2 * D; ++k) tab32[k * ld + j] *= full ? 2.0f : 0.5f;
                }
            }
            __syncthreads();
        }
    };
    int status = PIT_OK, iters = 0, passes = 0;
    const bool carry_ok = (f0 == nullptr) && (a.g == nullptr) && (a.guess == nullptr) && !a.sdirk && !a.ext;
    // MIXED also carries its residual across an additive forcing g (x_s <- x_s
    // + g_s after the solve): with b_{s+1} = x_s + g_s and the guess x_s (the
    // solve's result before g), r0 = b_{s+1} - A x_s = r_s + (x_s + g_s - b_s),
    // again without a stencil pass (no extrapolation then)
    const bool carry_g = (f0 == nullptr) && (a.guess == nullptr) && !a.sdirk && !a.ext;
    // Two-stage SDIRK steps (a.sdirk, coarse propagators; dt is the stage
    // step gamma dT, gamma = 1 - 1/sqrt 2): stage 1 solves (I + dt L) U1 = u_n,
    // stage 2 (I + dt L) U2 = (1 - beta) u_n + beta U1 with beta =
    // (1 - gamma) / gamma = 1 + sqrt 2, and u_{n+1} = U2 (L-stable, second
    // order; see the MGRIT options of the interface)
    // Extrapolated backward-Euler steps (a.ext, coarse propagators, MIXED
    // heat; dt is the half step dT/2): U1 and U2 by two half steps from u_n,
    // U3 by one full step (I + 2 dt L) U3 = u_n, u_{n+1} = 2 U2 - U3; u_n and
    // then U2 wait in the carried-residual array, which these steps leave
    // unused.
    const int nstage = a.sdirk ? 2 : a.ext ? 3 : 1;
    constexpr double SD_BETA = 2.4142135623730950488, SD_ALPHA = -1.4142135623730950488;
    // MIXED: carried initial residual of the next step (see the file comment).
    // FP32 copies of FP64 vectors are scaled by a power of two 2^k chosen from
    // ||b|| (exact, folded into the conversion), so they stay inside the normal
    // FP32 range for states of any magnitude.
    bool have_r0 = false;
    double rn0_c = 0.0, bb_c = 0.0;
    int kr_c = 0;
    float *rv = f32 + ld, *pv = f32 + 2 * ld, *sv = f32 + 3 * ld, *wv = f32 + 4 * ld, *tv = f32 + 5 * ld;
    // MIXED: c = x_s - A x_s of the last completed step, in FP64 (the next
    // step's initial residual for the guess x_s, and with the one before it
    // the residual of the extrapolated guess); have_c: c holds c_{s-1} at the
    // start of step s + 1
    double *cvec = XG ? a.xg + ((long long)2 * a.n_batch + b) * a.n_total + GI.off : s64 + 2 * ld;
    bool have_c = false;

    for (int step = 1; step <= a.nsteps; ++step) {
        // forcing of this step: f_div consecutive steps share one forcing vector
        const double *f = f0 ? f0 + (long long)((step - 1) / a.f_div) * a.f_step : nullptr;
        __syncthreads();  // state complete
        if constexpr (PREC == PLAIN) {
            double *r = v64, *q1 = v64 + vs, *q2 = v64 + 2 * vs, *q3 = v64 + 3 * vs, *q4 = v64 + 4 * vs;
            double bb[1] = {0.0};
            if (a.guess) {
                // right-hand side kept in r, iterate replaced by the guess
                const long long sb0 = (long long)(step - 1);
                const double *gu = a.guess + (long long)b * a.guess_stride + sb0 * a.guess_step + GI.off;
                const double *gf = a.g ? a.g + (long long)b * a.g_stride + sb0 * a.g_step + GI.off : nullptr;
                for (int j = tid; j < n; j += nt) {
                    const double bj = f ? x[j] + dt * f[j] : x[j];
                    r[j] = bj;
                    bb[0] += bj * bj;
                    x[j] = gf ? gu[j] - gf[j] : gu[j];
                }
                __syncthreads();
                for (int j = tid; j < n; j += nt) r[j] -= A64(x, j);
            } else {
                for (int j = tid; j < n; j += nt) {
                    const double bj = f ? x[j] + dt * f[j] : x[j];
                    r[j] = RES64(bj, x, j);
                    bb[0] += bj * bj;
                }
            }
            R64.template sum<1>(bb);  // also orders the residual before x changes
            ++passes;
            const double stop2 = a.rtol * a.rtol * bb[0];
            int st, k;
            if constexpr (DRIFT) k = bicgstab_core<double, double>(T64, n, x, r, q1, q2, q3, q4, R64, stop2, a.maxit, st);
            else if constexpr (OP == PIT_OP_HEAT) k = cg_core<double, double>(H64, n, x, r, q1, q2, q3, R64, stop2, a.maxit, st);
            else k = cg_core<double, double>(T64, n, x, r, q1, q2, q3, R64, stop2, a.maxit, st);
            iters += k;
            if (st > status) status = st;
        } else if constexpr (PREC == SINGLE) {
            // FP32 Krylov on the scaled FP32 state xs = x 2^ks
            float *xs = f32, *r = f32 + ld, *q1 = f32 + 2 * ld, *q2 = f32 + 3 * ld, *q3 = f32 + 4 * ld,
                  *q4 = f32 + 5 * ld;
            const float dtf = (float)dt;
            // extrapolated steps: u_n, then U2, wait in the item's global scratch
            float *scr = a.scr ? a.scr + (long long)b * a.n_total + GI.off : nullptr;
            const bool use_pc0 = use_pc;
            const T diagTh = HT.diag;
#pragma unroll 1
          for (int stage = 0; stage < nstage; ++stage) {
            if (a.ext && stage == 2) table_full_step(true);
            if constexpr (OP == PIT_OP_HEAT) {
                if (a.ext && stage == 2) {
                    // the full step I + 2 dt L, without the line preconditioner
#pragma unroll
                    for (int i = 0; i < D; ++i) HT.off[i] *= (T)2;
                    HT.diag = (T)(2.0 * H64.diag - 1.0);
                    use_pc = false;
                }
            }
            float bb[1] = {0.0f};
            if (stage == 1 && a.ext) {
                // second half step from U1 (in xs): b = U1
                for (int j = tid; j < n; j += nt) {
                    float Ax;
                    if constexpr (OP == PIT_OP_HEAT) Ax = HT(xs, j);
                    else Ax = T32(xs, j);
                    const float xj = xs[j];
                    r[j] = xj - Ax;
                    bb[0] += xj * xj;
                }
            } else if (stage == 2) {
                // full step from u_n, started from U2, which takes u_n's place
                for (int j = tid; j < n; j += nt) {
                    float Ax;
                    if constexpr (OP == PIT_OP_HEAT) Ax = HT(xs, j);
                    else Ax = T32(xs, j);
                    const float un = scr[j];
                    scr[j] = xs[j];
                    r[j] = un - Ax;
                    bb[0] += un * un;
                }
            } else if (stage == 1) {
                // second stage: b = (1 - beta) u_n + beta U1 with u_n = A U1
                // (the first stage's equation, met to its tolerance), so
                // b = beta U1 - sqrt 2 A U1 from U1 (in xs) alone, and
                // r = b - A U1 = beta (U1 - A U1)
                for (int j = tid; j < n; j += nt) {
                    float Ax;
                    if constexpr (OP == PIT_OP_HEAT) Ax = HT(xs, j);
                    else Ax = T32(xs, j);
                    const float xj = xs[j];
                    const float bj = (float)SD_BETA * xj + (float)SD_ALPHA * Ax;
                    r[j] = (float)SD_BETA * (xj - Ax);
                    bb[0] += bj * bj;
                }
            } else if (a.guess) {
                const long long sb0 = (long long)(step - 1);
                const double *gu = a.guess + (long long)b * a.guess_stride + sb0 * a.guess_step + GI.off;
                const double *gf = a.g ? a.g + (long long)b * a.g_stride + sb0 * a.g_step + GI.off : nullptr;
                for (int j = tid; j < n; j += nt) {
                    const float bj = f ? xs[j] + dtf * to_f32(f[j], ks) : xs[j];
                    r[j] = bj;
                    if (a.ext) scr[j] = bj;
                    bb[0] += bj * bj;
                    xs[j] = to_f32(gf ? gu[j] - gf[j] : gu[j], ks);
                }
                __syncthreads();
                for (int j = tid; j < n; j += nt) {
                    if constexpr (OP == PIT_OP_HEAT) r[j] -= HT(xs, j);
                    else r[j] -= T32(xs, j);
                }
            } else {
                for (int j = tid; j < n; j += nt) {
                    const float bj = f ? xs[j] + dtf * to_f32(f[j], ks) : xs[j];
                    float Ax;
                    if constexpr (OP == PIT_OP_HEAT) Ax = HT(xs, j);
                    else Ax = T32(xs, j);
                    r[j] = bj - Ax;
                    if (a.ext) scr[j] = bj;
                    bb[0] += bj * bj;
                }
            }
            R32.template sum<1>(bb);  // also orders the residual before xs changes
            if (bb[0] > 0.0f && !(bb[0] >= 0x1p-60f && bb[0] <= 0x1p60f)) {
                // keep the FP32 state near unit size (the sweep's state can
                // start at zero and grow or fade by many orders): exact
                // power-of-two rescale of the linear quantities xs, r and of ks
                const int kq = scale_exp((double)bb[0]);
                const float sc = __uint_as_float((unsigned)(127 + kq) << 23);
                for (int j = tid; j < n; j += nt) {
                    xs[j] *= sc;
                    r[j] *= sc;
                    if (a.ext) scr[j] *= sc;  // u_n or U2, in the same scale
                }
                bb[0] = (bb[0] * sc) * sc;
                ks += kq;
            }
            const float rt = (float)a.rtol;
            const float stop2 = rt * rt * bb[0];
            int st, k;
            if constexpr (DRIFT) k = bicgstab_core<float, float>(T32, n, xs, r, q1, q2, q3, q4, R32, stop2, a.maxit, st);
            else if constexpr (OP == PIT_OP_HEAT) {
                if (use_pc) k = pcg_core<float, float>(HT, LM, n, xs, r, q4, q1, q2, q3, R32, stop2, a.maxit, st);
                else k = cg_core<float, float>(HT, n, xs, r, q1, q2, q3, R32, stop2, a.maxit, st);
            }
            else k = cg_core<float, float>(T32, n, xs, r, q1, q2, q3, R32, stop2, a.maxit, st);
            iters += k;
            if (st > status) status = st;
            __syncthreads();  // xs complete
          }
            if constexpr (OP == PIT_OP_VARHEAT) {
                if (a.ext) {
                    table_full_step(false);
                    for (int j = tid; j < n; j += nt) xs[j] = 2.0f * scr[j] - xs[j];
                }
            }
            if constexpr (OP == PIT_OP_HEAT) {
                if (a.ext) {
                    // back to the half step; u_{n+1} = 2 U2 - U3
#pragma unroll
                    for (int i = 0; i < D; ++i) HT.off[i] *= (T)0.5;
                    HT.diag = diagTh;
                    use_pc = use_pc0;
                    for (int j = tid; j < n; j += nt) xs[j] = 2.0f * scr[j] - xs[j];
                }
            }
            // forcing of this step and the stored outputs (FP64, own nodes only)
            const long long sb = (long long)(step - 1);
            if (a.g) {
                const double *gs = a.g + (long long)b * a.g_stride + sb * a.g_step + GI.off;
                for (int j = tid; j < n; j += nt) xs[j] += to_f32(gs[j], ks);
            }
            const double *hs = a.hs ? a.hs + (long long)b * a.hs_stride + sb * a.hs_step + GI.off : nullptr;
            if (step < a.nsteps) {
                if (a.out_steps) {
                    double *os = a.out_steps + (long long)b * a.os_stride + sb * a.os_step + GI.off;
                    for (int j = tid; j < n; j += nt) {
                        const double xj = to_f64(xs[j], -ks);
                        os[j] = hs ? xj + hs[j] : xj;
                    }
                }
            } else {
                double *ol = a.out_last + (long long)b * a.ol_stride + GI.off;
                const double *h = a.h ? a.h + (long long)b * a.h_stride + GI.off : nullptr;
                const double *cmp = a.cmp ? a.cmp + (long long)b * a.cmp_stride + GI.off : nullptr;
                double acc[1] = {0.0};
                for (int j = tid; j < n; j += nt) {
                    const double xj = to_f64(xs[j], -ks);
                    if (cmp) {
                        const double dlt = xj - cmp[j];
                        acc[0] += dlt * dlt;
                    }
                    ol[j] = a.out_scale * xj + (h ? a.out_hscale * h[j] : 0.0) + (hs ? hs[j] : 0.0);
                }
                if (cmp) {
                    R64.template sum<1>(acc);
                    if (tid == 0) a.norms[(long long)b * a.n_grids + g] = sqrt(acc[0]);
                }
            }
            continue;
        } else if constexpr (PREC == PAIR) {
            // Refinement on FP32 pairs of the state scaled by 2^ks: b - A x
            // from PairHeat (PairTab), the correction equation solved in FP32 as in
            // MIXED, the correction added to the pairs.  The residual copies
            // are in the state's scale (its norm is kept in [2^-10, 2^10]), so
            // no per-step rescaling of them is needed.
            float *e = f32;
            auto PR = [&](int j, float &xmb) -> float {
                if constexpr (OP == PIT_OP_HEAT) return PH(xp, bp, j, xmb);
                else return PT(xp, bp, j, xmb);
            };
            if (a.guess) {
                const long long sb0 = (long long)(step - 1);
                const double *gu = a.guess + (long long)b * a.guess_stride + sb0 * a.guess_step + GI.off;
                const double *gf = a.g ? a.g + (long long)b * a.g_stride + sb0 * a.g_step + GI.off : nullptr;
                for (int j = tid; j < n; j += nt) {
                    bp[j] = f ? pair_add(xp[j], split_pair(dt * f[j], ks)) : xp[j];
                    xp[j] = split_pair(gf ? gu[j] - gf[j] : gu[j], ks);
                }
            } else {
                for (int j = tid; j < n; j += nt) bp[j] = f ? pair_add(xp[j], split_pair(dt * f[j], ks)) : xp[j];
            }
            double rn2, bb;
            if (have_r0 && bb_c >= 0x1p-20 && bb_c <= 0x1p20) {
                // r0 = x_{s-1} - A x_{s-1}, from the last check of the previous step (in wv)
                float *t_ = rv; rv = wv; wv = t_;
                rn2 = rn0_c;
                bb = bb_c;
            } else {
                float acc[1] = {0.0f};
                for (int j = tid; j < n; j += nt) acc[0] += bp[j].x * bp[j].x;
                R32.template sum<1>(acc);  // also: bp and xp complete
                bb = to_f64(acc[0], 0);
                if (bb > 0.0 && !(bb >= 0x1p-20 && bb <= 0x1p20)) {
                    // exact power-of-two rescale of the state (it can fade or
                    // grow by many orders over a long sweep)
                    const int kq = scale_exp(bb);
                    const float sc = __uint_as_float((unsigned)(127 + kq) << 23);
                    for (int j = tid; j < n; j += nt) {
                        const float2 xj = xp[j], bj = bp[j];
                        xp[j] = make_float2(xj.x * sc, xj.y * sc);
                        bp[j] = make_float2(bj.x * sc, bj.y * sc);
                    }
                    bb = bb * pow2d(2 * kq);
                    ks += kq;
                    __syncthreads();
                }
                float accf[1] = {0.0f};
#pragma unroll 4
                for (int j = tid; j < n; j += nt) {
                    float xmb;
                    const float rf = PR(j, xmb);
                    rv[j] = rf;
                    accf[0] += rf * rf;
                }
                R32.template sum<1>(accf);
                ++passes;
                rn2 = to_f64(accf[0], 0);
            }
            have_r0 = false;
            const double stop2 = a.rtol * a.rtol * bb;
            int st_step = PIT_OK;
            bool carried = false;
            for (int pass = 0;; ++pass) {
                if (!(rn2 > stop2)) {
                    if (rn2 != rn2) st_step = PIT_ERR_NONFINITE;
                    else if (carry_ok && pass == 0) {
                        // x unchanged: its residual is the next step's r0
                        float *t_ = rv; rv = wv; wv = t_;
                        rn0_c = rn2;
                        bb_c = bb;
                        carried = true;
                    }
                    break;
                }
                if (pass >= a.ir_maxit) { st_step = PIT_ERR_NOCONV; break; }
                // the correction equation on rv 2^-kn (squared norm in [1, 4))
                const int kn = min(max(-scale_exp(rn2), -120), 120);
                const float inv = __uint_as_float((unsigned)(127 - kn) << 23);  // 2^-kn
                const float R2n = to_f32(rn2, -2 * kn);
                const float want = 0.5f * sqrtf(to_f32(stop2, -2 * kn) / R2n);
                const float tgt = want > a.inner_rtol ? want : (float)a.inner_rtol;
                const float stop32 = tgt * tgt * R2n;
                for (int j = tid; j < n; j += nt) {
                    rv[j] *= jac ? inv * tab32[j] : inv;
                    e[j] = 0.0f;
                }
                int st, k;
                if constexpr (OP == PIT_OP_HEAT) {
                    if (use_pc) k = pcg_core<float, float>(HT, LM, n, e, rv, f32 + 5 * ld, pv, sv, wv, R32, stop32, a.maxit, st);
                    else k = cg_core<float, float>(HT, n, e, rv, pv, sv, wv, R32, stop32, a.maxit, st);
                } else {
                    k = cg_core<float, float>(T32, n, e, rv, pv, sv, wv, R32, stop32, a.maxit, st);
                }
                iters += k;
                if (st == PIT_ERR_NONFINITE) { st_step = st; break; }
                // x += e 2^kn on the pairs (the scaling is exact; Jacobi: e = D^{-1/2} y)
                const float csf = __uint_as_float((unsigned)(127 + kn) << 23);
#pragma unroll 4
                for (int j = tid; j < n; j += nt) xp[j] = pair_add(xp[j], (jac ? e[j] * tab32[j] : e[j]) * csf);
                __syncthreads();  // x complete
                // check: r = b - A x; the next step's r0 = x - A x = r + (x - b)
                float accf[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll 4
                for (int j = tid; j < n; j += nt) {
                    float xmb;
                    const float rf = PR(j, xmb);
                    rv[j] = rf;
                    accf[0] += rf * rf;
                    if (carry_ok) {
                        const float cj = rf + xmb;
                        const float xf = xp[j].x;
                        wv[j] = cj;
                        accf[1] += cj * cj;
                        accf[2] += xf * xf;
                    }
                }
                R32.template sum<3>(accf);
                ++passes;
                rn2 = to_f64(accf[0], 0);
                if (carry_ok) {
                    rn0_c = to_f64(accf[1], 0);
                    bb_c = to_f64(accf[2], 0);
                    carried = true;
                }
            }
            if (st_step > status) status = st_step;
            have_r0 = carried && st_step == PIT_OK && step < a.nsteps;
            // forcing of this step and the stored outputs (FP64, own nodes only)
            const long long sb = (long long)(step - 1);
            if (a.g) {
                const double *gs = a.g + (long long)b * a.g_stride + sb * a.g_step + GI.off;
                for (int j = tid; j < n; j += nt) xp[j] = pair_add(xp[j], split_pair(gs[j], ks));
            }
            const double *hs = a.hs ? a.hs + (long long)b * a.hs_stride + sb * a.hs_step + GI.off : nullptr;
            if (step < a.nsteps) {
                if (a.out_steps) {
                    double *os = a.out_steps + (long long)b * a.os_stride + sb * a.os_step + GI.off;
                    for (int j = tid; j < n; j += nt) {
                        const double xj = pair_to_f64(xp[j], ks);
                        os[j] = hs ? xj + hs[j] : xj;
                    }
                }
            } else {
                double *ol = a.out_last + (long long)b * a.ol_stride + GI.off;
                const double *h = a.h ? a.h + (long long)b * a.h_stride + GI.off : nullptr;
                const double *cmp = a.cmp ? a.cmp + (long long)b * a.cmp_stride + GI.off : nullptr;
                double acc[1] = {0.0};
                for (int j = tid; j < n; j += nt) {
                    const double xj = pair_to_f64(xp[j], ks);
                    if (cmp) {
                        const double dlt = xj - cmp[j];
                        acc[0] += dlt * dlt;
                    }
                    ol[j] = a.out_scale * xj + (h ? a.out_hscale * h[j] : 0.0) + (hs ? hs[j] : 0.0);
                }
                if (cmp) {
                    R64.template sum<1>(acc);
                    if (tid == 0) a.norms[(long long)b * a.n_grids + g] = sqrt(acc[0]);
                }
            }
            continue;
        } else {
            float *e = f32;
            const bool use_pc0 = use_pc;
            const double diag64h = H64.diag;
            const T diagTh = HT.diag;
#pragma unroll 1
          for (int stage = 0; stage < nstage; ++stage) {
            if (a.ext && stage == 2) table_full_step(true);
            if constexpr (OP == PIT_OP_HEAT) {
                if (a.ext && stage == 2) {
                    // the full step: I + 2 dt L (off-diagonal entries doubled
                    // exactly, diagonal 2 diag - 1), without the line
                    // preconditioner, whose factors are those of the half step
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        H64.off[i] *= 2.0;
                        HT.off[i] *= (T)2;
                    }
                    H64.diag = 2.0 * H64.diag - 1.0;
                    HT.diag = (T)H64.diag;
                    use_pc = false;
                }
            }
            double rn2, bb;
            int kr;  // the stored FP32 residual rv holds r 2^kr
            if (have_r0) {
                // Step s + 1 without forcing: b = x_s, and rv holds r_s 2^kr_c,
                // r_s = x_{s-1} - A x_s, the FP64 residual of the last check of
                // step s.  With d = x_s - x_{s-1} (FP64), c_s = x_s - A x_s =
                // r_s + d.  Guess x_s: r0 = c_s.  Extrapolated guess
                // 2 x_s - x_{s-1} = x_s + d: A d = A x_s - A x_{s-1} =
                // (x_{s-1} - r_s) - (x_{s-1} - c_{s-1}), so
                // r0 = x_s - A x_s - A d = c_s - c_{s-1} + r_s, exact up to
                // rounding without a stencil pass (the residual of the guess is
                // about (dt lambda)^2 |x| for a smooth mode of decay rate lambda,
                // against dt lambda |x| for the guess x_s).
                const int kq = kr_c;
                const bool pred = a.predict && have_c;
                // additive forcing of the previous step (x holds x_s + g_s)
                const double *gp =
                    a.g ? a.g + (long long)b * a.g_stride + (long long)(step - 2) * a.g_step + GI.off : nullptr;
                float acc[2] = {0.0f, 0.0f};
#pragma unroll 4
                for (int j = tid; j < n; j += nt) {
                    const double xs = x[j], bo = bvec[j];
                    const float rs = rv[j];
                    const double d = xs - bo;
                    const double cn = to_f64(rs, -kq) + d;
                    float r0;
                    if (pred) {
                        r0 = to_f32_rn(cn - cvec[j], kq) + rs;
                        x[j] = xs + d;
                    } else {
                        r0 = to_f32_rn(cn, kq);
                        if (gp) x[j] = xs - gp[j];
                    }
                    if (!gp) cvec[j] = cn;
                    bvec[j] = xs;
                    rv[j] = r0;
                    const float xf = to_f32(xs, kq);
                    acc[0] += r0 * r0;
                    acc[1] += xf * xf;
                }
                R32.template sum<2>(acc);  // also: x, b and rv complete
                rn2 = to_f64(acc[0], -2 * kq);
                bb = to_f64(acc[1], -2 * kq);
                kr = kq;
                have_c = (gp == nullptr);
            } else {
                // right-hand side b = x_{s-1} + dt f; optional initial guess;
                // second SDIRK stage: b = (1 - beta) u_n + beta U1 (b holds u_n,
                // x holds U1, the stage's initial iterate)
                // (extrapolated steps: u_n saved at stage 0; stage 1 from U1;
                // stage 2 from u_n, with U2 moved to the saved place)
                if (stage > 0 && !a.ext) {
                    for (int j = tid; j < n; j += nt) bvec[j] = SD_ALPHA * bvec[j] + SD_BETA * x[j];
                } else if (stage == 1) {
                    for (int j = tid; j < n; j += nt) bvec[j] = x[j];
                } else if (stage == 2) {
                    for (int j = tid; j < n; j += nt) {
                        const double un = cvec[j];
                        cvec[j] = x[j];
                        bvec[j] = un;
                    }
                } else if (a.guess) {
                    const long long sb0 = (long long)(step - 1);
                    const double *gu = a.guess + (long long)b * a.guess_stride + sb0 * a.guess_step + GI.off;
                    const double *gf = a.g ? a.g + (long long)b * a.g_stride + sb0 * a.g_step + GI.off : nullptr;
                    for (int j = tid; j < n; j += nt) {
                        const double bj = f ? x[j] + dt * f[j] : x[j];
                        bvec[j] = bj;
                        if (a.ext) cvec[j] = bj;
                        x[j] = gf ? gu[j] - gf[j] : gu[j];
                    }
                } else {
                    for (int j = tid; j < n; j += nt) {
                        const double bj = f ? x[j] + dt * f[j] : x[j];
                        bvec[j] = bj;
                        if (a.ext) cvec[j] = bj;
                    }
                }
                double acc[1] = {0.0};
                for (int j = tid; j < n; j += nt) acc[0] += bvec[j] * bvec[j];
                R64.template sum<1>(acc);  // also: bvec and x complete
                bb = acc[0];
                kr = scale_exp(bb);
                float accf[1] = {0.0f};
                // without forcing x = b here, so r0 is c_{s-1} = x_{s-1} - A x_{s-1}
#pragma unroll 4
                for (int j = tid; j < n; j += nt) {
                    const double r = RES64(bvec[j], x, j);
                    const float rf = to_f32_rn(r, kr);
                    if (carry_ok) cvec[j] = r;
                    rv[j] = rf;
                    accf[0] += rf * rf;
                }
                R32.template sum<1>(accf);
                ++passes;
                rn2 = to_f64(accf[0], -2 * kr);
                have_c = carry_ok;
            }
            have_r0 = false;
            const double stop2 = a.rtol * a.rtol * bb;
            const int ks = scale_exp(bb);  // FP32 copies of this step: value 2^ks, ||b|| 2^ks in [1, 2)
            int st_step = PIT_OK;
            for (int pass = 0;; ++pass) {
                if (!(rn2 > stop2)) {
                    if (rn2 != rn2) st_step = PIT_ERR_NONFINITE;
                    break;
                }
                if (pass >= a.ir_maxit) { st_step = PIT_ERR_NOCONV; break; }
                // Scalars in FP32 on the scaled residual: rv 2^-kn has squared
                // norm R2n = ||r||^2 4^(kr - kn) in [1, 4); the power of two
                // makes the rescaling of the correction exact.
                const int kn = min(max(kr - scale_exp(rn2), -120), 120);
                const float inv = __uint_as_float((unsigned)(127 - kn) << 23);  // 2^-kn
                const float R2n = to_f32(rn2, 2 * (kr - kn));
                const float want = 0.5f * sqrtf(to_f32(stop2, 2 * (kr - kn)) / R2n);
                const float tgt = want > a.inner_rtol ? want : (float)a.inner_rtol;
                const float stop32 = tgt * tgt * R2n;
                for (int j = tid; j < n; j += nt) {
                    rv[j] *= jac ? inv * tab32[j] : inv;
                    e[j] = 0.0f;
                }
                int st, k;
                if constexpr (DRIFT) k = bicgstab_core<float, float>(T32, n, e, rv, pv, sv, wv, tv, R32, stop32, a.maxit, st);
                else if constexpr (OP == PIT_OP_HEAT) {
                    if (use_pc) k = pcg_core<float, float>(HT, LM, n, e, rv, f32 + 5 * ld, pv, sv, wv, R32, stop32, a.maxit, st);
                    else k = cg_core<float, float>(HT, n, e, rv, pv, sv, wv, R32, stop32, a.maxit, st);
                }
                else k = cg_core<float, float>(T32, n, e, rv, pv, sv, wv, R32, stop32, a.maxit, st);
                iters += k;
                if (st == PIT_ERR_NONFINITE) { st_step = st; break; }
                // a stalled or broken-down inner solve still gives a usable
                // correction; the FP64 residual decides.  x += e 2^(kn - kr)
                // (FP64, exact scaling)
                const double cs = pow2d(kn - kr);
                // (four nodes per thread are loaded before any is stored: x may
                // live in global memory, where the compiler cannot reorder
                // loads across the possibly aliasing stores)
                for (int j0 = tid; j0 < n; j0 += 4 * nt) {
                    double xv[4];
                    float ev[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int j = j0 + q * nt;
                        if (j < n) {
                            ev[q] = jac ? e[j] * tab32[j] : e[j];  // Jacobi: e = D^{-1/2} y
                            xv[q] = x[j];
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int j = j0 + q * nt;
                        if (j < n) x[j] = fma(to_f64(ev[q], 0), cs, xv[q]);
                    }
                }
                __syncthreads();  // x complete
                // FP64 check: r = b - A x; the stopping test works on the FP32
                // copy (its squared norm accumulated in FP32), which the next
                // step also reads for its carried initial residual
                float accf[1] = {0.0f};
                // (unrolled: independent nodes keep several FP64 stencil
                // chains in flight, the FP64 latency is long on GB300)
#pragma unroll 4
                for (int j = tid; j < n; j += nt) {
                    const float rf = to_f32_rn(RES64(bvec[j], x, j), ks);
                    rv[j] = rf;
                    accf[0] += rf * rf;
                }
                R32.template sum<1>(accf);
                ++passes;
                rn2 = to_f64(accf[0], -2 * ks);
                kr = ks;
            }
            if (st_step > status) status = st_step;
            // rv holds the FP64 residual of the final x (from its check, or
            // the unchanged initial residual when pass 0 met the tolerance)
            have_r0 = carry_g && st_step == PIT_OK && step < a.nsteps;
            kr_c = kr;
          }
            if constexpr (OP == PIT_OP_VARHEAT) {
                if (a.ext) {
                    table_full_step(false);
                    for (int j = tid; j < n; j += nt) x[j] = 2.0 * cvec[j] - x[j];
                }
            }
            if constexpr (OP == PIT_OP_HEAT) {
                if (a.ext) {
                    // back to the half step; u_{n+1} = 2 U2 - U3 (the last
                    // reduction ordered every read of the stage's x)
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        H64.off[i] *= 0.5;
                        HT.off[i] *= (T)0.5;
                    }
                    H64.diag = diag64h;
                    HT.diag = diagTh;
                    use_pc = use_pc0;
                    for (int j = tid; j < n; j += nt) x[j] = 2.0 * cvec[j] - x[j];
                }
            }
        }
        // forcing of this step and the stored outputs (own nodes only)
        const long long sb = (long long)(step - 1);
        if (a.g) {
            const double *gs = a.g + (long long)b * a.g_stride + sb * a.g_step + GI.off;
            for (int j = tid; j < n; j += nt) x[j] += gs[j];
        }
        const double *hs = a.hs ? a.hs + (long long)b * a.hs_stride + sb * a.hs_step + GI.off : nullptr;
        if (step < a.nsteps) {
            if (a.out_steps) {
                double *os = a.out_steps + (long long)b * a.os_stride + sb * a.os_step + GI.off;
                for (int j = tid; j < n; j += nt) os[j] = hs ? x[j] + hs[j] : x[j];
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
                ol[j] = a.out_scale * xj + (h ? a.out_hscale * h[j] : 0.0) + (hs ? hs[j] : 0.0);
            }
            if (cmp) {
                R64.template sum<1>(acc);
                if (tid == 0) a.norms[(long long)b * a.n_grids + g] = sqrt(acc[0]);
            }
        }
    }
    if (a.inexact && status == PIT_ERR_NOCONV) status = PIT_OK;  // fixed-iteration (inexact) solves
    if (tid == 0 && a.stats) {
        atomicAdd(&a.stats->sum_iters, (unsigned long long)iters);
        atomicAdd(&a.stats->items, (unsigned long long)a.nsteps);
        atomicAdd(&a.stats->point_iters, (unsigned long long)iters * (unsigned long long)n);
        atomicAdd(&a.stats->point_passes, (unsigned long long)passes * (unsigned long long)n);
        atomicAdd(&a.stats->point_steps, (unsigned long long)a.nsteps * (unsigned long long)n);
        atomicMax(&a.stats->max_iters, iters);
        atomicMax(&a.stats->max_refine, passes);
        if (status != PIT_OK) {
            atomicAdd(&a.stats->n_failed, 1);
            atomicMax(&a.stats->worst, status);
        }
    }
}

// Launchers, one translation unit per (operator, precision form): OPN names
// the operator (heat, varheat, ou), PN the form (fp64, mixed, fp32).
#define PIT_STEPS_DECL(OPN, PN)                                                                                   \
    cudaError_t steps_init_##OPN##_##PN(int bytes);                                                               \
    cudaError_t steps_launch_##OPN##_##PN(int d, const StepArgs &a, dim3 grid, dim3 block, size_t smem,           \
                                          cudaStream_t s, bool xg);
PIT_STEPS_DECL(heat, fp64) PIT_STEPS_DECL(heat, mixed) PIT_STEPS_DECL(heat, fp32)
PIT_STEPS_DECL(varheat, fp64) PIT_STEPS_DECL(varheat, mixed) PIT_STEPS_DECL(varheat, fp32)
PIT_STEPS_DECL(ou, fp64) PIT_STEPS_DECL(ou, mixed) PIT_STEPS_DECL(ou, fp32)
PIT_STEPS_DECL(lsde, fp64) PIT_STEPS_DECL(lsde, mixed) PIT_STEPS_DECL(lsde, fp32)
PIT_STEPS_DECL(cme, fp64) PIT_STEPS_DECL(cme, mixed) PIT_STEPS_DECL(cme, fp32)
PIT_STEPS_DECL(heat, pair) PIT_STEPS_DECL(varheat, pair)

// Instantiates the attribute setter and launcher of one operator and form for
// D = 1..6 (XGV: whether the form has the global-state variant).
#define PIT_STEPS_SET1(OPV, PV, XGV, D)                                                                           \
    set((const void *)steps_kernel<OPV, PV, D>);                                                                  \
    if constexpr (XGV) set((const void *)steps_kernel<OPV, PV, D, XGV>);
#define PIT_STEPS_CASE1(OPV, PV, XGV, D)                                                                          \
    case D:                                                                                                       \
        if constexpr (XGV) {                                                                                      \
            if (xg) { steps_kernel<OPV, PV, D, XGV><<<grid, block, smem, s>>>(a); break; }                        \
        }                                                                                                         \
        steps_kernel<OPV, PV, D><<<grid, block, smem, s>>>(a);                                                    \
        break;
#define PIT_STEPS_OP_PREC(OPN, PN, OPV, PV, XGV)                                                                  \
    cudaError_t steps_init_##OPN##_##PN(int bytes)                                                                \
    {                                                                                                             \
        cudaError_t e = cudaSuccess;                                                                              \
        auto set = [&](const void *fn) {                                                                          \
            if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes); \
        };                                                                                                        \
        PIT_STEPS_SET1(OPV, PV, XGV, 1) PIT_STEPS_SET1(OPV, PV, XGV, 2) PIT_STEPS_SET1(OPV, PV, XGV, 3)           \
        PIT_STEPS_SET1(OPV, PV, XGV, 4) PIT_STEPS_SET1(OPV, PV, XGV, 5) PIT_STEPS_SET1(OPV, PV, XGV, 6)           \
        return e;                                                                                                 \
    }                                                                                                             \
    cudaError_t steps_launch_##OPN##_##PN(int d, const StepArgs &a, dim3 grid, dim3 block, size_t smem,           \
                                          cudaStream_t s, bool xg)                                                \
    {                                                                                                             \
        if (xg && !XGV) return cudaErrorInvalidValue;                                                             \
        switch (d) {                                                                                              \
        PIT_STEPS_CASE1(OPV, PV, XGV, 1) PIT_STEPS_CASE1(OPV, PV, XGV, 2) PIT_STEPS_CASE1(OPV, PV, XGV, 3)        \
        PIT_STEPS_CASE1(OPV, PV, XGV, 4) PIT_STEPS_CASE1(OPV, PV, XGV, 5) PIT_STEPS_CASE1(OPV, PV, XGV, 6)        \
        default: return cudaErrorInvalidValue;                                                                    \
        }                                                                                                         \
        return cudaGetLastError();                                                                                \
    }

}  // namespace pit
