// Host-side dispatch of the multi-step backward-Euler kernels (pit_phi.cuh):
// shared-memory sizing, attribute set-up and launch by operator, precision
// form and dimension.
#include "pit_phi.cuh"

namespace pit {

size_t phi_smem_bytes(int prec, int op, int d, int n, int na)
{
    const size_t ld = (size_t)((n + 3) & ~3);
    return (size_t)n_f64(op, prec, d) * ld * 8 + (size_t)n_f32(op, prec, d) * ld * 4 + ld * 2 + 16 +
           (size_t)line_pc_bytes(op, prec, false, na);
}

size_t phi_smem_bytes_xg(int prec, int op, int d, int n)
{
    // (the FP32 form's oversize grids run the refinement form's global-state kernel)
    if (prec == SINGLE) prec = MIXED;
    // the FP64 form keeps its coefficient table in global memory as well
    const size_t ld = (size_t)((n + 3) & ~3);
    return (size_t)(prec == PLAIN ? 0 : n_tab(op, d)) * ld * 8 + (size_t)n_f32(op, prec, d, true) * ld * 4 + ld * 2 +
           16;
}

int xg_slabs(int prec, int op, int d)
{
    // PLAIN: x, the Krylov vectors and the coefficient table; MIXED: x, b and
    // the carried x - A x; PAIR uses two
    return prec == PLAIN ? 1 + krylov_vecs(op, PLAIN) + n_tab(op, d) : 3;
}

static size_t g_max_smem = 0;

cudaError_t phi_kernels_init(size_t max_smem)
{
    const int bytes = (int)max_smem;
    cudaError_t e = cudaSuccess;
    cudaError_t (*inits[])(int) = {steps_init_heat_fp64,    steps_init_heat_mixed,    steps_init_heat_fp32,
                                   steps_init_varheat_fp64, steps_init_varheat_mixed, steps_init_varheat_fp32,
                                   steps_init_ou_fp64,      steps_init_ou_mixed,      steps_init_ou_fp32,
                                   steps_init_lsde_fp64,    steps_init_lsde_mixed,    steps_init_lsde_fp32,
                                   steps_init_cme_fp64,     steps_init_cme_mixed,     steps_init_cme_fp32,
                                   steps_init_heat_pair,    steps_init_varheat_pair};
    for (auto f : inits)
        if (e == cudaSuccess) e = f(bytes);
    if (e == cudaSuccess) g_max_smem = max_smem;
    return e;
}

cudaError_t launch_steps(int prec, const StepArgs &a, int threads, size_t smem, cudaStream_t s, bool xg)
{
    const long long blocks = (long long)a.n_batch * a.n_order;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL || smem > g_max_smem || threads < 32 || threads > 512 || (threads & 31))
        return cudaErrorInvalidConfiguration;
    const dim3 grid((unsigned)blocks), block(threads);
    if (prec == SINGLE && xg) {
        // the FP32 form has no global-state variant: grids whose FP32 state does
        // not fit on chip take the refinement form's global-state kernel (FP64
        // state in global memory, FP32 Krylov vectors on chip), which meets the
        // same tolerance on the true residual
        StepArgs m = a;
        if (!(m.inner_rtol > 0.0f && m.inner_rtol < 1.0f)) m.inner_rtol = 1e-4f;
        if (m.ir_maxit < 4) m.ir_maxit = 12;
        switch (a.op.op) {
        case PIT_OP_HEAT: return steps_launch_heat_mixed(a.op.d, m, grid, block, smem, s, true);
        case PIT_OP_VARHEAT: return steps_launch_varheat_mixed(a.op.d, m, grid, block, smem, s, true);
        case PIT_OP_OU: return steps_launch_ou_mixed(a.op.d, m, grid, block, smem, s, true);
        case PIT_OP_LSDE: return steps_launch_lsde_mixed(a.op.d, m, grid, block, smem, s, true);
        case PIT_OP_CME: return steps_launch_cme_mixed(a.op.d, m, grid, block, smem, s, true);
        default: return cudaErrorInvalidValue;
        }
    }
    if (prec == PAIR) {
        // symmetric operators only (the plan rejects the drift operator)
        if (a.op.op == PIT_OP_HEAT) return steps_launch_heat_pair(a.op.d, a, grid, block, smem, s, xg);
        if (a.op.op == PIT_OP_VARHEAT) return steps_launch_varheat_pair(a.op.d, a, grid, block, smem, s, xg);
        return cudaErrorInvalidValue;
    }
    switch (a.op.op) {
#define PIT_BY_PREC(OPN)                                                                                          \
    switch (prec) {                                                                                               \
    case PLAIN: return steps_launch_##OPN##_fp64(a.op.d, a, grid, block, smem, s, xg);                            \
    case MIXED: return steps_launch_##OPN##_mixed(a.op.d, a, grid, block, smem, s, xg);                           \
    case SINGLE: return steps_launch_##OPN##_fp32(a.op.d, a, grid, block, smem, s, xg);                           \
    default: return cudaErrorInvalidValue;                                                                        \
    }
    case PIT_OP_HEAT: PIT_BY_PREC(heat)
    case PIT_OP_VARHEAT: PIT_BY_PREC(varheat)
    case PIT_OP_OU: PIT_BY_PREC(ou)
    case PIT_OP_LSDE: PIT_BY_PREC(lsde)
    case PIT_OP_CME: PIT_BY_PREC(cme)
#undef PIT_BY_PREC
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace pit
