// Host side of the learned coarse propagator (device code in pit_net.cuh,
// instantiated per dimension in pit_net_d1.cu .. pit_net_d6.cu): shared-memory
// sizes, kernel set-up, launch dispatch by dimension, and the Adam step.
#include "pit_net.cuh"

namespace pit {

// Sum of the per-item gradient rows in item order, then one Adam step on the
// FP32 master weights and their BF16 rounding (round to nearest even).
__device__ __forceinline__ float round_bf16(float v)
{
    uint32_t b = __float_as_uint(v);
    if ((b & 0x7f800000u) == 0x7f800000u) return v;  // Inf / NaN unchanged
    b += 0x7fffu + ((b >> 16) & 1u);
    return __uint_as_float(b & 0xffff0000u);
}

__global__ void net_adam_kernel(const float *grad_rows, int n_rows, float scale, float *master, float *m, float *v,
                                float *w_bf16, float lr, float b1, float b2, float eps, int t, float *grad_out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= PIT_NET_PARAMS) return;
    float gsum = 0.0f;
    for (int r = 0; r < n_rows; ++r) gsum += grad_rows[(long long)r * PIT_NET_PARAMS + p];
    const float gr = gsum * scale;
    if (grad_out) grad_out[p] = gsum;
    if (!master) return;
    const float mm = b1 * m[p] + (1.0f - b1) * gr;
    const float vv = b2 * v[p] + (1.0f - b2) * gr * gr;
    m[p] = mm;
    v[p] = vv;
    const float mh = mm / (1.0f - powf(b1, (float)t));
    const float vh = vv / (1.0f - powf(b2, (float)t));
    const float th = master[p] - lr * mh / (sqrtf(vh) + eps);
    master[p] = th;
    w_bf16[p] = round_bf16(th);
}

// ----------------------------------------------------------------------------
size_t net_smem_bytes(int n)
{
    const size_t ld = (size_t)((n + 3) & ~3);
    return ld * 8 + ld * 4 + 35 * ld * 4 + 16;
}

size_t net_act_floats(int n, bool train)
{
    const size_t ld = (size_t)((n + 3) & ~3);
    return train ? 84 * ld : 35 * ld;
}

static size_t g_net_max_smem = 0;

cudaError_t net_kernels_init(size_t max_smem)
{
    cudaError_t e = cudaSuccess;
    const int bytes = (int)max_smem;
    cudaError_t (*inits[])(int) = {net_init_d1, net_init_d2, net_init_d3, net_init_d4, net_init_d5, net_init_d6};
    for (auto f : inits)
        if (e == cudaSuccess) e = f(bytes);
    if (e == cudaSuccess) g_net_max_smem = max_smem;
    return e;
}

cudaError_t launch_net_steps(const StepArgs &a, const NetWeights &W, float *act, long long act_stride, size_t smem,
                             cudaStream_t s, int n_items)
{
    const long long blocks = n_items;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL || smem > g_net_max_smem) return cudaErrorInvalidConfiguration;
    const dim3 grid((unsigned)blocks), block(256);
    switch (a.op.d) {
    case 1: net_launch_steps_d1(a, W, act, act_stride, grid, block, smem, s); break;
    case 2: net_launch_steps_d2(a, W, act, act_stride, grid, block, smem, s); break;
    case 3: net_launch_steps_d3(a, W, act, act_stride, grid, block, smem, s); break;
    case 4: net_launch_steps_d4(a, W, act, act_stride, grid, block, smem, s); break;
    case 5: net_launch_steps_d5(a, W, act, act_stride, grid, block, smem, s); break;
    case 6: net_launch_steps_d6(a, W, act, act_stride, grid, block, smem, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_net_train(const GridInfo *grids, const NetTrainItem *items, int n_items, const double *u,
                             const double *y, double dT, const float *w, float *act, long long act_stride,
                             float *grad_rows, double *loss_items, OpParams op, cudaStream_t s)
{
    if (n_items <= 0) return cudaSuccess;
    const NetTrainItem *it = items;
    const dim3 grid(n_items), block(256);
    switch (op.d) {
    case 1: net_launch_train_d1(grids, it, u, y, dT, w, act, act_stride, grad_rows, loss_items, op, grid, block, s); break;
    case 2: net_launch_train_d2(grids, it, u, y, dT, w, act, act_stride, grad_rows, loss_items, op, grid, block, s); break;
    case 3: net_launch_train_d3(grids, it, u, y, dT, w, act, act_stride, grad_rows, loss_items, op, grid, block, s); break;
    case 4: net_launch_train_d4(grids, it, u, y, dT, w, act, act_stride, grad_rows, loss_items, op, grid, block, s); break;
    case 5: net_launch_train_d5(grids, it, u, y, dT, w, act, act_stride, grad_rows, loss_items, op, grid, block, s); break;
    case 6: net_launch_train_d6(grids, it, u, y, dT, w, act, act_stride, grad_rows, loss_items, op, grid, block, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_net_adam(const float *grad_rows, int n_rows, float scale, float *master, float *m, float *v,
                            float *w_bf16, float lr, float b1, float b2, float eps, int t, float *grad_out,
                            cudaStream_t s)
{
    net_adam_kernel<<<(PIT_NET_PARAMS + 255) / 256, 256, 0, s>>>(grad_rows, n_rows, scale, master, m, v, w_bf16, lr,
                                                                  b1, b2, eps, t, grad_out);
    return cudaGetLastError();
}

}  // namespace pit
