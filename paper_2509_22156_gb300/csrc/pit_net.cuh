// Learned coarse propagator (not in the paper; it replaces the coarse-level
// backward-Euler step Phi_c of Sec. 3.3.1 inside MGRIT): an axis-separable
// 1-D convolutional network, 4 layers of width-5 convolutions along every
// axis with one weight set shared by all axes, channels (u, a, s) -> 16 -> 16
// -> 16 -> 1, ReLU on the hidden layers, applied to the state normalised by
// its RMS sigma:  Phi_hat(u) = u + sigma * h4(u / sigma).  Input channels: the
// normalised state, the diffusion coefficient a at the nodes (1 for constant-
// coefficient operators) and, per axis, s_i = 1 / (1 + 4 dT / h_i^2); taps
// outside the grid read zero (Dirichlet).
//
// Weights are rounded to BF16 (round to nearest even) from FP32 master
// weights; activations and accumulation are FP32; the state and sigma FP64.
// Because the weights are shared across axes, sum_i conv_i(h; W) equals
// sum_t W_t * z_t with z_t = sum_i h(j + (t-2) e_i): each layer forms the
// axis sums once per node and mixes channels once, not d times.  In the
// inference kernel the weights travel as a kernel parameter, so every FMA
// takes its weight from the constant bank (no shared-memory traffic).
#pragma once

#include <cmath>

#include "pit_internal.cuh"

namespace pit {

__host__ __device__ constexpr int net_cin(int k) { return k == 0 ? 3 : 17; }
__host__ __device__ constexpr int net_cout(int k) { return k == 3 ? 1 : 16; }
__host__ __device__ constexpr int net_wo(int k)
{
    return k == 0 ? 0 : net_wo(k - 1) + net_cout(k - 1) * net_cin(k - 1) * 5 + net_cout(k - 1);
}
__host__ __device__ constexpr int net_bo(int k) { return net_wo(k) + net_cout(k) * net_cin(k) * 5; }
static_assert(net_bo(3) + 1 == PIT_NET_PARAMS, "parameter layout");

// Weight access from the kernel-parameter bank or from global memory.
struct WParam {
    const NetWeights &w;
    __device__ __forceinline__ float operator()(int i) const { return w.w[i]; }
};
struct WGlobal {
    const float *w;
    __device__ __forceinline__ float operator()(int i) const { return __ldg(w + i); }
};

// Tap validity of node j along axis i for offset t-2 (t = 0..4): bits of the
// extended mask (4 bits per axis: -1, +1, -2, +2).
__device__ __forceinline__ bool tap_ok(uint32_t mk, int i, int t)
{
    if (t == 2) return true;
    const int bit = (t == 1) ? 0 : (t == 3) ? 1 : (t == 0) ? 2 : 3;
    return (mk >> (4 * i + bit)) & 1u;
}

template <int D>
__device__ __forceinline__ uint32_t ext_mask(const GridInfo &G, int j)
{
    uint32_t mk = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        const int c = (j / G.S[i]) % G.N[i];
        if (c >= 1) mk |= 1u << (4 * i);
        if (c + 1 < G.N[i]) mk |= 1u << (4 * i + 1);
        if (c >= 2) mk |= 1u << (4 * i + 2);
        if (c + 2 < G.N[i]) mk |= 1u << (4 * i + 3);
    }
    return mk;
}

// Diffusion coefficient at the nodes (the network's second input channel).
__device__ inline double node_coef(const OpParams &op, const GridInfo &G, int j, int d)
{
    if (op.op != PIT_OP_VARHEAT) return 1.0;
    double prod = 1.0;
    for (int i = 0; i < d; ++i) {
        const double x = op.lo[i] + (double)((j / G.S[i]) % G.N[i] + 1) * G.h[i];
        prod *= (i % 2 == 0) ? sin(2.0 * M_PI * x) : cos(2.0 * M_PI * x);
    }
    return 1.0 + op.vamp * prod;
}

// One convolution layer: out[o][j] = act(b_o + sum_t sum_c W[o][c][t] z_{c,t}(j)),
// z_{c,t}(j) = sum_i in[c][j + (t-2) S_i] over valid taps; the last input
// channel is the per-axis constant s_i.
template <int D, int CIN, int COUT, bool RELU, class WA>
__device__ __forceinline__ void conv_layer(const WA &W, int wo, int bo, const float *in, float *out, int n, int ld,
                                           const uint32_t *mk2, const int *S, const float *sf)
{
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        float acc[COUT];
#pragma unroll
        for (int o = 0; o < COUT; ++o) acc[o] = W(bo + o);
        const uint32_t mk = mk2[j];
#pragma unroll
        for (int t = 0; t < 5; ++t) {
#pragma unroll
            for (int c = 0; c < CIN - 1; ++c) {
                float z = 0.0f;
#pragma unroll
                for (int i = 0; i < D; ++i)
                    if (tap_ok(mk, i, t)) z += in[c * ld + j + (t - 2) * S[i]];
#pragma unroll
                for (int o = 0; o < COUT; ++o) acc[o] = fmaf(W(wo + (o * CIN + c) * 5 + t), z, acc[o]);
            }
            float zs = 0.0f;
#pragma unroll
            for (int i = 0; i < D; ++i)
                if (tap_ok(mk, i, t)) zs += sf[i];
#pragma unroll
            for (int o = 0; o < COUT; ++o) acc[o] = fmaf(W(wo + (o * CIN + CIN - 1) * 5 + t), zs, acc[o]);
        }
#pragma unroll
        for (int o = 0; o < COUT; ++o) out[o * ld + j] = RELU ? fmaxf(acc[o], 0.0f) : acc[o];
    }
}

// Deterministic block sum in FP64 (shuffles, one barrier, same tree in every warp).
__device__ __forceinline__ double block_sum64(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();  // red free
    if (lane == 0) red[w] = v;
    __syncthreads();
    double x = (lane < nw) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return __shfl_sync(0xffffffffu, x, 0);
}

// Full forward pass of one item on normalised input already in A0 (channel 0:
// u / sigma, channel 1: a).  Result (layer-4 pre-activation) in O[0..n).
// H holds 3 x 16 channels when keep is set (training), else 2 x 16 (ping-pong).
template <int D, class WA>
__device__ void net_forward(const WA &W, const float *A0, float *H, float *O, int n, int ld, const uint32_t *mk2,
                            const int *S, const float *sf, bool keep)
{
    float *H1 = H, *H2 = H + 16 * ld, *H3 = keep ? H + 32 * ld : H;
    conv_layer<D, 3, 16, true>(W, net_wo(0), net_bo(0), A0, H1, n, ld, mk2, S, sf);
    __syncthreads();
    conv_layer<D, 17, 16, true>(W, net_wo(1), net_bo(1), H1, H2, n, ld, mk2, S, sf);
    __syncthreads();
    conv_layer<D, 17, 16, true>(W, net_wo(2), net_bo(2), H2, H3, n, ld, mk2, S, sf);
    __syncthreads();
    conv_layer<D, 17, 1, false>(W, net_wo(3), net_bo(3), H3, O, n, ld, mk2, S, sf);
    __syncthreads();
}

// ----------------------------------------------------------------------------
// Inference: multi-step application of the network with the StepArgs
// semantics of the backward-Euler kernels (forcing g after each step, stored
// steps, out_last = out_scale * x + h).  One CTA per item; activations in
// shared memory (act == NULL) or in a per-item global slab.
template <int D>
__global__ void __launch_bounds__(256) net_steps_kernel(StepArgs a, const __grid_constant__ NetWeights W, float *act,
                                                        long long act_stride)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ GridInfo GI;
    __shared__ double red[32];
    __shared__ int S[D];
    __shared__ float sf[D];
    const int item = a.item0 + (int)blockIdx.x;
    const int g = a.order[item / a.n_batch];
    const int b = item % a.n_batch;
    if (a.active && !a.active[g]) return;
    if (threadIdx.x == 0) GI = a.grids[g];
    __syncthreads();
    const int tid = threadIdx.x, nt = blockDim.x, n = GI.n, ld = (n + 3) & ~3;
    if (tid < D) {
        S[tid] = GI.S[tid];
        sf[tid] = (float)(1.0 / (1.0 + 4.0 * a.dt / (GI.h[tid] * GI.h[tid])));
    }
    double *x = reinterpret_cast<double *>(smem);
    uint32_t *mk2 = reinterpret_cast<uint32_t *>(x + ld);
    float *base = act ? act + (long long)blockIdx.x * act_stride : reinterpret_cast<float *>(mk2 + ld);
    float *A0 = base, *H = base + 2 * ld, *O = base + 34 * ld;
    const double *in = a.in + (long long)b * a.in_stride + GI.off;
    for (int j = tid; j < n; j += nt) {
        x[j] = in[j];
        mk2[j] = ext_mask<D>(GI, j);
        A0[ld + j] = (float)node_coef(a.op, GI, j, D);
    }
    for (int step = 1; step <= a.nsteps; ++step) {
        __syncthreads();
        double ss = 0.0;
        for (int j = tid; j < n; j += nt) ss += x[j] * x[j];
        ss = block_sum64(ss, red);
        const double sigma = sqrt(ss / (double)n);
        if (sigma > 0.0) {
            const double inv = 1.0 / sigma;
            for (int j = tid; j < n; j += nt) A0[j] = (float)(x[j] * inv);
            __syncthreads();
            net_forward<D>(WParam{W}, A0, H, O, n, ld, mk2, S, sf, false);
            for (int j = tid; j < n; j += nt) x[j] += sigma * (double)O[j];
        }
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
            for (int j = tid; j < n; j += nt)
                ol[j] = a.out_scale * x[j] + (h ? a.out_hscale * h[j] : 0.0) + (hs ? hs[j] : 0.0);
        }
    }
    if (tid == 0 && a.stats) {
        atomicAdd(&a.stats->items, (unsigned long long)a.nsteps);
        atomicAdd(&a.stats->point_steps, (unsigned long long)a.nsteps * (unsigned long long)n);
    }
}

// ----------------------------------------------------------------------------
// Training: one CTA per item (a grid of one pair): forward with stored
// activations, relative squared loss ||Phi_hat(u) - y||^2 / ||y||^2, and the
// gradient with respect to every parameter, written as one row per item
// (reduced later in a fixed order, so the gradient is deterministic).
template <int D>
__global__ void __launch_bounds__(256) net_train_kernel(const GridInfo *grids, const NetTrainItem *items, const double *u,
                                                        const double *y, double dT, const float *w, float *act,
                                                        long long act_stride, float *grad_rows, double *loss_items,
                                                        OpParams op)
{
    __shared__ GridInfo GI;
    __shared__ double red[32];
    __shared__ int S[D];
    __shared__ float sf[D];
    __shared__ float gacc[3][16 * 17 * 5 + 16];  // per node-group partial weight gradients of one layer
    const NetTrainItem it = items[blockIdx.x];
    if (threadIdx.x == 0) GI = grids[it.g];
    __syncthreads();
    const int tid = threadIdx.x, nt = blockDim.x, n = GI.n, ld = (n + 3) & ~3;
    if (tid < D) {
        S[tid] = GI.S[tid];
        sf[tid] = (float)(1.0 / (1.0 + 4.0 * dT / (GI.h[tid] * GI.h[tid])));
    }
    float *base = act + (long long)blockIdx.x * act_stride;
    float *A0 = base, *H = base + 2 * ld, *O = base + 50 * ld, *DA = base + 51 * ld, *DB = base + 67 * ld;
    uint32_t *mk2 = reinterpret_cast<uint32_t *>(base + 83 * ld);
    const double *ui = u + it.off, *yi = y + it.off;
    float *grow = grad_rows + (long long)blockIdx.x * PIT_NET_PARAMS;
    double ss = 0.0, yy = 0.0;
    for (int j = tid; j < n; j += nt) {
        mk2[j] = ext_mask<D>(GI, j);
        A0[ld + j] = (float)node_coef(op, GI, j, D);
        ss += ui[j] * ui[j];
        yy += yi[j] * yi[j];
    }
    ss = block_sum64(ss, red);
    yy = block_sum64(yy, red);
    const double sigma = sqrt(ss / (double)n);
    if (!(yy > 0.0)) yy = 1.0;
    if (!(sigma > 0.0)) {
        // identity map: the loss does not depend on the parameters
        double l = 0.0;
        for (int j = tid; j < n; j += nt) l += (ui[j] - yi[j]) * (ui[j] - yi[j]);
        l = block_sum64(l, red);
        for (int p = tid; p < PIT_NET_PARAMS; p += nt) grow[p] = 0.0f;
        if (tid == 0) loss_items[blockIdx.x] = l / yy;
        return;
    }
    const double inv = 1.0 / sigma;
    for (int j = tid; j < n; j += nt) A0[j] = (float)(ui[j] * inv);
    __syncthreads();
    WGlobal W{w};
    net_forward<D>(W, A0, H, O, n, ld, mk2, S, sf, true);
    // loss and dL/d(layer-4 pre-activation) = 2 e sigma / ||y||^2
    double l = 0.0;
    for (int j = tid; j < n; j += nt) {
        const double e = ui[j] + sigma * (double)O[j] - yi[j];
        l += e * e;
        DA[j] = (float)(2.0 * e * sigma / yy);
    }
    l = block_sum64(l, red);
    if (tid == 0) loss_items[blockIdx.x] = l / yy;
    __syncthreads();

    // backward, layer k = 3..0: dpre_k in DCUR (Cout x ld); layer input IN (Cin-1 data channels)
    float *DCUR = DA, *DNXT = DB;
    for (int k = 3; k >= 0; --k) {
        const int cout = net_cout(k);
        const int cind = net_cin(k) - 1;  // data channels (2 or 16)
        const float *IN = (k == 0) ? A0 : H + (k - 1) * 16 * ld;
        const int wo = net_wo(k), bo = net_bo(k);
        const int nw = cout * (cind + 1) * 5;
        // weight and bias gradients: 85 (c,t) pairs (35 for layer 0) x 3 node groups
        const int pairs = (cind + 1) * 5;
        for (int q = tid; q < 3 * (nw + cout); q += nt) gacc[q / (nw + cout)][q % (nw + cout)] = 0.0f;
        __syncthreads();
        for (int q = tid; q < 3 * pairs; q += nt) {
            const int grp = q / pairs, pc = q % pairs;
            const int c = pc / 5, t = pc % 5;
            float accw[16];
#pragma unroll
            for (int o = 0; o < 16; ++o) accw[o] = 0.0f;
            float accb[16];
#pragma unroll
            for (int o = 0; o < 16; ++o) accb[o] = 0.0f;
            for (int j = grp; j < n; j += 3) {
                const uint32_t mk = mk2[j];
                float z = 0.0f;
                for (int i = 0; i < D; ++i)
                    if (tap_ok(mk, i, t)) z += (c < cind) ? IN[c * ld + j + (t - 2) * S[i]] : sf[i];
#pragma unroll
                for (int o = 0; o < 16; ++o) {
                    if (o < cout) {
                        const float dp = DCUR[o * ld + j];
                        accw[o] = fmaf(dp, z, accw[o]);
                        accb[o] += dp;
                    }
                }
            }
            for (int o = 0; o < cout; ++o) gacc[grp][(o * (cind + 1) + c) * 5 + t] = accw[o];
            if (pc == 0)
                for (int o = 0; o < cout; ++o) gacc[grp][nw + o] = accb[o];
        }
        __syncthreads();
        for (int p = tid; p < nw + cout; p += nt)
            grow[wo + p] = (gacc[0][p] + gacc[1][p]) + gacc[2][p];  // wo + nw == bo
        (void)bo;
        if (k == 0) break;
        // input gradient of layer k through the ReLU of layer k-1:
        // din[c][jj] = sum_t sum_o W[o][c][t] sum_i dpre[o][jj - (t-2) e_i]
        const float *HPREV = H + (k - 1) * 16 * ld;
        for (int j = tid; j < n; j += nt) {
            const uint32_t mk = mk2[j];
            float din[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) din[c] = 0.0f;
#pragma unroll
            for (int t = 0; t < 5; ++t) {
                for (int o = 0; o < cout; ++o) {
                    float qv = 0.0f;
#pragma unroll
                    for (int i = 0; i < D; ++i)
                        if (tap_ok(mk, i, 4 - t)) qv += DCUR[o * ld + j - (t - 2) * S[i]];
#pragma unroll
                    for (int c = 0; c < 16; ++c) din[c] = fmaf(W(wo + (o * 17 + c) * 5 + t), qv, din[c]);
                }
            }
#pragma unroll
            for (int c = 0; c < 16; ++c) DNXT[c * ld + j] = HPREV[c * ld + j] > 0.0f ? din[c] : 0.0f;
        }
        __syncthreads();
        float *tmp = DCUR;
        DCUR = DNXT;
        DNXT = tmp;
    }
}

// Per-dimension launchers (one translation unit per d, pit_net_d<d>.cu).
#define PIT_NET_DECL(D)                                                                                          \
    cudaError_t net_init_d##D(int bytes);                                                                        \
    void net_launch_steps_d##D(const StepArgs &a, const NetWeights &W, float *act, long long act_stride,         \
                               dim3 grid, dim3 block, size_t smem, cudaStream_t s);                              \
    void net_launch_train_d##D(const GridInfo *grids, const NetTrainItem *it, const double *u, const double *y,   \
                               double dT, const float *w, float *act, long long act_stride, float *grad_rows,    \
                               double *loss_items, OpParams op, dim3 grid, dim3 block, cudaStream_t s);
PIT_NET_DECL(1) PIT_NET_DECL(2) PIT_NET_DECL(3) PIT_NET_DECL(4) PIT_NET_DECL(5) PIT_NET_DECL(6)

#define PIT_NET_DIM(D)                                                                                           \
    cudaError_t net_init_d##D(int bytes)                                                                         \
    {                                                                                                            \
        return cudaFuncSetAttribute((const void *)net_steps_kernel<D>,                                           \
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);                         \
    }                                                                                                            \
    void net_launch_steps_d##D(const StepArgs &a, const NetWeights &W, float *act, long long act_stride,         \
                               dim3 grid, dim3 block, size_t smem, cudaStream_t s)                               \
    {                                                                                                            \
        net_steps_kernel<D><<<grid, block, smem, s>>>(a, W, act, act_stride);                                    \
    }                                                                                                            \
    void net_launch_train_d##D(const GridInfo *grids, const NetTrainItem *it, const double *u, const double *y,   \
                               double dT, const float *w, float *act, long long act_stride, float *grad_rows,    \
                               double *loss_items, OpParams op, dim3 grid, dim3 block, cudaStream_t s)           \
    {                                                                                                            \
        net_train_kernel<D><<<grid, block, 0, s>>>(grids, it, u, y, dT, w, act, act_stride, grad_rows,           \
                                                   loss_items, op);                                              \
    }

}  // namespace pit
