// Auxiliary kernels of libpit: stencil application, initial values, face
// coefficients of the variable-coefficient operator, the combination sum and
// the MGRIT residual norms.
#include "pit_internal.cuh"

namespace pit {

__device__ __forceinline__ int axis_coord(const GridInfo &G, int j, int i) { return (j / G.S[i]) % G.N[i]; }

// Variable diffusion coefficient a(x) = 1 + A prod_i f_i(x_i), f alternating
// sin(2 pi x), cos(2 pi x), ... (d = 3: 1 + A sin(2 pi x1) cos(2 pi x2) sin(2 pi x3)).
__device__ double varcoef(const OpParams &op, const double *x)
{
    double prod = 1.0;
    for (int i = 0; i < op.d; ++i) prod *= (i % 2 == 0) ? sin(2.0 * M_PI * x[i]) : cos(2.0 * M_PI * x[i]);
    return 1.0 + op.vamp * prod;
}

// (I + dt L) p at node j of grid GI, FP64 with coefficients evaluated per
// node (the reference application of the operator).
__device__ double apply_node(const GridInfo &GI, int j, const double *pg, double dt, const double *faces,
                             const OpParams &op)
{
    const int d = op.d;
    double s = 0.0, diag = 1.0;
    for (int i = 0; i < d; ++i) {
        const int c = axis_coord(GI, j, i);
        const double h = GI.h[i], ih2 = 1.0 / (h * h);
        double dd, dm, dp;
        if (op.op == PIT_OP_HEAT) {
            dd = 2.0 * ih2; dm = -ih2; dp = -ih2;
        } else if (op.op == PIT_OP_VARHEAT) {
            const double am = faces[(GI.off + j) * (2 * d) + 2 * i];
            const double ap = faces[(GI.off + j) * (2 * d) + 2 * i + 1];
            dd = (am + ap) * ih2; dm = -am * ih2; dp = -ap * ih2;
        } else if (op.op == PIT_OP_OU) {
            const double x = op.lo[i] + (double)(c + 1) * h;
            const double vp = -op.theta * (x + 0.5 * h), vm = -op.theta * (x - 0.5 * h);
            const double s2 = 0.5 * op.sigma * op.sigma * ih2;
            drift_coef(vp, vm, h, false, dd, dm, dp);
            dd += 2.0 * s2;
            dm -= s2;
            dp -= s2;
        } else if (op.op == PIT_OP_CME) {
            double xc[PIT_D];
            for (int k = 0; k < d; ++k) xc[k] = op.lo[k] + (double)(axis_coord(GI, j, k) + 1) * GI.h[k];
            cme_coef(cme_production(op, i, xc, d), op.cg[i], xc[i], h, op.central != 0, dd, dm, dp);
        } else {
            // linear SDE: face velocities (A x)_i at x -+ h/2 e_i, diagonal diffusion
            double ax = 0.0;
            for (int k = 0; k < d; ++k)
                ax += op.A[i * d + k] * (op.lo[k] + (double)(axis_coord(GI, j, k) + 1) * GI.h[k]);
            const double vp = ax + 0.5 * h * op.A[i * d + i], vm = ax - 0.5 * h * op.A[i * d + i];
            const double s2 = 0.5 * op.H[i * d + i] * ih2;
            drift_coef(vp, vm, h, op.central != 0, dd, dm, dp);
            dd += 2.0 * s2;
            dm -= s2;
            dp -= s2;
        }
        diag += dt * dd;
        if (c > 0) s += dt * dm * pg[j - GI.S[i]];
        if (c < GI.N[i] - 1) s += dt * dp * pg[j + GI.S[i]];
    }
    if (op.op == PIT_OP_LSDE) {
        // mixed derivatives: -(H_ik + H_ki)/2 (p_{++} - p_{+-} - p_{-+} + p_{--}) / (4 h_i h_k)
        for (int i = 0; i < d; ++i) {
            const int ci = axis_coord(GI, j, i);
            for (int k = i + 1; k < d; ++k) {
                const int ck = axis_coord(GI, j, k);
                const double w = -dt * 0.5 * (op.H[i * d + k] + op.H[k * d + i]) / (4.0 * GI.h[i] * GI.h[k]);
                double c4 = 0.0;
                if (ci < GI.N[i] - 1 && ck < GI.N[k] - 1) c4 += pg[j + GI.S[i] + GI.S[k]];
                if (ci < GI.N[i] - 1 && ck > 0) c4 -= pg[j + GI.S[i] - GI.S[k]];
                if (ci > 0 && ck < GI.N[k] - 1) c4 -= pg[j - GI.S[i] + GI.S[k]];
                if (ci > 0 && ck > 0) c4 += pg[j - GI.S[i] - GI.S[k]];
                s += w * c4;
            }
        }
    }
    return diag * pg[j] + s;
}

// q = (I + dt L) p, one CTA per (batch entry, grid).
__global__ void apply_kernel(const GridInfo *grids, int G, long long ntot, double dt, const double *p, double *q,
                             const double *faces, OpParams op)
{
    const int g = blockIdx.x % G, b = blockIdx.x / G;
    const GridInfo GI = grids[g];
    const double *pg = p + (long long)b * ntot + GI.off;
    double *qg = q + (long long)b * ntot + GI.off;
    for (int j = threadIdx.x; j < GI.n; j += blockDim.x) qg[j] = apply_node(GI, j, pg, dt, faces, op);
}

// Space-time residual of the backward-Euler equation at a C-point (the
// residual mode of MGRIT): rho_b = x_b + dt f_b - (I + dt L) u_b, written as
// scale * rho_b, with ||rho_b||_2 per grid in norms[b * G + g]; active grids
// only (others untouched).  One CTA of 256 threads per (batch entry, grid).
__global__ void st_resid_kernel(const GridInfo *grids, int G, long long ntot, double dt, const double *x,
                                long long xs, const double *f, long long fs, const double *u, long long us,
                                double scale, double *out, long long os, double *norms, const int *active,
                                const double *faces, OpParams op)
{
    const int g = blockIdx.x % G, b = blockIdx.x / G;
    if (active && !active[g]) return;
    const GridInfo GI = grids[g];
    const double *xg = x + b * xs + GI.off, *ug = u + b * us + GI.off;
    const double *fg = f ? f + b * fs + GI.off : nullptr;
    double *og = out + b * os + GI.off;
    double acc = 0.0;
    for (int j = threadIdx.x; j < GI.n; j += blockDim.x) {
        const double r = xg[j] + (fg ? dt * fg[j] : 0.0) - apply_node(GI, j, ug, dt, faces, op);
        og[j] = scale * r;
        acc += r * r;
    }
    __shared__ double part[8];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        norms[(long long)b * G + g] = sqrt(t);
    }
}

cudaError_t launch_st_resid(const GridInfo *grids, int G, long long ntot, int nb, double dt, const double *x,
                            long long xs, const double *f, long long fs, const double *u, long long us, double scale,
                            double *out, long long os, double *norms, const int *active, const double *faces,
                            OpParams op, cudaStream_t s)
{
    const long long blocks = (long long)G * nb;
    if (blocks == 0) return cudaSuccess;
    st_resid_kernel<<<(unsigned)blocks, 256, 0, s>>>(grids, G, ntot, dt, x, xs, f, fs, u, us, scale, out, os, norms,
                                                      active, faces, op);
    return cudaGetLastError();
}

cudaError_t launch_apply(const GridInfo *grids, int G, long long ntot, int n_batch, double dt, const double *p,
                         double *q, const double *faces, OpParams op, cudaStream_t s)
{
    const long long blocks = (long long)G * n_batch;
    if (blocks == 0) return cudaSuccess;
    apply_kernel<<<(unsigned)blocks, 256, 0, s>>>(grids, G, ntot, dt, p, q, faces, op);
    return cudaGetLastError();
}

// Initial values at the interior nodes (kind 0: sum of product-sine modes,
// kind 1: product Gaussian); one CTA per grid.
__global__ void initial_kernel(const GridInfo *grids, OpParams op, const double *hi, int kind, const double *prm,
                               double *u)
{
    const GridInfo GI = grids[blockIdx.x];
    const int d = op.d;
    for (int j = threadIdx.x; j < GI.n; j += blockDim.x) {
        double x[PIT_D];
        for (int i = 0; i < d; ++i) x[i] = op.lo[i] + (double)(axis_coord(GI, j, i) + 1) * GI.h[i];
        double v = 0.0;
        if (kind == 0) {
            const int K = (int)prm[0];
            for (int k = 0; k < K; ++k) {
                const double *pk = prm + 1 + k * (d + 1);
                double prod = pk[0];
                for (int i = 0; i < d; ++i) prod *= sin(M_PI * pk[1 + i] * (x[i] - op.lo[i]) / (hi[i] - op.lo[i]));
                v += prod;
            }
        } else if (kind == 4) {
            // normal density with the covariance's Cholesky factor R (prm[d..]) and
            // log det R (prm[d + d*d]), prepared on the host
            double z[PIT_D], q = 0.0;
            for (int i = 0; i < d; ++i) {
                double r = x[i] - prm[i];
                for (int k = 0; k < i; ++k) r -= prm[d + i * d + k] * z[k];
                z[i] = r / prm[d + i * d + i];
                q += z[i] * z[i];
            }
            v = exp(-0.5 * q - prm[d + d * d] - 0.5 * d * log(2.0 * M_PI));
        } else if (kind == 1) {
            v = 1.0;
            for (int i = 0; i < d; ++i) {
                const double z = (x[i] - prm[i]) / prm[d + i];
                v *= exp(-0.5 * z * z) / (prm[d + i] * sqrt(2.0 * M_PI));
            }
        } else {
            // heat experiment (Sec. 4.2): u*(x,t) = rho e^{-t} S(x), rho = sqrt(|x|^2 + t^2),
            // S = prod_i sin(pi xi_i), xi_i = (x_i - a_i) / w_i; kind 3 gives
            // f = du*/dt - Laplace u* = e^{-t} [S (t/rho - rho) - S (d/rho - |x|^2/rho^3)
            //     - 2 sum_i (x_i/rho) dS/dx_i + rho pi^2 S sum_i 1/w_i^2]
            const double t = prm[0];
            double r2 = 0.0, S = 1.0, sn[PIT_D], cs[PIT_D], w[PIT_D];
            for (int i = 0; i < d; ++i) {
                w[i] = hi[i] - op.lo[i];
                sincospi((x[i] - op.lo[i]) / w[i], &sn[i], &cs[i]);
                S *= sn[i];
                r2 += x[i] * x[i];
            }
            const double rho = sqrt(r2 + t * t), et = exp(-t);
            if (kind == 2) {
                v = rho * et * S;
            } else {
                double grad = 0.0, iw2 = 0.0;
                for (int i = 0; i < d; ++i) {
                    double dS = M_PI / w[i] * cs[i];
                    for (int k = 0; k < d; ++k)
                        if (k != i) dS *= sn[k];
                    grad += x[i] / rho * dS;
                    iw2 += 1.0 / (w[i] * w[i]);
                }
                v = et * (S * (t / rho - rho) - S * (d / rho - r2 / (rho * rho * rho)) - 2.0 * grad +
                          rho * M_PI * M_PI * S * iw2);
            }
        }
        u[GI.off + j] = v;
    }
}

cudaError_t launch_initial(const GridInfo *grids, int G, OpParams op, const double *hi, int kind,
                           const double *params_dev, int n_params, double *u, cudaStream_t s)
{
    (void)n_params;
    initial_kernel<<<G, 256, 0, s>>>(grids, op, hi, kind, params_dev, u);
    return cudaGetLastError();
}

// Face values a(x -+ h_i/2 e_i) of every node (2d per node, packed like the
// state vectors), computed once per problem.
__global__ void faces_kernel(const GridInfo *grids, OpParams op, double *faces)
{
    const GridInfo GI = grids[blockIdx.x];
    const int d = op.d;
    for (int j = threadIdx.x; j < GI.n; j += blockDim.x) {
        double x[PIT_D];
        for (int i = 0; i < d; ++i) x[i] = op.lo[i] + (double)(axis_coord(GI, j, i) + 1) * GI.h[i];
        for (int i = 0; i < d; ++i) {
            const double xi = x[i];
            x[i] = xi - 0.5 * GI.h[i];
            faces[(GI.off + j) * (2 * d) + 2 * i] = varcoef(op, x);
            x[i] = xi + 0.5 * GI.h[i];
            faces[(GI.off + j) * (2 * d) + 2 * i + 1] = varcoef(op, x);
            x[i] = xi;
        }
    }
}

__global__ void masks_kernel(const GridInfo *grids, int d, uint16_t *masks)
{
    const GridInfo GI = grids[blockIdx.x];
    for (int j = threadIdx.x; j < GI.n; j += blockDim.x) {
        unsigned mk = 0;
        for (int i = 0; i < d; ++i) {
            const int c = axis_coord(GI, j, i);
            if (c > 0) mk |= 1u << (2 * i);
            if (c < GI.N[i] - 1) mk |= 1u << (2 * i + 1);
        }
        masks[GI.off + j] = (uint16_t)mk;
    }
}

cudaError_t launch_masks(const GridInfo *grids, int G, int d, uint16_t *masks, cudaStream_t s)
{
    masks_kernel<<<G, 256, 0, s>>>(grids, d, masks);
    return cudaGetLastError();
}

cudaError_t launch_faces(const GridInfo *grids, int G, OpParams op, double *faces, cudaStream_t s)
{
    faces_kernel<<<G, 256, 0, s>>>(grids, op, faces);
    return cudaGetLastError();
}

// Combination sum (Eq. "combination_technique_solution") at arbitrary points:
// out[k] = sum_g coef_g I_g[u_g](x_k), I_g piecewise d-linear with zero
// boundary values.  One thread per point; blockIdx.y takes a contiguous chunk
// of grids in canonical order.  With one chunk the thread writes the sum;
// with several it writes its chunk's partial sum to part[chunk][k] and
// combine_sum_kernel adds the chunks in chunk order.  (One thread per point
// over all grids would keep only n_pts / 128 SMs busy, 33 of 152 for the
// 4,100 points of the d = 6 workload, on FP64 interpolation work.)
__global__ void combine_kernel(const GridInfo *grids, const double *coef, const int *levels, int G, OpParams op,
                               const double *u, int n_pts, const double *pts, int gchunk, double *dst)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_pts) return;
    const int g0 = (int)blockIdx.y * gchunk;
    const int g1 = min(G, g0 + gchunk);
    const int d = op.d;
    // position in units of the domain, once per point: the cell coordinate on
    // a grid of level l is then xr 2^l, an exact scaling (no division per grid)
    double xr[PIT_D];
    for (int i = 0; i < d; ++i) {
        // domain extent hi - lo = h 2^l of any grid (exact: h was (hi - lo) / 2^l)
        const double ext = ldexp(grids[0].h[i], levels[i]);
        xr[i] = (pts[(long long)k * d + i] - op.lo[i]) / ext;
    }
    const int dl = d / 2;  // corner weights: products over the first dl axes times the rest
    double acc = 0.0;
    for (int g = g0; g < g1; ++g) {
        const GridInfo &GI = grids[g];
        int cell[PIT_D];
        double t[PIT_D];
        for (int i = 0; i < d; ++i) {
            const int l = levels[g * d + i];
            const int M = 1 << l;
            const double s = ldexp(xr[i], l);
            int c = (int)floor(s);
            c = c < 0 ? 0 : (c > M - 1 ? M - 1 : c);
            cell[i] = c;
            t[i] = s - (double)c;
        }
        double wlo[8], whi[8];
        wlo[0] = 1.0;
        for (int i = 0; i < dl; ++i)
            for (int q = (1 << i) - 1; q >= 0; --q) {
                wlo[2 * q + 1] = wlo[q] * t[i];
                wlo[2 * q] = wlo[q] * (1.0 - t[i]);
            }
        whi[0] = 1.0;
        for (int i = dl; i < d; ++i)
            for (int q = (1 << (i - dl)) - 1; q >= 0; --q) {
                whi[2 * q + 1] = whi[q] * t[i];
                whi[2 * q] = whi[q] * (1.0 - t[i]);
            }
        double val = 0.0;
        for (int corner = 0; corner < (1 << d); ++corner) {
            long long idx = 0;
            bool inside = true;
            int lo_bits = 0, hi_bits = 0;
            for (int i = 0; i < d; ++i) {
                const int bit = (corner >> i) & 1;
                const int node = cell[i] + bit;  // 0 and 2^l are boundary nodes
                if (i < dl) lo_bits |= bit << (dl - 1 - i);
                else hi_bits |= bit << (d - 1 - i);
                if (node <= 0 || node > GI.N[i]) inside = false;
                else idx += (long long)(node - 1) * GI.S[i];
            }
            if (inside) val += (wlo[lo_bits] * whi[hi_bits]) * u[GI.off + idx];
        }
        acc += coef[g] * val;
    }
    dst[(long long)blockIdx.y * n_pts + k] = acc;
}

__global__ void combine_sum_kernel(const double *part, int n_chunks, int n_pts, double *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_pts) return;
    double s = 0.0;
    for (int c = 0; c < n_chunks; ++c) s += part[(long long)c * n_pts + k];
    out[k] = s;
}

int combine_chunks(int G, int n_pts, int n_sm)
{
    const int blocks = (n_pts + 127) / 128;
    const int want = 4 * (n_sm > 0 ? n_sm : 1);  // about four 128-thread blocks per SM
    int chunks = (want + blocks - 1) / blocks;
    chunks = chunks < 1 ? 1 : (chunks > G ? G : chunks);
    const int gchunk = (G + chunks - 1) / chunks;
    return (G + gchunk - 1) / gchunk;
}

cudaError_t launch_combine(const GridInfo *grids, const double *coef, const int *levels, int G, OpParams op,
                           const double *u, int n_pts, const double *pts, double *out, int n_chunks, double *part,
                           cudaStream_t s)
{
    if (n_pts == 0 || G == 0) return cudaSuccess;
    if (n_chunks < 1 || (n_chunks > 1 && !part)) return cudaErrorInvalidValue;
    const int gchunk = (G + n_chunks - 1) / n_chunks;
    const int chunks = (G + gchunk - 1) / gchunk;
    const dim3 grid((unsigned)((n_pts + 127) / 128), (unsigned)chunks);
    combine_kernel<<<grid, 128, 0, s>>>(grids, coef, levels, G, op, u, n_pts, pts, gchunk, chunks > 1 ? part : out);
    if (chunks > 1) combine_sum_kernel<<<(n_pts + 127) / 128, 128, 0, s>>>(part, chunks, n_pts, out);
    return cudaGetLastError();
}

// resid[j*G + g] = ||a_j - b_j||_2 over grid g (one CTA per (j, g), fixed-order
// reduction).
__global__ void resid_norm_kernel(const GridInfo *grids, int G, const double *a, long long a_stride,
                                  const double *b, long long b_stride, const int *active, double *resid)
{
    const int g = blockIdx.x % G, j = blockIdx.x / G;
    if (active && !active[g]) return;
    const GridInfo GI = grids[g];
    const double *aj = a + (long long)j * a_stride + GI.off;
    const double *bj = b + (long long)j * b_stride + GI.off;
    double s = 0.0;
    for (int t = threadIdx.x; t < GI.n; t += blockDim.x) {
        const double r = aj[t] - bj[t];
        s += r * r;
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        resid[(long long)j * G + g] = sqrt(tot);
    }
}

cudaError_t launch_resid_norms(const GridInfo *grids, int G, long long ntot, int nb, const double *a,
                               long long a_stride, const double *b, long long b_stride, const int *active,
                               double *resid, cudaStream_t s)
{
    (void)ntot;
    const long long blocks = (long long)nb * G;
    if (blocks == 0) return cudaSuccess;
    resid_norm_kernel<<<(unsigned)blocks, 256, 0, s>>>(grids, G, a, a_stride, b, b_stride, active, resid);
    return cudaGetLastError();
}

// out_k = x_k + y_k on the active grids of nb consecutive states.
__global__ void add_states_kernel(const GridInfo *grids, int G, long long ntot, const double *x, const double *y,
                                  double *out, const int *active)
{
    const int g = blockIdx.x % G, k = blockIdx.x / G;
    if (active && !active[g]) return;
    const GridInfo GI = grids[g];
    const long long o = (long long)k * ntot + GI.off;
    for (int j = threadIdx.x; j < GI.n; j += blockDim.x) out[o + j] = x[o + j] + y[o + j];
}

cudaError_t launch_add_states(const GridInfo *grids, int G, long long ntot, int nb, const double *x, const double *y,
                              double *out, const int *active, cudaStream_t s)
{
    const long long blocks = (long long)nb * G;
    if (blocks == 0) return cudaSuccess;
    add_states_kernel<<<(unsigned)blocks, 256, 0, s>>>(grids, G, ntot, x, y, out, active);
    return cudaGetLastError();
}

__global__ void resid_max_kernel(int G, int nb, const double *resid, const int *active, double *rmax)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    if (active && !active[g]) return;
    double m = 0.0;
    for (int j = 0; j < nb; ++j) {
        const double r = resid[(long long)j * G + g];
        if (r > m || r != r) m = r;
        if (m != m) break;
    }
    rmax[g] = m;
}

cudaError_t launch_resid_max(int G, int nb, const double *resid, const int *active, double *rmax, cudaStream_t s)
{
    resid_max_kernel<<<(G + 127) / 128, 128, 0, s>>>(G, nb, resid, active, rmax);
    return cudaGetLastError();
}

}  // namespace pit
