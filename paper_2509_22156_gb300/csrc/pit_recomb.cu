// Recombination of the component-grid solutions (Sec. 2.2.2): the operator
// Q = H^{-1} Qbar H of Eq. "overall_combination_operator".  H hierarchizes
// every grid's nodal values (surplus of each node over the linear
// interpolant of its two hierarchical parents along every axis), Qbar gives
// every node the sum over all grids that share the node of their
// combination coefficient times their surplus there (Eq.
// "recombination_operator"), and H^{-1} dehierarchizes.  The result on grid
// l is the nodal interpolant of the combined solution on Omega_l.
//
// GPU layout: the surpluses of the sparse grid are stored once, block by
// block: one block per hierarchical increment lam (a level multi-index that
// some grid contains), its 2^{|lam|_1 - d} nodes in C order.  Three launches:
//   hier_kernel    one CTA per grid: hierarchize in place (level by level,
//                  a barrier between levels), scale by the grid's coefficient
//   gather_kernel  one thread per sparse-grid node: sum the scaled surpluses
//                  of the grids that contain its increment, in grid order
//                  (deterministic, no atomics)
//   dehier_kernel  one CTA per grid: read the sums of its nodes, then
//                  dehierarchize level by level.
// Work and traffic are linear in the number of nodes of all grids.
#include "pit_internal.cuh"

namespace pit {

namespace {

__device__ __forceinline__ int level_of(int N) { return 31 - __clz(N + 1); }  // N = 2^l - 1

// One level of the 1-D (de)hierarchization along axis `ax` on a grid's
// values v: every node whose 1-based index J has t trailing zero bits gets
// -/+ the mean of its parents J -/+ 2^t (zero on the boundary).
__device__ void hier_level(double *v, const GridInfo &G, int ax, int t, double sgn)
{
    const int N = G.N[ax], S = G.S[ax], step = 1 << t;
    for (int j = threadIdx.x; j < G.n; j += blockDim.x) {
        const int J = (j / S) % N + 1;
        if ((__ffs(J) - 1) != t) continue;
        const double left = (J - step >= 1) ? v[j - step * S] : 0.0;
        const double right = (J + step <= N) ? v[j + step * S] : 0.0;
        v[j] += sgn * 0.5 * (left + right);
    }
}

template <int D>
__global__ void hier_kernel(const GridInfo *grids, const double *coef, int n_grids, long long ntot, const double *u,
                            double *H)
{
    const int g = blockIdx.x % n_grids;
    const long long b = blockIdx.x / n_grids;  // state of the batch
    const GridInfo G = grids[g];
    const double *src = u + b * ntot + G.off;
    double *v = H + b * ntot + G.off;
    for (int j = threadIdx.x; j < G.n; j += blockDim.x) v[j] = src[j];
    __syncthreads();
#pragma unroll
    for (int ax = 0; ax < D; ++ax) {
        const int lev = level_of(G.N[ax]);
        for (int t = 0; t < lev; ++t) {  // finest level first: parents still nodal
            hier_level(v, G, ax, t, -1.0);
            __syncthreads();
        }
    }
    const double c = coef[g];
    for (int j = threadIdx.x; j < G.n; j += blockDim.x) v[j] *= c;
}

template <int D>
__global__ void gather_kernel(RecombPlan R, const GridInfo *grids, long long ntot, int nb, const double *Hb, double *Sb)
{
    const long long qb = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (qb >= R.n_sparse * nb) return;
    const long long bst = qb / R.n_sparse, q = qb - bst * R.n_sparse;  // state of the batch, sparse node
    const double *H = Hb + bst * ntot;
    double *S = Sb + bst * R.n_sparse;
    // block of the node: last b with blk_off[b] <= q
    int lo = 0, hi = R.n_blk - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (R.blk_off[mid] <= q) lo = mid;
        else hi = mid - 1;
    }
    const int b = lo;
    long long r = q - R.blk_off[b];
    int lam[D], p[D];
#pragma unroll
    for (int i = 0; i < D; ++i) lam[i] = R.blk_lam[b * D + i];
#pragma unroll
    for (int i = D - 1; i >= 0; --i) {  // C order, last axis fastest
        const int e = 1 << (lam[i] - 1);
        p[i] = (int)(r % e);
        r /= e;
    }
    double acc = 0.0;
    for (int k = R.list_off[b]; k < R.list_off[b + 1]; ++k) {
        const GridInfo &G = grids[R.list[k]];
        long long idx = 0;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const int J = (2 * p[i] + 1) << (level_of(G.N[i]) - lam[i]);
            idx += (long long)(J - 1) * G.S[i];
        }
        acc += H[G.off + idx];
    }
    S[q] = acc;
}

template <int D>
__global__ void dehier_kernel(RecombPlan R, const GridInfo *grids, int n_grids, long long ntot, const double *Sb,
                              double *out)
{
    const int g = blockIdx.x % n_grids;
    const long long bst = blockIdx.x / n_grids;
    const GridInfo G = grids[g];
    const double *S = Sb + bst * R.n_sparse;
    double *v = out + bst * ntot + G.off;
    for (int j = threadIdx.x; j < G.n; j += blockDim.x) {
        int code = 0;
        long long pos = 0;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const int J = (j / G.S[i]) % G.N[i] + 1;
            const int t = __ffs(J) - 1;
            const int lam = level_of(G.N[i]) - t;
            code = code * R.radix + lam;
            pos = (pos << (lam - 1)) + (J >> (t + 1));
        }
        const int b = R.lookup[code];
        v[j] = S[R.blk_off[b] + pos];
    }
    __syncthreads();
#pragma unroll
    for (int ax = 0; ax < D; ++ax) {
        const int lev = level_of(G.N[ax]);
        for (int t = lev - 1; t >= 0; --t) {  // coarsest level first: parents already nodal
            hier_level(v, G, ax, t, 1.0);
            __syncthreads();
        }
    }
}

template <int D>
cudaError_t launch_recombine_d(const RecombPlan &R, const GridInfo *grids, const double *coef, int G, long long ntot,
                               int nb, const double *u, double *H, double *S, double *out, cudaStream_t s)
{
    const long long cta = (long long)G * nb, nodes = R.n_sparse * nb;
    if (cta > 0x7fffffffLL || (nodes + 255) / 256 > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    hier_kernel<D><<<(unsigned)cta, 256, 0, s>>>(grids, coef, G, ntot, u, H);
    gather_kernel<D><<<(unsigned)((nodes + 255) / 256), 256, 0, s>>>(R, grids, ntot, nb, H, S);
    dehier_kernel<D><<<(unsigned)cta, 256, 0, s>>>(R, grids, G, ntot, S, out);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_recombine(const RecombPlan &R, int d, const GridInfo *grids, const double *coef, int G,
                             long long ntot, int nb, const double *u, double *H, double *S, double *out,
                             cudaStream_t s)
{
    if (nb <= 0) return cudaSuccess;
    switch (d) {
    case 1: return launch_recombine_d<1>(R, grids, coef, G, ntot, nb, u, H, S, out, s);
    case 2: return launch_recombine_d<2>(R, grids, coef, G, ntot, nb, u, H, S, out, s);
    case 3: return launch_recombine_d<3>(R, grids, coef, G, ntot, nb, u, H, S, out, s);
    case 4: return launch_recombine_d<4>(R, grids, coef, G, ntot, nb, u, H, S, out, s);
    case 5: return launch_recombine_d<5>(R, grids, coef, G, ntot, nb, u, H, S, out, s);
    case 6: return launch_recombine_d<6>(R, grids, coef, G, ntot, nb, u, H, S, out, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace pit
