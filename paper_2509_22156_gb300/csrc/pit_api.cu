// C ABI of libpit (declared in include/pit.h): problem set-up, the batched
// backward-Euler propagator, time-sequential stepping, the MGRIT driver and
// the combination sum.  Method: Griebel, Schweitzer, Troska, arXiv 2509.22156.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pit_internal.cuh"

using namespace pit;

namespace {

thread_local std::string g_err;

pit_status fail(pit_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CU(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(e_ == cudaErrorMemoryAllocation ? PIT_ERR_OOM : PIT_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                       \
    } while (0)

#define TRY(expr)                          \
    do {                                   \
        pit_status s_ = (expr);            \
        if (s_ != PIT_OK) return s_;       \
    } while (0)

// Device buffer that only grows.
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t want)
    {
        if (want <= bytes) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&p, want);
        if (e == cudaSuccess) bytes = want;
        return e;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    double *d() const { return (double *)p; }
};

struct Bucket {
    int threads;
    size_t smem;
    int n;           // grids
    int *d_grids;    // device list
};

}  // namespace

struct pit_problem {
    pit_problem_desc desc;
    cudaStream_t stream = nullptr;
    int device = 0;
    size_t max_smem = 0;
    int G = 0;
    long long ntot = 0;
    std::vector<int> levels;      // G*d
    std::vector<double> coef;     // G
    std::vector<long long> off;   // G+1
    std::vector<GridInfo> info;   // G
    OpParams op;
    GridInfo *d_grids = nullptr;
    double *d_coef = nullptr;
    int *d_levels = nullptr;
    double *d_hi = nullptr;
    double *d_faces = nullptr;
    DevStats *d_stats = nullptr;
    DevStats *h_stats = nullptr;  // pinned
    std::vector<Bucket> buckets[2];
    bool planned[2] = {false, false};
    // workspaces
    DBuf w_in, w_out, w_pts, w_u, w_prm;
    DBuf m_U, m_W0, m_W1, m_UT, m_GC, m_res, m_rmax, m_UT1, m_GC1, m_T0, m_T1, m_act;
    double *h_rmax = nullptr;  // pinned, G
    int *h_act = nullptr;      // pinned, G
};

namespace {

int ptr_is_device(const void *p)
{
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Component grids of Eq. "combination_technique_solution": for w = 0..d-1 all
// l with l_i >= L0 and |l|_1 = L + d - 1 - w, lexicographically ascending.
void enumerate_levels(int d, int L, int L0, std::vector<int> &lev, std::vector<int> &layer)
{
    lev.clear();
    layer.clear();
    for (int w = 0; w < d; ++w) {
        const int target = L + d - 1 - w;
        if (target < d * L0) continue;
        // odometer over the first d-1 components; the last one is fixed by the sum
        std::vector<int> l(d, L0);
        for (;;) {
            int rest = target;
            for (int i = 0; i < d - 1; ++i) rest -= l[i];
            if (rest >= L0) {
                l[d - 1] = rest;
                lev.insert(lev.end(), l.begin(), l.end());
                layer.push_back(w);
            }
            // advance the odometer (last of the first d-1 digits fastest)
            int i = d - 2;
            while (i >= 0) {
                int used = 0;
                for (int k = 0; k <= i; ++k) used += l[k];
                if (used + 1 + (d - 1 - i) * L0 <= target) {
                    ++l[i];
                    for (int k = i + 1; k < d - 1; ++k) l[k] = L0;
                    break;
                }
                --i;
            }
            if (i < 0) break;
        }
    }
}

double binomial(int a, int b)
{
    double r = 1.0;
    for (int k = 1; k <= b; ++k) r = r * (a - b + k) / k;
    return r;
}

pit_status check_solve_opts(const pit_solve_opts *o)
{
    if (!o) return fail(PIT_ERR_INVALID_ARG, "solve options are NULL");
    if (o->prec != PIT_PREC_FP64 && o->prec != PIT_PREC_MIXED)
        return fail(PIT_ERR_INVALID_ARG, "unknown precision %d", o->prec);
    if (!(o->rtol >= 0.0) || o->maxit < 1) return fail(PIT_ERR_INVALID_ARG, "rtol must be >= 0 and maxit >= 1");
    if (o->prec == PIT_PREC_MIXED && (!(o->inner_rtol > 0.0 && o->inner_rtol < 1.0) || o->ir_maxit < 1))
        return fail(PIT_ERR_INVALID_ARG, "mixed precision needs 0 < inner_rtol < 1 and ir_maxit >= 1");
    return PIT_OK;
}

// Threads of the CTA that owns a grid of n nodes: about four nodes per
// thread, a whole number of warps, at most 512 (the kernels' launch bound).
int threads_for(int n)
{
    int t = (n + 3) / 4;
    t = (t + 31) & ~31;
    if (t < 32) t = 32;
    if (t > 512) t = 512;
    return t;
}

pit_status plan(pit_problem *P, int prec)
{
    if (P->planned[prec]) return PIT_OK;
    std::vector<std::vector<int>> groups;
    std::vector<int> thr;
    std::vector<size_t> sm;
    for (int g = 0; g < P->G; ++g) {
        const int n = P->info[g].n;
        const int t = threads_for(n);
        const size_t bytes = phi_smem_bytes(prec, P->desc.op, P->desc.d, n);
        if (bytes > P->max_smem)
            return fail(PIT_ERR_UNSUPPORTED,
                        "grid %d (%d nodes) needs %zu bytes of shared memory for the on-chip solve; this device "
                        "offers %zu",
                        g, n, bytes, P->max_smem);
        size_t k = 0;
        while (k < thr.size() && thr[k] != t) ++k;
        if (k == thr.size()) {
            thr.push_back(t);
            sm.push_back(0);
            groups.emplace_back();
        }
        groups[k].push_back(g);
        if (bytes > sm[k]) sm[k] = bytes;
    }
    for (size_t k = 0; k < groups.size(); ++k) {
        Bucket B;
        B.threads = thr[k];
        B.smem = sm[k];
        B.n = (int)groups[k].size();
        CU(cudaMalloc(&B.d_grids, sizeof(int) * B.n));
        CU(cudaMemcpy(B.d_grids, groups[k].data(), sizeof(int) * B.n, cudaMemcpyHostToDevice));
        P->buckets[prec].push_back(B);
    }
    P->planned[prec] = true;
    return PIT_OK;
}

struct PhiCall {
    double dt;
    int nb;
    const double *in;
    long long is;
    const double *f;
    long long fs;
    const double *gp;
    long long gs;
    double scale;
    double *out;
    long long os;
};

pit_status run_phi(pit_problem *P, const pit_solve_opts &o, const PhiCall &c, const int *active)
{
    const int prec = o.prec == PIT_PREC_MIXED ? MIXED : PLAIN;
    TRY(plan(P, prec));
    PhiArgs a;
    a.grids = P->d_grids;
    a.n_batch = c.nb;
    a.dt = c.dt;
    a.in = c.in;
    a.in_stride = c.is;
    a.f = c.f;
    a.f_stride = c.fs;
    a.gpost = c.gp;
    a.g_stride = c.gs;
    a.post_scale = c.scale;
    a.out = c.out;
    a.out_stride = c.os;
    a.active = active;
    a.faces = P->d_faces;
    a.op = P->op;
    a.rtol = o.rtol;
    a.maxit = o.maxit;
    a.inner_rtol = (float)o.inner_rtol;
    a.ir_maxit = o.ir_maxit;
    a.stats = P->d_stats;
    for (const Bucket &B : P->buckets[prec]) {
        a.bucket_grids = B.d_grids;
        a.n_bucket = B.n;
        CU(launch_phi_bucket(prec, a, B.threads, B.smem, P->stream));
    }
    return PIT_OK;
}

pit_status reset_stats(pit_problem *P)
{
    CU(cudaMemsetAsync(P->d_stats, 0, sizeof(DevStats), P->stream));
    return PIT_OK;
}

pit_status read_stats(pit_problem *P, DevStats &s)
{
    CU(cudaMemcpyAsync(P->h_stats, P->d_stats, sizeof(DevStats), cudaMemcpyDeviceToHost, P->stream));
    CU(cudaStreamSynchronize(P->stream));
    s = *P->h_stats;
    return PIT_OK;
}

void fill_phi_stats(const DevStats &s, pit_phi_stats *st)
{
    st->n_items = (int)s.items;
    st->n_failed = s.n_failed;
    st->max_iters = s.max_iters;
    st->sum_iters = (long long)s.sum_iters;
    st->max_refine = s.max_refine;
    st->status = s.worst;
}

pit_status status_of(const DevStats &s)
{
    if (s.n_failed == 0) return PIT_OK;
    return fail((pit_status)s.worst, "%d backward-Euler solves failed (worst status %d)", s.n_failed, s.worst);
}

// Brings a host-or-device input vector onto the device.
pit_status stage_in(pit_problem *P, DBuf &buf, const double *src, size_t count, const double **dev)
{
    if (ptr_is_device(src)) {
        *dev = src;
        return PIT_OK;
    }
    CU(buf.ensure(count * sizeof(double)));
    CU(cudaMemcpyAsync(buf.p, src, count * sizeof(double), cudaMemcpyHostToDevice, P->stream));
    *dev = buf.d();
    return PIT_OK;
}

}  // namespace

extern "C" {

const char *pit_last_error(void) { return g_err.c_str(); }

pit_status pit_problem_create(const pit_problem_desc *desc, void *stream, pit_problem_t *out)
{
    if (!desc || !out) return fail(PIT_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    const int d = desc->d;
    if (d < 1 || d > PIT_MAX_DIM) return fail(PIT_ERR_INVALID_ARG, "d = %d outside 1..%d", d, PIT_MAX_DIM);
    if (desc->level0 < 1 || desc->level_n < desc->level0 || desc->level_n > 30)
        return fail(PIT_ERR_INVALID_ARG, "levels must satisfy 1 <= level0 <= level_n <= 30");
    if (desc->op < PIT_OP_HEAT || desc->op > PIT_OP_OU) return fail(PIT_ERR_INVALID_ARG, "unknown operator %d", desc->op);
    for (int i = 0; i < d; ++i)
        if (!(desc->hi[i] > desc->lo[i])) return fail(PIT_ERR_INVALID_ARG, "empty box on axis %d", i);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(PIT_ERR_CUDA, "no CUDA device");
    }
    pit_problem *P = new pit_problem();
    P->desc = *desc;
    P->stream = (cudaStream_t)stream;
    cudaGetDevice(&P->device);
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device);
    // static shared memory of the kernels (grid record, reduction buffers) is reserved
    P->max_smem = smem_optin > 4096 ? (size_t)smem_optin - 4096 : 0;

    std::vector<int> layer;
    enumerate_levels(d, desc->level_n, desc->level0, P->levels, layer);
    P->G = (int)layer.size();
    if (P->G == 0) {
        delete P;
        return fail(PIT_ERR_INVALID_ARG, "the grid set is empty");
    }
    P->off.assign(P->G + 1, 0);
    P->coef.resize(P->G);
    P->info.resize(P->G);
    for (int g = 0; g < P->G; ++g) {
        GridInfo &I = P->info[g];
        memset(&I, 0, sizeof(I));
        long long n = 1;
        for (int i = 0; i < d; ++i) {
            const int l = P->levels[g * d + i];
            I.N[i] = (1 << l) - 1;
            I.h[i] = (desc->hi[i] - desc->lo[i]) / (double)(1LL << l);
            n *= I.N[i];
        }
        if (n > 0x7fffffffLL) {
            delete P;
            return fail(PIT_ERR_UNSUPPORTED, "grid %d has %lld nodes", g, n);
        }
        int s = 1;
        for (int i = d - 1; i >= 0; --i) {
            I.S[i] = s;
            s *= I.N[i];
        }
        I.n = (int)n;
        I.off = P->off[g];
        P->off[g + 1] = P->off[g] + n;
        const int w = layer[g];
        P->coef[g] = (w % 2 ? -1.0 : 1.0) * binomial(d - 1, w);
    }
    P->ntot = P->off[P->G];
    memset(&P->op, 0, sizeof(P->op));
    P->op.op = desc->op;
    P->op.d = d;
    for (int i = 0; i < d; ++i) P->op.lo[i] = desc->lo[i];
    P->op.theta = desc->theta;
    P->op.sigma = desc->sigma;
    P->op.vamp = desc->vamp;

    auto bail = [&](pit_status st) {
        pit_problem_destroy(P);
        return st;
    };
#define CUB(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return bail(fail(e_ == cudaErrorMemoryAllocation ? PIT_ERR_OOM : PIT_ERR_CUDA, "%s: %s", #call, \
                             cudaGetErrorString(e_)));                                              \
    } while (0)
    CUB(phi_kernels_init(P->max_smem));
    CUB(cudaMalloc(&P->d_grids, sizeof(GridInfo) * P->G));
    CUB(cudaMemcpy(P->d_grids, P->info.data(), sizeof(GridInfo) * P->G, cudaMemcpyHostToDevice));
    CUB(cudaMalloc(&P->d_coef, sizeof(double) * P->G));
    CUB(cudaMemcpy(P->d_coef, P->coef.data(), sizeof(double) * P->G, cudaMemcpyHostToDevice));
    CUB(cudaMalloc(&P->d_levels, sizeof(int) * P->G * d));
    CUB(cudaMemcpy(P->d_levels, P->levels.data(), sizeof(int) * P->G * d, cudaMemcpyHostToDevice));
    CUB(cudaMalloc(&P->d_hi, sizeof(double) * PIT_MAX_DIM));
    CUB(cudaMemcpy(P->d_hi, desc->hi, sizeof(double) * PIT_MAX_DIM, cudaMemcpyHostToDevice));
    CUB(cudaMalloc(&P->d_stats, sizeof(DevStats)));
    CUB(cudaMallocHost(&P->h_stats, sizeof(DevStats)));
    CUB(cudaMallocHost(&P->h_rmax, sizeof(double) * P->G));
    CUB(cudaMallocHost(&P->h_act, sizeof(int) * P->G));
    if (desc->op == PIT_OP_VARHEAT) {
        CUB(cudaMalloc(&P->d_faces, sizeof(double) * P->ntot * 2 * d));
        CUB(launch_faces(P->d_grids, P->G, P->op, P->d_faces, P->stream));
    }
    CUB(cudaStreamSynchronize(P->stream));
#undef CUB
    *out = P;
    return PIT_OK;
}

pit_status pit_problem_destroy(pit_problem_t P)
{
    if (!P) return PIT_OK;
    cudaStreamSynchronize(P->stream);
    for (int k = 0; k < 2; ++k)
        for (Bucket &B : P->buckets[k]) cudaFree(B.d_grids);
    cudaFree(P->d_grids);
    cudaFree(P->d_coef);
    cudaFree(P->d_levels);
    cudaFree(P->d_hi);
    cudaFree(P->d_faces);
    cudaFree(P->d_stats);
    if (P->h_stats) cudaFreeHost(P->h_stats);
    if (P->h_rmax) cudaFreeHost(P->h_rmax);
    if (P->h_act) cudaFreeHost(P->h_act);
    DBuf *bufs[] = {&P->w_in, &P->w_out, &P->w_pts, &P->w_u, &P->w_prm, &P->m_U, &P->m_W0, &P->m_W1, &P->m_UT,
                    &P->m_GC, &P->m_res, &P->m_rmax, &P->m_UT1, &P->m_GC1, &P->m_T0, &P->m_T1, &P->m_act};
    for (DBuf *b : bufs) b->release();
    delete P;
    return PIT_OK;
}

pit_status pit_problem_info(pit_problem_t P, int *n_grids, long long *n_total, int *levels, double *coef,
                            long long *offsets)
{
    if (!P) return fail(PIT_ERR_INVALID_ARG, "NULL problem");
    if (n_grids) *n_grids = P->G;
    if (n_total) *n_total = P->ntot;
    if (levels) memcpy(levels, P->levels.data(), sizeof(int) * P->levels.size());
    if (coef) memcpy(coef, P->coef.data(), sizeof(double) * P->G);
    if (offsets) memcpy(offsets, P->off.data(), sizeof(long long) * (P->G + 1));
    return PIT_OK;
}

pit_status pit_sample_initial(pit_problem_t P, int kind, const double *params, int n_params, double *u0)
{
    if (!P || !params || !u0) return fail(PIT_ERR_INVALID_ARG, "NULL argument");
    const int d = P->desc.d;
    if (kind == 0) {
        if (n_params < 1) return fail(PIT_ERR_INVALID_ARG, "missing mode count");
        const int K = (int)params[0];
        if (K < 0 || n_params < 1 + K * (d + 1)) return fail(PIT_ERR_INVALID_ARG, "need 1 + K(d+1) parameters");
    } else if (kind == 1) {
        if (n_params < 2 * d) return fail(PIT_ERR_INVALID_ARG, "need 2d parameters");
        for (int i = 0; i < d; ++i)
            if (!(params[d + i] > 0.0)) return fail(PIT_ERR_INVALID_ARG, "std must be positive");
    } else {
        return fail(PIT_ERR_INVALID_ARG, "unknown initial-value kind %d", kind);
    }
    CU(P->w_prm.ensure(sizeof(double) * n_params));
    CU(cudaMemcpyAsync(P->w_prm.p, params, sizeof(double) * n_params, cudaMemcpyHostToDevice, P->stream));
    const bool dev = ptr_is_device(u0);
    double *target = u0;
    if (!dev) {
        CU(P->w_u.ensure(sizeof(double) * P->ntot));
        target = P->w_u.d();
    }
    CU(launch_initial(P->d_grids, P->G, P->op, P->d_hi, kind, P->w_prm.d(), n_params, target, P->stream));
    if (!dev) CU(cudaMemcpyAsync(u0, target, sizeof(double) * P->ntot, cudaMemcpyDeviceToHost, P->stream));
    CU(cudaStreamSynchronize(P->stream));
    return PIT_OK;
}

pit_status pit_apply(pit_problem_t P, double dt, int n_batch, const double *pv, double *qv)
{
    if (!P || !pv || !qv || n_batch < 0) return fail(PIT_ERR_INVALID_ARG, "bad argument");
    if (!ptr_is_device(pv) || !ptr_is_device(qv)) return fail(PIT_ERR_INVALID_ARG, "p and q must be device memory");
    CU(launch_apply(P->d_grids, P->G, P->ntot, n_batch, dt, pv, qv, P->d_faces, P->op, P->stream));
    return PIT_OK;
}

pit_status pit_phi_batch(pit_problem_t P, double dt, int n_batch, const double *u_prev, const double *f,
                         double *u_next, const pit_solve_opts *opts, pit_phi_stats *stats)
{
    if (!P || !u_prev || !u_next || n_batch < 0) return fail(PIT_ERR_INVALID_ARG, "bad argument");
    if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(PIT_ERR_INVALID_ARG, "dt must be finite and >= 0");
    TRY(check_solve_opts(opts));
    if (!ptr_is_device(u_prev) || !ptr_is_device(u_next) || (f && !ptr_is_device(f)))
        return fail(PIT_ERR_INVALID_ARG, "u_prev, f and u_next must be device memory");
    if (n_batch == 0) return PIT_OK;
    const size_t bytes = sizeof(double) * P->ntot * n_batch;
    const char *a0 = (const char *)u_prev, *b0 = (const char *)u_next;
    const bool alias = (a0 == b0);
    if (!alias && a0 < b0 + bytes && b0 < a0 + bytes)
        return fail(PIT_ERR_INVALID_ARG, "u_next overlaps u_prev without being the same vector");
    double *target = u_next;
    if (alias) {
        CU(P->w_out.ensure(bytes));
        target = P->w_out.d();
    }
    if (stats) TRY(reset_stats(P));
    PhiCall c{dt, n_batch, u_prev, P->ntot, f, P->ntot, nullptr, 0, 1.0, target, P->ntot};
    TRY(run_phi(P, *opts, c, nullptr));
    if (alias) CU(cudaMemcpyAsync(u_next, target, bytes, cudaMemcpyDeviceToDevice, P->stream));
    if (stats) {
        DevStats s;
        TRY(read_stats(P, s));
        fill_phi_stats(s, stats);
        TRY(status_of(s));
    }
    return PIT_OK;
}

pit_status pit_sequential_solve(pit_problem_t P, const double *u0, double dt, int nsteps,
                                const pit_solve_opts *opts, double *uT, pit_phi_stats *stats)
{
    if (!P || !u0 || !uT || nsteps < 0) return fail(PIT_ERR_INVALID_ARG, "bad argument");
    TRY(check_solve_opts(opts));
    const size_t bytes = sizeof(double) * P->ntot;
    CU(P->m_T0.ensure(bytes));
    CU(P->m_T1.ensure(bytes));
    const double *src;
    TRY(stage_in(P, P->w_in, u0, P->ntot, &src));
    CU(cudaMemcpyAsync(P->m_T0.p, src, bytes, cudaMemcpyDeviceToDevice, P->stream));
    TRY(reset_stats(P));
    double *a = P->m_T0.d(), *b = P->m_T1.d();
    for (int s = 0; s < nsteps; ++s) {
        PhiCall c{dt, 1, a, P->ntot, nullptr, 0, nullptr, 0, 1.0, b, P->ntot};
        TRY(run_phi(P, *opts, c, nullptr));
        std::swap(a, b);
    }
    CU(cudaMemcpyAsync(uT, a, bytes, ptr_is_device(uT) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       P->stream));
    DevStats s;
    TRY(read_stats(P, s));
    if (stats) fill_phi_stats(s, stats);
    TRY(status_of(s));
    return PIT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// MGRIT driver (Sec. 3.3, Alg. 2 with FCF relaxation; Alg. 3 per grid).
namespace {

struct Mg {
    pit_problem *P;
    const pit_mgrit_opts *o;
    double dt;
    long long nt;
    const int *active;
};

// One step of level `lev` for nb states: out_k = scale * Phi_lev(in_k) + gp_k.
pit_status mg_step(Mg &M, int lev, int nb, const double *in, long long is, const double *gp, long long gs,
                   double scale, double *out, long long os)
{
    pit_problem *P = M.P;
    if (nb <= 0) return PIT_OK;
    if (lev == 1 && M.o->coarse == PIT_COARSE_EXACT) {
        // m fine steps; intermediate states in T0/T1
        const size_t bytes = sizeof(double) * M.nt * nb;
        CU(P->m_T0.ensure(bytes));
        CU(P->m_T1.ensure(bytes));
        const double *src = in;
        long long sst = is;
        double *bufs[2] = {P->m_T0.d(), P->m_T1.d()};
        for (int s = 0; s < M.o->m; ++s) {
            const bool last = (s == M.o->m - 1);
            double *dst = last ? out : bufs[s & 1];
            PhiCall c{M.dt, nb, src, sst, nullptr, 0, last ? gp : nullptr, gs, last ? scale : 1.0, dst,
                      last ? os : M.nt};
            TRY(run_phi(P, M.o->fine, c, M.active));
            src = dst;
            sst = M.nt;
        }
        return PIT_OK;
    }
    double dtl = M.dt;
    for (int q = 0; q < lev; ++q) dtl *= M.o->m;
    const pit_solve_opts &so = lev == 0 ? M.o->fine : M.o->crs;
    PhiCall c{dtl, nb, in, is, nullptr, 0, gp, gs, scale, out, os};
    return run_phi(P, so, c, M.active);
}

// Level-1 two-level cycle of a three-level hierarchy: the level-1 points are
// the level-0 C-points V[0..N1] (all stored), forcing of point k is F[k-1];
// coarsest level solved by a sequential sweep.
pit_status mg_level1_cycle(Mg &M, double *V, int N1, const double *F)
{
    pit_problem *P = M.P;
    const int m = M.o->m, Nc = N1 / m;
    const long long nt = M.nt, sm = (long long)m * nt;
    auto Vp = [&](int k) { return V + (long long)k * nt; };
    auto Fp = [&](int k) { return F + (long long)(k - 1) * nt; };  // forcing of level-1 point k >= 1
    for (int pass = 0; pass < 2; ++pass) {
        for (int i = 1; i < m; ++i) TRY(mg_step(M, 1, Nc, Vp(i - 1), sm, Fp(i), sm, 1.0, Vp(i), sm));
        if (pass == 0) TRY(mg_step(M, 1, Nc, Vp(m - 1), sm, Fp(m), sm, 1.0, Vp(m), sm));
    }
    CU(P->m_UT1.ensure(sizeof(double) * nt * Nc));
    CU(P->m_GC1.ensure(sizeof(double) * nt * Nc));
    double *UT1 = P->m_UT1.d(), *GC1 = P->m_GC1.d();
    TRY(mg_step(M, 1, Nc, Vp(m - 1), sm, Fp(m), sm, 1.0, UT1, nt));          // utilde_j, j = 1..Nc
    TRY(mg_step(M, 2, Nc, Vp(0), sm, UT1, nt, -1.0, GC1, nt));               // gc_j = utilde_j - Phi_2(v_{(j-1)m})
    for (int j = 1; j <= Nc; ++j)
        TRY(mg_step(M, 2, 1, Vp((j - 1) * m), nt, GC1 + (long long)(j - 1) * nt, nt, 1.0, Vp(j * m), nt));
    return PIT_OK;
}

}  // namespace

extern "C" pit_status pit_mgrit_solve(pit_problem_t P, const double *u0, const pit_mgrit_opts *o, double *uT,
                                      pit_mgrit_stats *stats)
{
    auto t_start = std::chrono::steady_clock::now();
    if (!P || !u0 || !uT || !o) return fail(PIT_ERR_INVALID_ARG, "NULL argument");
    TRY(check_solve_opts(&o->fine));
    TRY(check_solve_opts(&o->crs));
    if (o->m < 2 || o->levels < 2 || o->levels > 3 || o->nsteps < 1 || o->maxit < 1 || !(o->tol >= 0.0) ||
        !(o->t1 > o->t0))
        return fail(PIT_ERR_INVALID_ARG, "need m >= 2, levels in {2,3}, nsteps >= 1, maxit >= 1, tol >= 0, t1 > t0");
    if (o->coarse != PIT_COARSE_IMPLICIT && o->coarse != PIT_COARSE_EXACT)
        return fail(PIT_ERR_UNSUPPORTED, "coarse propagator %d is not available", o->coarse);
    long long div = o->m;
    if (o->levels == 3) div *= o->m;
    if (o->nsteps % div != 0) return fail(PIT_ERR_INVALID_ARG, "nsteps must be a multiple of m^(levels-1)");
    const int G = P->G, m = o->m, Nc = o->nsteps / m;
    const long long nt = P->ntot;
    const size_t vb = sizeof(double) * nt;
    CU(P->m_U.ensure(vb * (Nc + 1)));
    CU(P->m_W0.ensure(vb * Nc));
    CU(P->m_W1.ensure(vb * Nc));
    CU(P->m_UT.ensure(vb * Nc));
    CU(P->m_GC.ensure(vb * Nc));
    CU(P->m_res.ensure(sizeof(double) * G * Nc));
    CU(P->m_rmax.ensure(sizeof(double) * G));
    CU(P->m_act.ensure(sizeof(int) * G));
    double *U = P->m_U.d(), *UT = P->m_UT.d(), *GC = P->m_GC.d();
    double *W[2] = {P->m_W0.d(), P->m_W1.d()};
    int *act = (int *)P->m_act.p;
    const double *src;
    TRY(stage_in(P, P->w_in, u0, nt, &src));
    for (int j = 0; j <= Nc; ++j)
        CU(cudaMemcpyAsync(U + (long long)j * nt, src, vb, cudaMemcpyDeviceToDevice, P->stream));
    for (int g = 0; g < G; ++g) P->h_act[g] = 1;
    CU(cudaMemcpyAsync(act, P->h_act, sizeof(int) * G, cudaMemcpyHostToDevice, P->stream));
    TRY(reset_stats(P));

    Mg M{P, o, (o->t1 - o->t0) / o->nsteps, nt, act};
    pit_mgrit_stats st;
    memset(&st, 0, sizeof(st));
    std::vector<int> cycles(G, 0);
    int n_active = G, it = 0;
    while (n_active > 0 && it < o->maxit) {
        // FCF relaxation; only the C-points are stored, W holds the F-values
        int cur = 0;
        for (int pass = 0; pass < 2; ++pass) {
            TRY(mg_step(M, 0, Nc, U, nt, nullptr, 0, 1.0, W[0], nt));
            cur = 0;
            for (int i = 2; i < m; ++i) {
                TRY(mg_step(M, 0, Nc, W[cur], nt, nullptr, 0, 1.0, W[cur ^ 1], nt));
                cur ^= 1;
            }
            if (pass == 0) TRY(mg_step(M, 0, Nc, W[cur], nt, nullptr, 0, 1.0, U + nt, nt));  // C-relaxation
        }
        // utilde_j = Phi(u_{jm-1}) and the C-point residuals r_j = utilde_j - u_{jm}
        TRY(mg_step(M, 0, Nc, W[cur], nt, nullptr, 0, 1.0, UT, nt));
        CU(launch_resid_norms(P->d_grids, G, nt, Nc, UT, nt, U + nt, nt, act, P->m_res.d(), P->stream));
        CU(launch_resid_max(G, Nc, P->m_res.d(), act, P->m_rmax.d(), P->stream));
        CU(cudaMemcpyAsync(P->h_rmax, P->m_rmax.d(), sizeof(double) * G, cudaMemcpyDeviceToHost, P->stream));
        // coarse FAS problem: gc_j = utilde_j - Phi_c(u_{(j-1)m}); v_j = Phi_c(v_{j-1}) + gc_j
        TRY(mg_step(M, 1, Nc, U, nt, UT, nt, -1.0, GC, nt));
        if (o->levels == 2) {
            for (int j = 0; j < Nc; ++j)
                TRY(mg_step(M, 1, 1, U + (long long)j * nt, nt, GC + (long long)j * nt, nt, 1.0,
                            U + (long long)(j + 1) * nt, nt));
        } else {
            TRY(mg_level1_cycle(M, U, Nc, GC));
        }
        CU(cudaStreamSynchronize(P->stream));
        double rmax = 0.0;
        n_active = 0;
        for (int g = 0; g < G; ++g) {
            if (!P->h_act[g]) continue;
            const double r = P->h_rmax[g];
            ++cycles[g];
            if (!(r <= rmax) ) rmax = r;
            if (r <= o->tol) P->h_act[g] = 0;
            else ++n_active;
        }
        if (it < PIT_MAX_HIST) st.res_hist[it] = rmax;
        ++it;
        if (n_active > 0) CU(cudaMemcpyAsync(act, P->h_act, sizeof(int) * G, cudaMemcpyHostToDevice, P->stream));
        if (!(rmax == rmax)) break;  // NaN: stop at once
    }
    CU(cudaMemcpyAsync(uT, U + (long long)Nc * nt, vb,
                       ptr_is_device(uT) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, P->stream));
    DevStats ds;
    TRY(read_stats(P, ds));
    st.max_cycles = it;
    st.n_converged = G - n_active;
    st.phi_items = (long long)ds.items;
    st.krylov_iters = (long long)ds.sum_iters;
    st.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    if (stats) *stats = st;
    TRY(status_of(ds));
    if (n_active > 0) return fail(PIT_ERR_NOCONV, "%d grids did not meet tol within %d cycles", n_active, it);
    return PIT_OK;
}

extern "C" pit_status pit_combine(pit_problem_t P, const double *u, int n_pts, const double *pts, double *out)
{
    if (!P || !u || !pts || !out || n_pts < 0) return fail(PIT_ERR_INVALID_ARG, "bad argument");
    if (n_pts == 0) return PIT_OK;
    const double *du, *dp;
    TRY(stage_in(P, P->w_u, u, P->ntot, &du));
    TRY(stage_in(P, P->w_pts, pts, (size_t)n_pts * P->desc.d, &dp));
    const bool dev_out = ptr_is_device(out);
    double *target = out;
    if (!dev_out) {
        CU(P->w_out.ensure(sizeof(double) * n_pts));
        target = P->w_out.d();
    }
    CU(launch_combine(P->d_grids, P->d_coef, P->d_levels, P->G, P->op, du, n_pts, dp, target, P->stream));
    if (!dev_out) {
        CU(cudaMemcpyAsync(out, target, sizeof(double) * n_pts, cudaMemcpyDeviceToHost, P->stream));
        CU(cudaStreamSynchronize(P->stream));
    }
    return PIT_OK;
}
