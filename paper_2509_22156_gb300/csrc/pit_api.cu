// C ABI of libpit (declared in include/pit.h): problem set-up, the batched
// backward-Euler propagator, time-sequential stepping, the MGRIT driver and
// the combination sum.  Method: Griebel, Schweitzer, Troska, arXiv 2509.22156.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
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
    int *d_order = nullptr;          // grids by decreasing size
    uint16_t *d_masks = nullptr;     // neighbour masks, packed like a state
    size_t smem_need[2] = {0, 0};    // per precision form
    bool planned[2] = {false, false};
    int threads[2][2] = {{0, 0}, {0, 0}};  // [prec][wide batch]; 0 = not tuned yet
    int forced_threads[2] = {0, 0};        // pit_tune override [wide batch]
    // workspaces
    DBuf w_in, w_out, w_pts, w_u, w_prm;
    DBuf m_U, m_R, m_UT, m_GC, m_res, m_UT1, m_GC1, m_T0, m_act, w_tune;
    std::vector<double> h_res;
    double *h_rmax = nullptr;  // pinned, G
    int *h_act = nullptr;      // pinned, G
    // kernel timing (pit_profile_enable / pit_profile_read)
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<int, size_t>> prof_recs;  // (family, first event index)
    long long prof_items = 0, prof_point_iters = 0, prof_point_passes = 0;
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

// Records a CUDA event pair around the next launch when profiling is on.
struct ProfScope {
    pit_problem *P;
    long long idx = -1;
    ProfScope(pit_problem *P_, int family) : P(P_)
    {
        if (!P->prof_on) return;
        while (P->ev_pool.size() < P->ev_used + 2) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return; }
            P->ev_pool.push_back(e);
        }
        idx = (long long)P->ev_used;
        P->ev_used += 2;
        P->prof_recs.push_back({family, (size_t)idx});
        cudaEventRecord(P->ev_pool[idx], P->stream);
    }
    ~ProfScope()
    {
        if (idx >= 0) cudaEventRecord(P->ev_pool[idx + 1], P->stream);
    }
};

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

// Shared memory the multi-step kernel needs for the largest grid.
pit_status plan(pit_problem *P, int prec)
{
    if (P->planned[prec]) return PIT_OK;
    size_t need = 0;
    int gmax = 0;
    for (int g = 0; g < P->G; ++g) {
        const size_t bytes = phi_smem_bytes(prec, P->desc.op, P->desc.d, P->info[g].n);
        if (bytes > need) { need = bytes; gmax = g; }
    }
    if (need > P->max_smem)
        return fail(PIT_ERR_UNSUPPORTED,
                    "grid %d (%d nodes) needs %zu bytes of shared memory for the on-chip solve in this precision "
                    "form; the device offers %zu",
                    gmax, P->info[gmax].n, need, P->max_smem);
    P->smem_need[prec] = need;
    P->planned[prec] = true;
    return PIT_OK;
}

// One multi-step launch (see StepArgs).
struct StepCall {
    double dt;
    int nb;
    int nsteps;
    const double *in;
    long long is;
    const double *f = nullptr;
    long long fs = 0;
    const double *g = nullptr;
    long long gs = 0, gst = 0;
    double *out_steps = nullptr;
    long long oss = 0, osst = 0;
    double *out_last = nullptr;
    long long ols = 0;
    double scale = 1.0;
    const double *h = nullptr;
    long long hs = 0;
    const double *cmp = nullptr;
    long long cs = 0;
    double *norms = nullptr;
};

StepArgs make_args(pit_problem *P, const pit_solve_opts &o, const StepCall &c, const int *active)
{
    StepArgs a;
    a.grids = P->d_grids;
    a.masks = P->d_masks;
    a.order = P->d_order;
    a.n_grids = P->G;
    a.n_batch = c.nb;
    a.nsteps = c.nsteps;
    a.dt = c.dt;
    a.in = c.in;
    a.in_stride = c.is;
    a.f = c.f;
    a.f_stride = c.fs;
    a.g = c.g;
    a.g_stride = c.gs;
    a.g_step = c.gst;
    a.out_steps = c.out_steps;
    a.os_stride = c.oss;
    a.os_step = c.osst;
    a.out_last = c.out_last;
    a.ol_stride = c.ols;
    a.out_scale = c.scale;
    a.h = c.h;
    a.h_stride = c.hs;
    a.cmp = c.cmp;
    a.cmp_stride = c.cs;
    a.norms = c.norms;
    a.active = active;
    a.faces = P->d_faces;
    a.op = P->op;
    a.rtol = o.rtol;
    a.maxit = o.maxit;
    a.inner_rtol = (float)o.inner_rtol;
    a.ir_maxit = o.ir_maxit;
    a.stats = P->d_stats;
    return a;
}

// Autotuner: the CTA size of a launch class (precision form x wide/narrow
// batch) is chosen once per problem by timing one backward-Euler step of the
// first real call of that class with every candidate, output to scratch.
pit_status tune(pit_problem *P, int prec, bool wide, const pit_solve_opts &o, const StepCall &c, const int *active)
{
    int &slot = P->threads[prec][wide ? 1 : 0];
    if (slot) return PIT_OK;
    if (P->forced_threads[wide ? 1 : 0]) {
        slot = P->forced_threads[wide ? 1 : 0];
        return PIT_OK;
    }
    const int cand[4] = {64, 128, 256, 512};
    CU(P->w_tune.ensure(sizeof(double) * P->ntot * c.nb));
    StepCall t;
    t.dt = c.dt;
    t.nb = c.nb;
    t.nsteps = 1;
    t.in = c.in;
    t.is = c.is;
    t.out_last = P->w_tune.d();
    t.ols = P->ntot;
    StepArgs a = make_args(P, o, t, active);
    a.stats = nullptr;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_t = 128;
    for (int k = 0; k < 4; ++k) {
        for (int rep = 0; rep < 2; ++rep) {  // first repetition warms up
            CU(cudaEventRecord(e0, P->stream));
            CU(launch_steps(prec, a, cand[k], P->smem_need[prec], P->stream));
            CU(cudaEventRecord(e1, P->stream));
        }
        CU(cudaEventSynchronize(e1));
        float ms = 0.0f;
        CU(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) { best = ms; best_t = cand[k]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    slot = best_t;
    return PIT_OK;
}

pit_status run_steps(pit_problem *P, const pit_solve_opts &o, const StepCall &c, const int *active)
{
    const int prec = o.prec == PIT_PREC_MIXED ? MIXED : PLAIN;
    TRY(plan(P, prec));
    if (c.nb <= 0 || c.nsteps <= 0) return PIT_OK;
    const bool wide = c.nb >= 8;
    TRY(tune(P, prec, wide, o, c, active));
    StepArgs a = make_args(P, o, c, active);
    ProfScope ps(P, 0);
    CU(launch_steps(prec, a, P->threads[prec][wide ? 1 : 0], P->smem_need[prec], P->stream));
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
    if (P->prof_on) {
        P->prof_items += (long long)s.items;
        P->prof_point_iters += (long long)s.point_iters;
        P->prof_point_passes += (long long)s.point_passes;
    }
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
    {
        std::vector<int> order(P->G);
        for (int g = 0; g < P->G; ++g) order[g] = g;
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return P->info[a].n > P->info[b].n; });
        CUB(cudaMalloc(&P->d_order, sizeof(int) * P->G));
        CUB(cudaMemcpy(P->d_order, order.data(), sizeof(int) * P->G, cudaMemcpyHostToDevice));
    }
    CUB(cudaMalloc(&P->d_masks, sizeof(uint16_t) * P->ntot));
    CUB(launch_masks(P->d_grids, P->G, d, P->d_masks, P->stream));
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
    cudaFree(P->d_order);
    cudaFree(P->d_masks);
    cudaFree(P->d_grids);
    cudaFree(P->d_coef);
    cudaFree(P->d_levels);
    cudaFree(P->d_hi);
    cudaFree(P->d_faces);
    cudaFree(P->d_stats);
    if (P->h_stats) cudaFreeHost(P->h_stats);
    if (P->h_rmax) cudaFreeHost(P->h_rmax);
    if (P->h_act) cudaFreeHost(P->h_act);
    DBuf *bufs[] = {&P->w_in, &P->w_out, &P->w_pts, &P->w_u,   &P->w_prm, &P->m_U,  &P->m_R, &P->m_UT,
                    &P->m_GC, &P->m_res, &P->m_UT1, &P->m_GC1, &P->m_T0,  &P->m_act, &P->w_tune};
    for (DBuf *b : bufs) b->release();
    for (cudaEvent_t e : P->ev_pool) cudaEventDestroy(e);
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
    {
        ProfScope ps(P, 3);
        CU(launch_initial(P->d_grids, P->G, P->op, P->d_hi, kind, P->w_prm.d(), n_params, target, P->stream));
    }
    if (!dev) CU(cudaMemcpyAsync(u0, target, sizeof(double) * P->ntot, cudaMemcpyDeviceToHost, P->stream));
    CU(cudaStreamSynchronize(P->stream));
    return PIT_OK;
}

pit_status pit_apply(pit_problem_t P, double dt, int n_batch, const double *pv, double *qv)
{
    if (!P || !pv || !qv || n_batch < 0) return fail(PIT_ERR_INVALID_ARG, "bad argument");
    if (!ptr_is_device(pv) || !ptr_is_device(qv)) return fail(PIT_ERR_INVALID_ARG, "p and q must be device memory");
    ProfScope ps(P, 3);
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
    const bool want = stats || P->prof_on;
    if (want) TRY(reset_stats(P));
    StepCall c;
    c.dt = dt;
    c.nb = n_batch;
    c.nsteps = 1;
    c.in = u_prev;
    c.is = P->ntot;
    c.f = f;
    c.fs = P->ntot;
    c.out_last = target;
    c.ols = P->ntot;
    TRY(run_steps(P, *opts, c, nullptr));
    if (alias) CU(cudaMemcpyAsync(u_next, target, bytes, cudaMemcpyDeviceToDevice, P->stream));
    if (want) {
        DevStats s;
        TRY(read_stats(P, s));
        if (stats) {
            fill_phi_stats(s, stats);
            TRY(status_of(s));
        }
    }
    return PIT_OK;
}

pit_status pit_sequential_solve(pit_problem_t P, const double *u0, double dt, int nsteps,
                                const pit_solve_opts *opts, double *uT, pit_phi_stats *stats)
{
    if (!P || !u0 || !uT || nsteps < 0) return fail(PIT_ERR_INVALID_ARG, "bad argument");
    if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(PIT_ERR_INVALID_ARG, "dt must be finite and >= 0");
    TRY(check_solve_opts(opts));
    const size_t bytes = sizeof(double) * P->ntot;
    const double *src;
    TRY(stage_in(P, P->w_in, u0, P->ntot, &src));
    const bool dev_out = ptr_is_device(uT);
    double *target = uT;
    if (!dev_out || src == uT) {
        CU(P->m_T0.ensure(bytes));
        target = P->m_T0.d();
    }
    TRY(reset_stats(P));
    if (nsteps == 0) {
        CU(cudaMemcpyAsync(target, src, bytes, cudaMemcpyDeviceToDevice, P->stream));
    } else {
        // every grid is one CTA that takes all nsteps steps on chip
        StepCall c;
        c.dt = dt;
        c.nb = 1;
        c.nsteps = nsteps;
        c.in = src;
        c.is = P->ntot;
        c.out_last = target;
        c.ols = P->ntot;
        TRY(run_steps(P, *opts, c, nullptr));
    }
    if (target != uT)
        CU(cudaMemcpyAsync(uT, target, bytes, dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, P->stream));
    DevStats s;
    TRY(read_stats(P, s));
    if (stats) fill_phi_stats(s, stats);
    TRY(status_of(s));
    return PIT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// MGRIT driver (Sec. 3.3, Alg. 2 with FCF relaxation; Alg. 3 per grid).
//
// Level 0 stores C-points only (Sec. 3.3.2): U[j] = u_{jm}, j = 0..Nc.  One
// cycle is four launches of the multi-step kernel:
//   FC    R[j+1]  = Phi^m(U[j])            (F-relaxation + C-relaxation)
//   F     UT[j]   = Phi^m(R[j]),  res[j] = ||UT[j] - R[j+1]||   (F-relaxation,
//                  C-point residual r_{j+1} = Phi(u_{(j+1)m-1}) - u_{(j+1)m})
//   FAS   GC[j]   = UT[j] - Phi_c(R[j])    (restricted residual + Phi_c of the
//                  restricted solution: the coarse right-hand side of Alg. 2)
//   sweep U[j+1]  = Phi_c(U[j]) + GC[j]    (coarse solve; its result is the
//                  corrected C-point, the F-points follow from the next FC)
// R[0] = U[0] = u0.  With three levels the sweep is replaced by one two-level
// cycle of the level-1 problem (points R[0..Nc], forcing GC), written into U.
namespace {

struct Mg {
    pit_problem *P;
    const pit_mgrit_opts *o;
    double dt;
    long long nt;
    const int *active;
};

// Coarse propagator of level 1: backward Euler with m dt, or m fine steps.
void coarse_call(Mg &M, StepCall &c, int level)
{
    if (level == 1 && M.o->coarse == PIT_COARSE_EXACT) {
        c.dt = M.dt;
        c.nsteps *= M.o->m;
    } else {
        double dtl = M.dt;
        for (int q = 0; q < level; ++q) dtl *= M.o->m;
        c.dt = dtl;
    }
}

// Two-level cycle of level 1 in a three-level hierarchy: level-1 points are V
// (read) -> W (written), Nc1 = N1/m intervals, forcing of level-1 point k is
// F[k-1]; the level-2 problem is solved by a sequential sweep.
pit_status mg_level1_cycle(Mg &M, const double *V, double *W, int N1, const double *F)
{
    pit_problem *P = M.P;
    const int m = M.o->m, Nc = N1 / m;
    const long long nt = M.nt, sm = (long long)m * nt;
    const pit_solve_opts &so = M.o->crs;
    CU(P->m_UT1.ensure(sizeof(double) * nt * Nc));
    CU(P->m_GC1.ensure(sizeof(double) * nt * Nc));
    double *UT1 = P->m_UT1.d(), *GC1 = P->m_GC1.d();
    if (W != V) CU(cudaMemcpyAsync(W, V, sizeof(double) * nt, cudaMemcpyDeviceToDevice, P->stream));
    const double dt1 = M.dt * m;
    // FC: F-points and C-point of every interval from the old C-points
    StepCall fc;
    fc.dt = dt1;
    fc.nb = Nc;
    fc.nsteps = m;
    fc.in = V;
    fc.is = sm;
    fc.g = F;
    fc.gs = sm;
    fc.gst = nt;
    fc.out_steps = W + nt;
    fc.oss = sm;
    fc.osst = nt;
    fc.out_last = W + sm;
    fc.ols = sm;
    TRY(run_steps(P, so, fc, M.active));
    // F-relaxation from the new C-points (F-points in place) and utilde
    StepCall fr = fc;
    fr.in = W;
    fr.out_last = UT1;
    fr.ols = nt;
    TRY(run_steps(P, so, fr, M.active));
    // coarse right-hand side and the level-2 sweep into the C-points of W
    StepCall gc;
    gc.dt = M.dt * m * m;
    gc.nb = Nc;
    gc.nsteps = 1;
    gc.in = W;
    gc.is = sm;
    gc.out_last = GC1;
    gc.ols = nt;
    gc.scale = -1.0;
    gc.h = UT1;
    gc.hs = nt;
    TRY(run_steps(P, so, gc, M.active));
    StepCall sw;
    sw.dt = M.dt * m * m;
    sw.nb = 1;
    sw.nsteps = Nc;
    sw.in = W;
    sw.is = nt;
    sw.g = GC1;
    sw.gst = nt;
    sw.out_steps = W + sm;
    sw.osst = sm;
    sw.out_last = W + (long long)Nc * sm;
    sw.ols = nt;
    TRY(run_steps(P, so, sw, M.active));
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
    if (o->levels == 3 && o->coarse == PIT_COARSE_EXACT)
        return fail(PIT_ERR_UNSUPPORTED, "the exact coarse propagator is a two-level option");
    const int G = P->G, m = o->m, Nc = o->nsteps / m;
    const long long nt = P->ntot;
    const size_t vb = sizeof(double) * nt;
    CU(P->m_U.ensure(vb * (Nc + 1)));
    CU(P->m_R.ensure(vb * (Nc + 1)));
    CU(P->m_UT.ensure(vb * Nc));
    CU(P->m_GC.ensure(vb * Nc));
    CU(P->m_res.ensure(sizeof(double) * G * Nc));
    CU(P->m_act.ensure(sizeof(int) * G));
    P->h_res.resize((size_t)G * Nc);
    double *U = P->m_U.d(), *R = P->m_R.d(), *UT = P->m_UT.d(), *GC = P->m_GC.d(), *res = P->m_res.d();
    int *act = (int *)P->m_act.p;
    const double *src;
    TRY(stage_in(P, P->w_in, u0, nt, &src));
    for (int j = 0; j <= Nc; ++j)
        CU(cudaMemcpyAsync(U + (long long)j * nt, src, vb, cudaMemcpyDeviceToDevice, P->stream));
    CU(cudaMemcpyAsync(R, src, vb, cudaMemcpyDeviceToDevice, P->stream));
    for (int g = 0; g < G; ++g) P->h_act[g] = 1;
    CU(cudaMemcpyAsync(act, P->h_act, sizeof(int) * G, cudaMemcpyHostToDevice, P->stream));
    TRY(reset_stats(P));

    Mg M{P, o, (o->t1 - o->t0) / o->nsteps, nt, act};
    pit_mgrit_stats st;
    memset(&st, 0, sizeof(st));
    int n_active = G, it = 0;
    while (n_active > 0 && it < o->maxit) {
        StepCall fc;  // FC relaxation
        fc.dt = M.dt;
        fc.nb = Nc;
        fc.nsteps = m;
        fc.in = U;
        fc.is = nt;
        fc.out_last = R + nt;
        fc.ols = nt;
        TRY(run_steps(P, o->fine, fc, act));
        StepCall fr = fc;  // F relaxation, utilde and the C-point residuals
        fr.in = R;
        fr.out_last = UT;
        fr.cmp = R + nt;
        fr.cs = nt;
        fr.norms = res;
        TRY(run_steps(P, o->fine, fr, act));
        CU(cudaMemcpyAsync(P->h_res.data(), res, sizeof(double) * G * Nc, cudaMemcpyDeviceToHost, P->stream));
        StepCall gc;  // coarse right-hand side
        gc.nb = Nc;
        gc.nsteps = 1;
        gc.in = R;
        gc.is = nt;
        gc.out_last = GC;
        gc.ols = nt;
        gc.scale = -1.0;
        gc.h = UT;
        gc.hs = nt;
        coarse_call(M, gc, 1);
        TRY(run_steps(P, o->crs, gc, act));
        if (o->levels == 3) {
            TRY(mg_level1_cycle(M, R, U, Nc, GC));
        } else if (o->coarse == PIT_COARSE_EXACT) {
            for (int j = 0; j < Nc; ++j) {
                StepCall sw;
                sw.nb = 1;
                sw.nsteps = 1;
                sw.in = U + (long long)j * nt;
                sw.is = nt;
                sw.out_last = U + (long long)(j + 1) * nt;
                sw.ols = nt;
                sw.h = GC + (long long)j * nt;
                sw.hs = nt;
                coarse_call(M, sw, 1);
                TRY(run_steps(P, o->crs, sw, act));
            }
        } else {
            StepCall sw;  // sequential coarse sweep, one CTA per grid
            sw.nb = 1;
            sw.nsteps = Nc;
            sw.in = U;
            sw.is = nt;
            sw.g = GC;
            sw.gst = nt;
            sw.out_steps = U + nt;
            sw.osst = nt;
            sw.out_last = U + (long long)Nc * nt;
            sw.ols = nt;
            coarse_call(M, sw, 1);
            TRY(run_steps(P, o->crs, sw, act));
        }
        CU(cudaStreamSynchronize(P->stream));
        double rmax = 0.0;
        n_active = 0;
        for (int g = 0; g < G; ++g) {
            if (!P->h_act[g]) continue;
            double r = 0.0;
            for (int j = 0; j < Nc; ++j) {
                const double v = P->h_res[(size_t)j * G + g];
                if (!(v <= r)) r = v;  // NaN propagates
            }
            if (!(r <= rmax)) rmax = r;
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
    st.point_iters = (long long)ds.point_iters;
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
    {
        ProfScope ps(P, 2);
        CU(launch_combine(P->d_grids, P->d_coef, P->d_levels, P->G, P->op, du, n_pts, dp, target, P->stream));
    }
    if (!dev_out) {
        CU(cudaMemcpyAsync(out, target, sizeof(double) * n_pts, cudaMemcpyDeviceToHost, P->stream));
        CU(cudaStreamSynchronize(P->stream));
    }
    return PIT_OK;
}

extern "C" pit_status pit_profile_enable(pit_problem_t P, int on)
{
    if (!P) return fail(PIT_ERR_INVALID_ARG, "NULL problem");
    CU(cudaStreamSynchronize(P->stream));
    P->prof_on = on != 0;
    P->ev_used = 0;
    P->prof_recs.clear();
    P->prof_items = P->prof_point_iters = P->prof_point_passes = 0;
    return PIT_OK;
}

extern "C" pit_status pit_profile_read(pit_problem_t P, pit_profile *out)
{
    if (!P || !out) return fail(PIT_ERR_INVALID_ARG, "NULL argument");
    CU(cudaStreamSynchronize(P->stream));
    memset(out, 0, sizeof(*out));
    for (const auto &r : P->prof_recs) {
        float ms = 0.0f;
        CU(cudaEventElapsedTime(&ms, P->ev_pool[r.second], P->ev_pool[r.second + 1]));
        out->launches[r.first] += 1;
        out->ms[r.first] += ms;
    }
    out->phi_items = P->prof_items;
    out->point_iters = P->prof_point_iters;
    out->point_passes = P->prof_point_passes;
    return PIT_OK;
}

// ---------------------------------------------------------------------------
// In-place backward-Euler step that allocates nothing (see pit.h).  The staging
// buffer that pit_phi_batch allocates for in-place steps is replaced by one
// file-scope device array of PIT_STATIC_SCRATCH_DOUBLES doubles, present on
// every device that loads the library until the process exits.  Host code
// only holds a stand-in for that array's name; the device address is looked
// up once per device with cudaGetSymbolAddress and cached.
static __device__ __align__(256) double g_static_scratch[PIT_STATIC_SCRATCH_DOUBLES];

namespace {
std::mutex g_static_mu;
double *g_static_ptr[256] = {nullptr};
}  // namespace

extern "C" pit_status pit_phi_batch_inplace_static(pit_problem_t P, double dt, int n_batch, double *u,
                                                   const double *f, const pit_solve_opts *opts,
                                                   pit_phi_stats *stats)
{
    if (!P || !u || n_batch < 0) return fail(PIT_ERR_INVALID_ARG, "bad argument");
    if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(PIT_ERR_INVALID_ARG, "dt must be finite and >= 0");
    TRY(check_solve_opts(opts));
    const long long count = (long long)n_batch * P->ntot;
    if (count > (long long)PIT_STATIC_SCRATCH_DOUBLES)
        return fail(PIT_ERR_INVALID_ARG,
                    "n_batch * n_total = %lld exceeds the static scratch of %d doubles of "
                    "pit_phi_batch_inplace_static",
                    count, PIT_STATIC_SCRATCH_DOUBLES);
    if (!ptr_is_device(u) || (f && !ptr_is_device(f))) return fail(PIT_ERR_INVALID_ARG, "u and f must be device memory");
    if (n_batch == 0) return PIT_OK;
    int dev = -1;
    CU(cudaGetDevice(&dev));
    if (dev != P->device) return fail(PIT_ERR_INVALID_ARG, "the problem's device (%d) is not current (%d)", P->device, dev);
    if (dev < 0 || dev >= 256) return fail(PIT_ERR_UNSUPPORTED, "device ordinal %d", dev);
    double *scratch;
    {
        std::lock_guard<std::mutex> lock(g_static_mu);
        if (!g_static_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess || !p)
                return fail(PIT_ERR_CUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
            g_static_ptr[dev] = (double *)p;
        }
        scratch = g_static_ptr[dev];
    }
    const int prec = opts->prec == PIT_PREC_MIXED ? MIXED : PLAIN;
    TRY(plan(P, prec));
    const bool wide = n_batch >= 8;
    const int threads = P->threads[prec][wide ? 1 : 0] ? P->threads[prec][wide ? 1 : 0] : 128;
    StepCall c;
    c.dt = dt;
    c.nb = n_batch;
    c.nsteps = 1;
    c.in = u;
    c.is = P->ntot;
    c.f = f;
    c.fs = P->ntot;
    c.out_last = scratch;  // every node of every item is written: nothing needs clearing
    c.ols = P->ntot;
    StepArgs a = make_args(P, *opts, c, nullptr);
    if (stats) CU(cudaMemsetAsync(P->d_stats, 0, sizeof(DevStats), P->stream));
    else a.stats = nullptr;
    CU(launch_steps(prec, a, threads, P->smem_need[prec], P->stream));
    CU(cudaMemcpyAsync(u, scratch, sizeof(double) * count, cudaMemcpyDeviceToDevice, P->stream));
    if (stats) {
        CU(cudaMemcpyAsync(P->h_stats, P->d_stats, sizeof(DevStats), cudaMemcpyDeviceToHost, P->stream));
        CU(cudaStreamSynchronize(P->stream));
        const DevStats s = *P->h_stats;
        fill_phi_stats(s, stats);
        TRY(status_of(s));
    }
    return PIT_OK;
}
