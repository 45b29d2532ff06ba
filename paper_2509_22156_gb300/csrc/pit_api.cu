// C ABI of libpit (declared in include/pit.h): problem set-up, the batched
// backward-Euler propagator, time-sequential stepping, the MGRIT driver and
// the combination sum.  Method: Griebel, Schweitzer, Troska, arXiv 2509.22156.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
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

// Every device allocation of the library goes through dev_malloc, which counts
// it (process-wide; reported by pit_profile_read as device_allocs).
std::atomic<long long> g_dev_allocs{0};
cudaError_t dev_malloc(void **p, size_t bytes)
{
    g_dev_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMalloc(p, bytes);
}
template <typename T>
cudaError_t dev_malloc(T **p, size_t bytes)
{
    return dev_malloc((void **)p, bytes);
}

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
        cudaError_t e = dev_malloc(&p, want);
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

// A lane of the MGRIT driver: a subset of the grids with its own streams,
// launch plan and convergence state.  Grids are independent until the
// combination (Alg. 3), so the cycles of several lanes run concurrently and
// the latency-bound coarse sweep of one lane overlaps the relaxation of the
// others.
struct pit_lane {
    std::vector<int> grids;
    cudaStream_t s = nullptr;
    cudaStream_t sides[NPART - 1] = {};  // the launch parts other than the first
    cudaEvent_t fork = nullptr, join = nullptr, done = nullptr;
    bool planned[NPREC] = {};
    int n_cls[NPREC][2] = {};
    int split[NPREC][NBKT + 1] = {};  // class-0 positions where the shared-memory buckets start
    int *d_order_cls[NPREC][2] = {};
    int *d_act = nullptr;     // G flags, zero outside the lane
    int *h_act = nullptr;     // pinned, G
    double *h_res = nullptr;  // pinned, G x Nc
    size_t h_res_cap = 0;
    // per-solve state
    int it = 0, n_active = 0;
    bool busy = false;
    int tm = 1;  // steps per common step of the lane's grids (their own time partition)
};

struct pit_problem {
    pit_problem_desc desc;
    cudaStream_t stream = nullptr;
    int device = 0;
    size_t max_smem = 0;
    int n_sm = 0;  // streaming multiprocessors of the device
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
    DevStats *d_stats = nullptr;  // [0]: batches of 8 or more entries per grid, [1]: fewer
    DevStats *h_stats = nullptr;  // pinned, the same two
    int *d_order = nullptr;          // grids by decreasing size
    uint16_t *d_masks = nullptr;     // neighbour masks, packed like a state
    // launch plan per precision form: class 0 = grids whose FP64 state fits in
    // shared memory, class 1 = larger grids (MIXED only: state in global memory)
    bool planned[NPREC] = {};
    int n_cls[NPREC][2] = {};
    int *d_order_cls[NPREC][2] = {};
    std::vector<int> h_order_cls[NPREC][2];
    size_t smem_cls[NPREC][2] = {};
    size_t smem_need[NPREC] = {};    // class 0 (used by the allocation-free step)
    // class 0 runs as up to NBKT launches, one per shared-memory bucket: grids
    // needing more than half of the largest grid's shared memory, then more
    // than a quarter, and so on, each launch with its own allocation, so that
    // the CTAs of smaller grids pack more densely on an SM
    int split[NPREC][NBKT + 1] = {};
    size_t smem_bkt[NPREC][NBKT] = {};
    int threads[NPREC][2][NPART] = {};  // [prec][wide batch][part: buckets, then global state]; 0 = not tuned
    int forced_threads[2] = {0, 0};  // override [wide batch]
    cudaStream_t sides[NPART - 1] = {};  // streams of the launch parts beside the first
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    DBuf w_xg;                       // FP64 state of class-1 items
    DBuf w_scr;                      // FP32 scratch of extrapolated steps in the FP32 form
    std::vector<pit_lane> lanes;     // MGRIT lanes (built on first use)
    std::vector<int> lane_assign;    // grid -> lane when given explicitly; empty: balanced
    // workspaces
    DBuf w_in, w_out, w_pts, w_u, w_prm;
    DBuf w_part;  // partial sums of the chunked combination sum
    DBuf m_U, m_R, m_UT, m_GC, m_res, m_UT1, m_GC1, m_T0, m_act, w_tune, m_Z, m_E;
    std::vector<double> h_res;
    double *h_rmax = nullptr;  // pinned, G
    int *h_act = nullptr;      // pinned, G
    // learned coarse propagator
    bool have_net = false, net_accepted = false;
    NetWeights h_net;  // BF16-rounded parameters as used by the kernels
    DBuf n_master, n_m, n_v, n_w, n_rows, n_loss, n_act, n_items, n_U, n_Y, n_grad, n_tmp, n_prm;
    // kernel timing (pit_profile_enable / pit_profile_read)
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<int, size_t>> prof_recs;  // (family, first event index)
    long long prof_items = 0, prof_point_iters = 0, prof_point_passes = 0, prof_point_steps = 0;
    long long prof_kernels[4] = {0, 0, 0, 0};  // kernel launches per profile family
    long long prof_fam_iters[2] = {0, 0}, prof_fam_passes[2] = {0, 0}, prof_fam_steps[2] = {0, 0};
    long long prof_allocs0 = 0;  // process-wide device allocation count at pit_profile_enable
    // recombination (Sec. 2.2.2): sparse-grid block plan, built on first use
    bool rc_ready = false;
    RecombPlan rc{};
    int *rc_lam = nullptr, *rc_list_off = nullptr, *rc_list = nullptr, *rc_lookup = nullptr;
    long long *rc_off = nullptr;
    DBuf rc_H, rc_S, rc_cur;
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
// Counts kernel launches per profile family while profiling is enabled.
static inline void count_kernels(pit_problem *P, int family, long long n = 1)
{
    if (P->prof_on) P->prof_kernels[family] += n;
}

struct ProfScope {
    pit_problem *P;
    cudaStream_t s;
    long long idx = -1;
    ProfScope(pit_problem *P_, int family, cudaStream_t s_ = nullptr) : P(P_), s(s_ ? s_ : P_->stream)
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
        cudaEventRecord(P->ev_pool[idx], s);
    }
    ~ProfScope()
    {
        if (idx >= 0) cudaEventRecord(P->ev_pool[idx + 1], s);
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
    if (o->prec != PIT_PREC_FP64 && o->prec != PIT_PREC_MIXED && o->prec != PIT_PREC_FP32 &&
        o->prec != PIT_PREC_MIXED_PAIR)
        return fail(PIT_ERR_INVALID_ARG, "unknown precision %d", o->prec);
    if (!(o->rtol >= 0.0) || o->maxit < 1) return fail(PIT_ERR_INVALID_ARG, "rtol must be >= 0 and maxit >= 1");
    if (o->precond < PIT_PRECOND_DEFAULT || o->precond > PIT_PRECOND_JACOBI)
        return fail(PIT_ERR_INVALID_ARG, "unknown preconditioner %d", o->precond);
    if (o->guess < PIT_GUESS_DEFAULT || o->guess > PIT_GUESS_EXTRAPOLATE)
        return fail(PIT_ERR_INVALID_ARG, "unknown initial guess %d", o->guess);
    if ((o->prec == PIT_PREC_MIXED || o->prec == PIT_PREC_MIXED_PAIR) &&
        (!(o->inner_rtol > 0.0 && o->inner_rtol < 1.0) || o->ir_maxit < 1))
        return fail(PIT_ERR_INVALID_ARG, "mixed precision needs 0 < inner_rtol < 1 and ir_maxit >= 1");
    return PIT_OK;
}

// Launch plan of a precision form: grids whose on-chip state fits in shared
// memory form class 0; the others keep their FP64 vectors in global memory
// (class 1: the state x and b in the mixed form, x and the Krylov vectors in
// the FP64 form; the FP32 form has no class 1).  Class 0 lists its grids by
// decreasing shared-memory need, class 1 by decreasing size.
size_t grid_smem_bytes(const pit_problem *P, int prec, int g)
{
    const GridInfo &I = P->info[g];
    int na = 1;
    for (int i = 0; i < P->desc.d; ++i) na = I.N[i] > na ? I.N[i] : na;
    return phi_smem_bytes(prec, P->desc.op, P->desc.d, I.n, na);
}

pit_status plan(pit_problem *P, int prec)
{
    if (P->planned[prec]) return PIT_OK;
    if (prec == PAIR && (P->desc.op == PIT_OP_OU || P->desc.op == PIT_OP_LSDE || P->desc.op == PIT_OP_CME))
        return fail(PIT_ERR_UNSUPPORTED, "the pair precision form is implemented for the symmetric operators only");
    std::vector<int> order(P->G);
    for (int g = 0; g < P->G; ++g) order[g] = g;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return P->info[a].n > P->info[b].n; });
    std::vector<int> cls[2];
    size_t need[2] = {0, 0};
    for (int g : order) {
        const int n = P->info[g].n;
        const size_t bytes = grid_smem_bytes(P, prec, g);
        if (bytes <= P->max_smem) {
            cls[0].push_back(g);
            need[0] = bytes > need[0] ? bytes : need[0];
            continue;
        }
        // (class 1 of the FP32 form runs the refinement form's global-state kernel)
        const size_t bx = phi_smem_bytes_xg(prec, P->desc.op, P->desc.d, n);
        if (bx > P->max_smem)
            return fail(PIT_ERR_UNSUPPORTED,
                        "grid %d (%d nodes) needs %zu bytes of shared memory for the on-chip solve in this precision "
                        "form; the device offers %zu",
                        g, n, bx, P->max_smem);
        cls[1].push_back(g);
        need[1] = bx > need[1] ? bx : need[1];
    }
    {
        // buckets over class 0 in decreasing order of shared-memory need
        std::stable_sort(cls[0].begin(), cls[0].end(), [&](int a, int b) {
            return grid_smem_bytes(P, prec, a) > grid_smem_bytes(P, prec, b);
        });
        const int n0 = (int)cls[0].size();
        int k = 0;
        P->split[prec][0] = 0;
        for (int q = 0; q < NBKT; ++q) {
            P->smem_bkt[prec][q] = k < n0 ? grid_smem_bytes(P, prec, cls[0][k]) : 0;
            if (q == NBKT - 1) k = n0;
            else
                while (k < n0 && (grid_smem_bytes(P, prec, cls[0][k]) << (q + 1)) > need[0]) ++k;
            P->split[prec][q + 1] = k;
        }
    }
    for (int c = 0; c < 2; ++c) {
        P->n_cls[prec][c] = (int)cls[c].size();
        P->h_order_cls[prec][c] = cls[c];
        P->smem_cls[prec][c] = need[c];
        if (!cls[c].empty()) {
            CU(dev_malloc(&P->d_order_cls[prec][c], sizeof(int) * cls[c].size()));
            CU(cudaMemcpy(P->d_order_cls[prec][c], cls[c].data(), sizeof(int) * cls[c].size(), cudaMemcpyHostToDevice));
        }
    }
    P->smem_need[prec] = need[0];
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
    long long fs = 0, fst = 0;
    int fdiv = 1;
    const double *g = nullptr;
    long long gs = 0, gst = 0;
    double *out_steps = nullptr;
    long long oss = 0, osst = 0;
    double *out_last = nullptr;
    long long ols = 0;
    double scale = 1.0;
    double hscale = 1.0;
    const double *h = nullptr;
    long long hs = 0;
    const double *hstep = nullptr;  // added to every stored state (per-step stride hsst)
    long long hss = 0, hsst = 0;
    const double *cmp = nullptr;
    long long cs = 0;
    double *norms = nullptr;
    const double *guess = nullptr;
    long long gus = 0, gust = 0;
    int inexact = 0;  // fixed-iteration solves (residual mode): the iteration caps are not failures
    int sdirk = 0;    // two-stage SDIRK steps with stage step dt (coarse propagator PIT_COARSE_SDIRK2)
    int ext = 0;      // extrapolated backward-Euler steps with half step dt (PIT_COARSE_EXTRAP)
};

StepArgs make_args(pit_problem *P, const pit_solve_opts &o, const StepCall &c, const int *active)
{
    StepArgs a;
    a.item0 = 0;
    a.grids = P->d_grids;
    a.masks = P->d_masks;
    a.order = P->d_order;
    a.n_order = P->G;
    a.n_grids = P->G;
    a.n_total = P->ntot;
    a.xg = nullptr;
    a.bg = nullptr;
    a.n_batch = c.nb;
    a.nsteps = c.nsteps;
    a.dt = c.dt;
    a.in = c.in;
    a.in_stride = c.is;
    a.f = c.f;
    a.f_stride = c.fs;
    a.f_step = c.fst;
    a.f_div = c.fdiv;
    a.g = c.g;
    a.g_stride = c.gs;
    a.g_step = c.gst;
    a.out_steps = c.out_steps;
    a.os_stride = c.oss;
    a.os_step = c.osst;
    a.out_last = c.out_last;
    a.ol_stride = c.ols;
    a.out_scale = c.scale;
    a.out_hscale = c.hscale;
    a.h = c.h;
    a.h_stride = c.hs;
    a.hs = c.hstep;
    a.hs_stride = c.hss;
    a.hs_step = c.hsst;
    a.cmp = c.cmp;
    a.cmp_stride = c.cs;
    a.norms = c.norms;
    a.guess = c.guess;
    a.guess_stride = c.gus;
    a.guess_step = c.gust;
    a.active = active;
    a.faces = P->d_faces;
    a.op = P->op;
    a.rtol = o.rtol;
    a.maxit = o.maxit;
    a.inner_rtol = (float)o.inner_rtol;
    a.ir_maxit = o.ir_maxit;
    a.inexact = c.inexact;
    a.precond = o.precond;
    a.predict = o.guess != PIT_GUESS_PREVIOUS;
    a.sdirk = c.sdirk;
    a.ext = c.ext;
    // (the FP32 form's extrapolated steps keep u_n and U2 in a global slab per
    // item; run_steps and lanes_prime size it before any such launch)
    a.scr = (c.ext && prec_form(o.prec) == SINGLE) ? (float *)P->w_scr.p : nullptr;
    a.stats = P->d_stats;
    return a;
}

// Autotuner: the CTA size of a launch class (precision form x wide/narrow
// batch x grid class) is chosen once per problem by timing one backward-Euler
// step of the first real call of that class with every candidate, output to
// scratch.
// One launch part of a precision form (of a lane, when given): 0 = class-0
// grids above half the largest shared-memory need, 2 = the other class-0
// grids, 1 = class 1 (state in global memory).
struct PartView {
    const int *order;
    int n;
    size_t smem;
    bool xg;
};
PartView part_view(const pit_problem *P, const pit_lane *L, int prec, int part)
{
    if (part < NBKT) {
        const int *sp = L ? L->split[prec] : P->split[prec];
        int *o0 = L ? L->d_order_cls[prec][0] : P->d_order_cls[prec][0];
        return {o0 ? o0 + sp[part] : nullptr, sp[part + 1] - sp[part], P->smem_bkt[prec][part], false};
    }
    return {L ? L->d_order_cls[prec][1] : P->d_order_cls[prec][1], L ? L->n_cls[prec][1] : P->n_cls[prec][1],
            P->smem_cls[prec][1], true};
}

pit_status tune(pit_problem *P, int prec, bool wide, int cls, const pit_solve_opts &o, const StepCall &c,
                const int *active)
{
    int &slot = P->threads[prec][wide ? 1 : 0][cls];
    if (slot) return PIT_OK;
    const PartView v = part_view(P, nullptr, prec, cls);
    if (v.n <= 0) return PIT_OK;
    if (P->forced_threads[wide ? 1 : 0]) {
        slot = P->forced_threads[wide ? 1 : 0];
        return PIT_OK;
    }
    const int cand[4] = {64, 128, 256, 512};
    CU(P->w_tune.ensure(sizeof(double) * P->ntot * c.nb));
    // the trial keeps the call's inputs (a correction sweep starts from zero
    // and is driven by its forcing) and writes only scratch; it runs several
    // steps, so that the refinement forms' carried residual (every step but
    // the first) weighs as in the real launch: wide batches (relaxation
    // intervals) 4, narrow ones (sequential sweeps, latency bound) 8
    StepCall t;
    t.dt = c.dt;
    t.nb = c.nb;
    const int trial = wide ? 4 : 8;
    t.nsteps = c.nsteps < trial ? c.nsteps : trial;
    t.in = c.in;
    t.is = c.is;
    t.f = c.f;
    t.fs = c.fs;
    t.fst = c.fst;
    t.fdiv = c.fdiv;
    t.g = c.g;
    t.gs = c.gs;
    t.gst = c.gst;
    t.guess = c.guess;
    t.gus = c.gus;
    t.gust = c.gust;
    t.out_last = P->w_tune.d();
    t.ols = P->ntot;
    StepArgs a = make_args(P, o, t, active);
    a.stats = nullptr;
    a.order = v.order;
    a.n_order = v.n;
    if (v.xg) {
        a.xg = P->w_xg.d();
        a.bg = a.xg + (long long)c.nb * P->ntot;
    }
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_t = 128;
    for (int k = 0; k < 4; ++k) {
        for (int rep = 0; rep < 3; ++rep) {  // first repetition warms up; the last is timed
            CU(cudaEventRecord(e0, P->stream));
            CU(launch_steps(prec, a, cand[k], v.smem, P->stream, v.xg));
            count_kernels(P, wide ? 0 : 1);
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

// One multi-step launch of every grid (of a lane, when given): class 0 on the
// problem's (lane's) stream and, when present, class 1 (state in global
// memory) concurrently on the side stream, joined before returning.
pit_status run_steps(pit_problem *P, const pit_solve_opts &o, const StepCall &c, const int *active,
                     const pit_lane *L = nullptr)
{
    const int prec = prec_form(o.prec);
    TRY(plan(P, prec));
    if (c.nb <= 0 || c.nsteps <= 0) return PIT_OK;
    if (L && !L->planned[prec]) return fail(PIT_ERR_INVALID_ARG, "lane without a launch plan");
    const bool wide = c.nb >= 8;
    PartView v[NPART];
    int n_parts = 0;
    for (int q = 0; q < NPART; ++q) {
        v[q] = part_view(P, L, prec, q);
        if (v[q].n > 0) ++n_parts;
    }
    // the FP64 global-state variant of the table operators indexes its table
    // rows with a 32-bit stride of n_batch x n_total
    if (v[NBKT].n > 0 && prec == PLAIN && P->desc.op != PIT_OP_HEAT && (long long)c.nb * P->ntot >= (1LL << 31))
        return fail(PIT_ERR_UNSUPPORTED, "batch of %d states of %lld nodes too large for the FP64 global-state "
                                         "solver of this operator", c.nb, P->ntot);
    // (a lane's workspaces and CTA sizes are prepared before its first launch)
    if (v[NBKT].n > 0 && !L)
        CU(P->w_xg.ensure(sizeof(double) * P->ntot * (size_t)c.nb * xg_slabs(prec, P->desc.op, P->desc.d)));
    if (c.ext && prec == SINGLE && !L) CU(P->w_scr.ensure(sizeof(float) * P->ntot * (size_t)c.nb));
    if (c.ext && prec == SINGLE && P->w_scr.bytes < sizeof(float) * P->ntot * (size_t)c.nb)
        return fail(PIT_ERR_INVALID_ARG, "extrapolated FP32 steps without their scratch");
    if (!L)
        for (int q = 0; q < NPART; ++q) TRY(tune(P, prec, wide, q, o, c, active));
    cudaStream_t st[NPART];
    st[0] = L ? L->s : P->stream;
    for (int q = 1; q < NPART; ++q) st[q] = L ? L->sides[q - 1] : P->sides[q - 1];
    cudaEvent_t ef = L ? L->fork : P->ev_fork, ej = L ? L->join : P->ev_join;
    StepArgs a = make_args(P, o, c, active);
    a.stats = P->d_stats + (wide ? 0 : 1);  // counters per kernel family
    ProfScope ps(P, wide ? 0 : 1, st[0]);
    const bool fork = n_parts > 1;
    if (fork) {
        CU(cudaEventRecord(ef, st[0]));
        for (int q = 1; q < NPART; ++q)
            if (v[q].n > 0) CU(cudaStreamWaitEvent(st[q], ef, 0));
    }
    // a single part runs on the main stream; several run concurrently, the
    // largest grids on the main stream, the other parts each on its own stream
    for (int q = 0; q < NPART; ++q) {
        if (v[q].n <= 0) continue;
        StepArgs b = a;
        b.order = v[q].order;
        b.n_order = v[q].n;
        if (v[q].xg) {
            b.xg = P->w_xg.d();
            b.bg = b.xg + (long long)c.nb * P->ntot;
        }
        cudaStream_t sq = fork ? st[q] : st[0];
        CU(launch_steps(prec, b, P->threads[prec][wide ? 1 : 0][q], v[q].smem, sq, v[q].xg));
        count_kernels(P, wide ? 0 : 1);
    }
    if (fork) {
        for (int q = 1; q < NPART; ++q) {
            if (v[q].n <= 0) continue;
            CU(cudaEventRecord(ej, st[q]));
            CU(cudaStreamWaitEvent(st[0], ej, 0));
        }
    }
    return PIT_OK;
}

// Network application with StepArgs semantics; activations in shared memory
// when the largest grid fits, else in per-CTA global slabs (launch split into
// chunks of CTAs so that the slabs stay below 4 GiB).
pit_status run_net(pit_problem *P, const StepCall &c, const int *active)
{
    if (c.nb <= 0 || c.nsteps <= 0) return PIT_OK;
    pit_solve_opts dummy{PIT_PREC_FP64, 0.0, 1, 0.5, 1, PIT_PRECOND_DEFAULT};
    StepArgs a = make_args(P, dummy, c, active);
    int nmax = 0;
    for (const GridInfo &I : P->info) nmax = I.n > nmax ? I.n : nmax;
    const long long items = (long long)c.nb * P->G;
    size_t smem = net_smem_bytes(nmax);
    ProfScope ps(P, 0);
    if (smem <= P->max_smem) {
        CU(launch_net_steps(a, P->h_net, nullptr, 0, smem, P->stream, (int)items));
        count_kernels(P, 0);
        return PIT_OK;
    }
    const long long slab = (long long)net_act_floats(nmax, false);
    const long long limit = (4LL << 30) / (long long)(slab * sizeof(float));
    const long long chunk = items < limit ? items : (limit > 0 ? limit : 1);
    CU(P->n_act.ensure(sizeof(float) * (size_t)(slab * chunk)));
    smem = (size_t)((nmax + 3) & ~3) * 12 + 16;
    for (long long k0 = 0; k0 < items; k0 += chunk) {
        a.item0 = (int)k0;
        const long long cnt = (items - k0) < chunk ? (items - k0) : chunk;
        CU(launch_net_steps(a, P->h_net, (float *)P->n_act.p, slab, smem, P->stream, (int)cnt));
        count_kernels(P, 0);
    }
    return PIT_OK;
}

pit_status reset_stats(pit_problem *P)
{
    CU(cudaMemsetAsync(P->d_stats, 0, 2 * sizeof(DevStats), P->stream));
    return PIT_OK;
}

// Counters of both kernel families since the last reset, merged.
pit_status read_stats(pit_problem *P, DevStats &s)
{
    CU(cudaMemcpyAsync(P->h_stats, P->d_stats, 2 * sizeof(DevStats), cudaMemcpyDeviceToHost, P->stream));
    CU(cudaStreamSynchronize(P->stream));
    const DevStats &a = P->h_stats[0], &b = P->h_stats[1];
    s = a;
    s.sum_iters += b.sum_iters;
    s.items += b.items;
    s.point_iters += b.point_iters;
    s.point_passes += b.point_passes;
    s.point_steps += b.point_steps;
    s.max_iters = b.max_iters > s.max_iters ? b.max_iters : s.max_iters;
    s.n_failed += b.n_failed;
    s.max_refine = b.max_refine > s.max_refine ? b.max_refine : s.max_refine;
    s.worst = b.worst > s.worst ? b.worst : s.worst;
    if (P->prof_on) {
        P->prof_items += (long long)s.items;
        P->prof_point_iters += (long long)s.point_iters;
        P->prof_point_passes += (long long)s.point_passes;
        P->prof_point_steps += (long long)s.point_steps;
        for (int f = 0; f < 2; ++f) {
            P->prof_fam_iters[f] += (long long)P->h_stats[f].point_iters;
            P->prof_fam_passes[f] += (long long)P->h_stats[f].point_passes;
            P->prof_fam_steps[f] += (long long)P->h_stats[f].point_steps;
        }
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
    if (desc->op < PIT_OP_HEAT || desc->op > PIT_OP_CME) return fail(PIT_ERR_INVALID_ARG, "unknown operator %d", desc->op);
    if (desc->op == PIT_OP_LSDE)
        for (int k = 0; k < d * d; ++k)
            if (!std::isfinite(desc->drift[k]) || !std::isfinite(desc->diffusion[k]))
                return fail(PIT_ERR_INVALID_ARG, "drift and diffusion matrices must be finite");
    if (desc->drift_scheme != PIT_DRIFT_UPWIND && desc->drift_scheme != PIT_DRIFT_CENTRAL)
        return fail(PIT_ERR_INVALID_ARG, "unknown drift scheme %d", desc->drift_scheme);
    if (desc->drift_scheme != PIT_DRIFT_UPWIND && desc->op != PIT_OP_LSDE && desc->op != PIT_OP_CME)
        return fail(PIT_ERR_INVALID_ARG, "the central drift flux is offered for the linear-SDE and CME operators only");
    if (desc->op == PIT_OP_CME)
        for (int i = 0; i < d; ++i) {
            if (!std::isfinite(desc->cme_prod[i]) || !std::isfinite(desc->cme_sat[i]) ||
                !std::isfinite(desc->cme_exp[i]) || !std::isfinite(desc->cme_deg[i]))
                return fail(PIT_ERR_INVALID_ARG, "CME rates of species %d must be finite", i);
            if (desc->cme_prod[i] < 0.0 || desc->cme_deg[i] < 0.0 || !(desc->cme_sat[i] > 0.0))
                return fail(PIT_ERR_INVALID_ARG, "CME rates of species %d: production and degradation >= 0, "
                            "saturation > 0", i);
            if (!(desc->lo[i] >= 0.0))
                return fail(PIT_ERR_INVALID_ARG, "the CME box must lie in x >= 0 (axis %d)", i);
        }
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
    cudaDeviceGetAttribute(&P->n_sm, cudaDevAttrMultiProcessorCount, P->device);

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
    if (desc->op == PIT_OP_LSDE)
        for (int k = 0; k < d * d; ++k) {
            P->op.A[k] = desc->drift[k];
            P->op.H[k] = desc->diffusion[k];
        }
    P->op.central = desc->drift_scheme == PIT_DRIFT_CENTRAL ? 1 : 0;
    if (desc->op == PIT_OP_CME)
        for (int i = 0; i < d; ++i) {
            P->op.cp[i] = desc->cme_prod[i];
            P->op.cs[i] = desc->cme_sat[i];
            P->op.cb[i] = desc->cme_exp[i];
            P->op.cg[i] = desc->cme_deg[i];
        }

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
    for (auto &sq : P->sides) CUB(cudaStreamCreateWithFlags(&sq, cudaStreamNonBlocking));
    CUB(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
    CUB(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
    CUB(phi_kernels_init(P->max_smem));
    CUB(net_kernels_init(P->max_smem));
    CUB(dev_malloc(&P->d_grids, sizeof(GridInfo) * P->G));
    CUB(cudaMemcpy(P->d_grids, P->info.data(), sizeof(GridInfo) * P->G, cudaMemcpyHostToDevice));
    CUB(dev_malloc(&P->d_coef, sizeof(double) * P->G));
    CUB(cudaMemcpy(P->d_coef, P->coef.data(), sizeof(double) * P->G, cudaMemcpyHostToDevice));
    CUB(dev_malloc(&P->d_levels, sizeof(int) * P->G * d));
    CUB(cudaMemcpy(P->d_levels, P->levels.data(), sizeof(int) * P->G * d, cudaMemcpyHostToDevice));
    CUB(dev_malloc(&P->d_hi, sizeof(double) * PIT_MAX_DIM));
    CUB(cudaMemcpy(P->d_hi, desc->hi, sizeof(double) * PIT_MAX_DIM, cudaMemcpyHostToDevice));
    CUB(dev_malloc(&P->d_stats, 2 * sizeof(DevStats)));
    CUB(cudaMallocHost(&P->h_stats, 2 * sizeof(DevStats)));
    CUB(cudaMallocHost(&P->h_rmax, sizeof(double) * P->G));
    CUB(cudaMallocHost(&P->h_act, sizeof(int) * P->G));
    {
        std::vector<int> order(P->G);
        for (int g = 0; g < P->G; ++g) order[g] = g;
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return P->info[a].n > P->info[b].n; });
        CUB(dev_malloc(&P->d_order, sizeof(int) * P->G));
        CUB(cudaMemcpy(P->d_order, order.data(), sizeof(int) * P->G, cudaMemcpyHostToDevice));
    }
    CUB(dev_malloc(&P->d_masks, sizeof(uint16_t) * P->ntot));
    CUB(launch_masks(P->d_grids, P->G, d, P->d_masks, P->stream));
    if (desc->op == PIT_OP_VARHEAT) {
        CUB(dev_malloc(&P->d_faces, sizeof(double) * P->ntot * 2 * d));
        CUB(launch_faces(P->d_grids, P->G, P->op, P->d_faces, P->stream));
    }
    // launch plans of every precision form the problem supports, so that no
    // later call needs to allocate for one (pit_phi_batch_inplace_static
    // relies on this); a form that plan() rejects stays unplanned and is
    // rejected again, with its message, by the call that asks for it
    for (int prec = 0; prec < NPREC; ++prec) {
        const pit_status st = plan(P, prec);
        if (st == PIT_ERR_CUDA || st == PIT_ERR_OOM) return bail(st);
    }
    g_err.clear();
    CUB(cudaStreamSynchronize(P->stream));
#undef CUB
    *out = P;
    return PIT_OK;
}

pit_status pit_problem_destroy(pit_problem_t P)
{
    if (!P) return PIT_OK;
    cudaStreamSynchronize(P->stream);
    for (pit_lane &L : P->lanes) {
        if (L.s) cudaStreamSynchronize(L.s);
        for (auto sq : L.sides)
            if (sq) cudaStreamSynchronize(sq);
        for (int p = 0; p < NPREC; ++p)
            for (int c = 0; c < 2; ++c) cudaFree(L.d_order_cls[p][c]);
        cudaFree(L.d_act);
        cudaFreeHost(L.h_act);
        cudaFreeHost(L.h_res);
        if (L.s) cudaStreamDestroy(L.s);
        for (auto sq : L.sides)
            if (sq) cudaStreamDestroy(sq);
        if (L.fork) cudaEventDestroy(L.fork);
        if (L.join) cudaEventDestroy(L.join);
        if (L.done) cudaEventDestroy(L.done);
    }
    P->lanes.clear();
    cudaFree(P->d_order);
    cudaFree(P->d_masks);
    for (int p = 0; p < NPREC; ++p)
        for (int c = 0; c < 2; ++c) cudaFree(P->d_order_cls[p][c]);
    for (auto sq : P->sides)
        if (sq) {
            cudaStreamSynchronize(sq);
            cudaStreamDestroy(sq);
        }
    if (P->ev_fork) cudaEventDestroy(P->ev_fork);
    if (P->ev_join) cudaEventDestroy(P->ev_join);
    cudaFree(P->rc_lam);
    cudaFree(P->rc_off);
    cudaFree(P->rc_list_off);
    cudaFree(P->rc_list);
    cudaFree(P->rc_lookup);
    P->rc_H.release();
    P->rc_S.release();
    P->rc_cur.release();
    cudaFree(P->d_grids);
    cudaFree(P->d_coef);
    cudaFree(P->d_levels);
    cudaFree(P->d_hi);
    cudaFree(P->d_faces);
    cudaFree(P->d_stats);
    if (P->h_stats) cudaFreeHost(P->h_stats);
    if (P->h_rmax) cudaFreeHost(P->h_rmax);
    if (P->h_act) cudaFreeHost(P->h_act);
    DBuf *bufs[] = {&P->w_in,     &P->w_out,  &P->w_pts, &P->w_u,     &P->w_prm,  &P->m_U,     &P->m_R,
                    &P->m_UT,     &P->m_GC,   &P->m_res, &P->m_UT1,   &P->m_GC1,  &P->m_T0,    &P->m_act,
                    &P->w_tune,   &P->n_master, &P->n_m, &P->n_v,     &P->n_w,    &P->n_rows,  &P->n_loss,
                    &P->n_act,    &P->n_items, &P->n_U,  &P->n_Y,     &P->n_grad, &P->n_tmp,   &P->n_prm,
                    &P->w_xg,     &P->m_Z,     &P->m_E,   &P->w_part, &P->w_scr};
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
    } else if (kind == 2 || kind == 3) {
        if (n_params < 1 || !std::isfinite(params[0])) return fail(PIT_ERR_INVALID_ARG, "need the time t");
    } else if (kind == 4) {
        if (n_params < d + d * d) return fail(PIT_ERR_INVALID_ARG, "need d + d*d parameters");
    } else {
        return fail(PIT_ERR_INVALID_ARG, "unknown initial-value kind %d", kind);
    }
    std::vector<double> prm(params, params + n_params);
    if (kind == 4) {
        // the kernel takes the mean, the Cholesky factor R of the covariance
        // (C = R R^T, lower, row major) and log det R
        const double *C = params + d;
        std::vector<double> R((size_t)d * d, 0.0);
        double logdet = 0.0;
        for (int i = 0; i < d; ++i)
            for (int k = 0; k <= i; ++k) {
                double v = C[i * d + k];
                for (int q = 0; q < k; ++q) v -= R[i * d + q] * R[k * d + q];
                if (i == k) {
                    if (!(v > 0.0)) return fail(PIT_ERR_INVALID_ARG, "the covariance is not positive definite");
                    R[i * d + i] = sqrt(v);
                    logdet += log(R[i * d + i]);
                } else {
                    R[i * d + k] = v / R[k * d + k];
                }
            }
        prm.assign(params, params + d);
        prm.insert(prm.end(), R.begin(), R.end());
        prm.push_back(logdet);
        n_params = (int)prm.size();
    }
    CU(P->w_prm.ensure(sizeof(double) * n_params));
    CU(cudaMemcpyAsync(P->w_prm.p, prm.data(), sizeof(double) * n_params, cudaMemcpyHostToDevice, P->stream));
    const bool dev = ptr_is_device(u0);
    double *target = u0;
    if (!dev) {
        CU(P->w_u.ensure(sizeof(double) * P->ntot));
        target = P->w_u.d();
    }
    {
        ProfScope ps(P, 3);
        CU(launch_initial(P->d_grids, P->G, P->op, P->d_hi, kind, P->w_prm.d(), n_params, target, P->stream));
        count_kernels(P, 3);
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
    count_kernels(P, 3);
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

pit_status pit_sequential_solve_forced(pit_problem_t P, const double *u0, double dt, int nsteps, const double *forcing,
                                       const int *tmul, const pit_solve_opts *opts, double *uT, pit_phi_stats *stats)
{
    if (!P || !u0 || !uT || nsteps < 0) return fail(PIT_ERR_INVALID_ARG, "bad argument");
    if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(PIT_ERR_INVALID_ARG, "dt must be finite and >= 0");
    TRY(check_solve_opts(opts));
    if (forcing && !ptr_is_device(forcing)) return fail(PIT_ERR_INVALID_ARG, "forcing must be device memory");
    // grids grouped by their own time partition (steps per common step)
    std::vector<int> tm_vals, group(P->G, 0);
    if (tmul) {
        for (int g = 0; g < P->G; ++g) {
            const int t = tmul[g];
            if (t < 1 || t > 4096) return fail(PIT_ERR_INVALID_ARG, "tmul[%d] = %d outside 1..4096", g, t);
            auto pos = std::find(tm_vals.begin(), tm_vals.end(), t);
            if (pos == tm_vals.end()) {
                tm_vals.push_back(t);
                group[g] = (int)tm_vals.size() - 1;
            } else {
                group[g] = (int)(pos - tm_vals.begin());
            }
        }
    } else {
        tm_vals.push_back(1);
    }
    const int n_groups = (int)tm_vals.size();
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
        int *masks = nullptr;
        if (n_groups > 1) {
            // one activity mask per group, uploaded once
            CU(P->m_act.ensure(sizeof(int) * (size_t)P->G * n_groups));
            std::vector<int> h((size_t)P->G * n_groups, 0);
            for (int g = 0; g < P->G; ++g) h[(size_t)group[g] * P->G + g] = 1;
            masks = (int *)P->m_act.p;
            CU(cudaMemcpyAsync(masks, h.data(), sizeof(int) * h.size(), cudaMemcpyHostToDevice, P->stream));
            CU(cudaStreamSynchronize(P->stream));  // h is freed on return
        }
        for (int q = 0; q < n_groups; ++q) {
            // every grid is one CTA that takes all its steps on chip; grid g
            // takes tm steps of dt / tm per common step, each with the common
            // step's forcing
            const int tm = tm_vals[q];
            StepCall c;
            c.dt = dt / tm;
            c.nb = 1;
            c.nsteps = nsteps * tm;
            c.in = src;
            c.is = P->ntot;
            if (forcing) {
                c.f = forcing;
                c.fst = P->ntot;
                c.fdiv = tm;
            }
            c.out_last = target;
            c.ols = P->ntot;
            TRY(run_steps(P, *opts, c, masks ? masks + (size_t)q * P->G : nullptr));
        }
    }
    if (target != uT)
        CU(cudaMemcpyAsync(uT, target, bytes, dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, P->stream));
    DevStats s;
    TRY(read_stats(P, s));
    if (stats) fill_phi_stats(s, stats);
    TRY(status_of(s));
    return PIT_OK;
}

pit_status pit_sequential_solve(pit_problem_t P, const double *u0, double dt, int nsteps,
                                const pit_solve_opts *opts, double *uT, pit_phi_stats *stats)
{
    return pit_sequential_solve_forced(P, u0, dt, nsteps, nullptr, nullptr, opts, uT, stats);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Recombination (Sec. 2.2.2, Eq. "overall_combination_operator"): the block
// plan of the sparse grid's hierarchical increments, built once per problem.
namespace {

pit_status recomb_plan(pit_problem *P)
{
    if (P->rc_ready) return PIT_OK;
    const int d = P->desc.d, G = P->G;
    int Lmax = 1;
    for (int l : P->levels) Lmax = l > Lmax ? l : Lmax;
    const int R = Lmax + 1;
    double cells = 1.0;
    for (int i = 0; i < d; ++i) cells *= R;
    if (cells > (double)(1 << 24))
        return fail(PIT_ERR_UNSUPPORTED, "recombination: the increment table would need %.0f entries (levels up to %d "
                                         "in %d dimensions)", cells, Lmax, d);
    const int ncell = (int)cells;
    auto code_of = [&](const int *lam) {
        int c = 0;
        for (int i = 0; i < d; ++i) c = c * R + lam[i];
        return c;
    };
    // every increment lam <= l of every grid l (odometer over the box 1..l)
    std::vector<char> used(ncell, 0);
    auto for_box = [&](int g, auto &&fn) {
        const int *l = &P->levels[(size_t)g * d];
        int lam[PIT_MAX_DIM];
        for (int i = 0; i < d; ++i) lam[i] = 1;
        for (;;) {
            fn(lam);
            int i = d - 1;
            while (i >= 0 && lam[i] == l[i]) lam[i--] = 1;
            if (i < 0) break;
            ++lam[i];
        }
    };
    for (int g = 0; g < G; ++g) for_box(g, [&](const int *lam) { used[code_of(lam)] = 1; });
    std::vector<int> lookup(ncell, -1), blk_lam;
    std::vector<long long> blk_off(1, 0);
    int n_blk = 0;
    for (int c = 0; c < ncell; ++c) {
        if (!used[c]) continue;
        int lam[PIT_MAX_DIM], r = c, e = 0;
        for (int i = d - 1; i >= 0; --i) {
            lam[i] = r % R;
            r /= R;
            e += lam[i] - 1;
        }
        lookup[c] = n_blk++;
        blk_lam.insert(blk_lam.end(), lam, lam + d);
        blk_off.push_back(blk_off.back() + (1LL << e));
    }
    std::vector<std::vector<int>> lists(n_blk);
    for (int g = 0; g < G; ++g) for_box(g, [&](const int *lam) { lists[lookup[code_of(lam)]].push_back(g); });
    std::vector<int> list_off(1, 0), list;
    for (auto &L : lists) {
        list.insert(list.end(), L.begin(), L.end());
        list_off.push_back((int)list.size());
    }
    auto up = [&](auto *&dst, const auto &v) -> cudaError_t {
        cudaError_t e = dev_malloc(&dst, sizeof(v[0]) * v.size());
        if (e != cudaSuccess) return e;
        return cudaMemcpy(dst, v.data(), sizeof(v[0]) * v.size(), cudaMemcpyHostToDevice);
    };
    CU(up(P->rc_lam, blk_lam));
    CU(up(P->rc_off, blk_off));
    CU(up(P->rc_list_off, list_off));
    CU(up(P->rc_list, list));
    CU(up(P->rc_lookup, lookup));
    P->rc = RecombPlan{n_blk, R, blk_off.back(), P->rc_lam, P->rc_off, P->rc_list_off, P->rc_list, P->rc_lookup};
    P->rc_ready = true;
    return PIT_OK;
}

// out_b = Q u_b for nb consecutive states on the problem's stream (out may alias u).
pit_status recombine(pit_problem *P, const double *u, double *out, int nb = 1)
{
    TRY(recomb_plan(P));
    CU(P->rc_H.ensure(sizeof(double) * P->ntot * (size_t)nb));
    CU(P->rc_S.ensure(sizeof(double) * P->rc.n_sparse * (size_t)nb));
    ProfScope ps(P, 3);
    CU(launch_recombine(P->rc, P->desc.d, P->d_grids, P->d_coef, P->G, P->ntot, nb, u, P->rc_H.d(), P->rc_S.d(), out,
                        P->stream));
    count_kernels(P, 3, 3);
    return PIT_OK;
}

}  // namespace

extern "C" pit_status pit_recombine(pit_problem_t P, const double *u, double *out)
{
    if (!P || !u || !out) return fail(PIT_ERR_INVALID_ARG, "NULL argument");
    if (!ptr_is_device(u) || !ptr_is_device(out)) return fail(PIT_ERR_INVALID_ARG, "u and out must be device memory");
    const size_t bytes = sizeof(double) * P->ntot;
    const char *a0 = (const char *)u, *b0 = (const char *)out;
    if (a0 != b0 && a0 < b0 + bytes && b0 < a0 + bytes)
        return fail(PIT_ERR_INVALID_ARG, "out overlaps u without being the same vector");
    return recombine(P, u, out);
}

// ---------------------------------------------------------------------------
// MGRIT driver (Sec. 3.3, Alg. 2 with FCF or F relaxation; Alg. 3 per grid).
//
// Level 0 stores C-points only (Sec. 3.3.2): U[j] = u_{jm}, j = 0..Nc.  One
// FCF cycle is three or four launches of the multi-step kernel:
//   FC    R[j+1]  = Phi^m(U[j])            (F-relaxation + C-relaxation)
//   F     UT[j]   = Phi^m(R[j]),  res[j] = ||UT[j] - R[j+1]||   (F-relaxation,
//                  C-point residual r_{j+1} = Phi(u_{(j+1)m-1}) - u_{(j+1)m})
// then, with a linear coarse propagator (correction form, the default):
//   sweep E[j+1]  = Phi_c(E[j]) + r_{j+1}, E[0] = 0, U[j+1] = R[j+1] + E[j+1]
//                  (the F launch writes r_{j+1} in place of UT[j])
// or, in the FAS form of Alg. 2 as printed (learned or exact Phi_c):
//   FAS   GC[j]   = UT[j] - Phi_c(R[j])    (restricted residual + Phi_c of the
//                  restricted solution: the coarse right-hand side of Alg. 2)
//   sweep U[j+1]  = Phi_c(U[j]) + GC[j]    (coarse solve; its result is the
//                  corrected C-point, the F-points follow from the next cycle)
// R[0] = U[0] = u0.  F-relaxation drops the FC launch: the relaxed C-points
// are U itself.  With three levels the sweep is replaced by one two-level FCF
// cycle of the level-1 problem, written into U.
namespace {

struct Mg {
    pit_problem *P;
    const pit_mgrit_opts *o;
    double dt;
    long long nt;
    const int *active;
    bool learned;    // level-1 coarse propagator is the network
    pit_lane *L;     // lane of the cycle; nullptr: every grid on the problem's stream
    cudaStream_t s;  // stream of the cycle
    // finest level of the cycle's grids (their own time partition, Sec. 2.2.1):
    // tm steps of dtf = dt / tm per common step, mf = m tm per coarse interval;
    // forcing F of the common steps (NULL: none); the coarse levels keep dT = m dt
    double dtf = 0.0;
    int mf = 0, tm = 1;
    const double *F = nullptr;
};

// Coarse propagator of level 1: backward Euler with m dt, or m fine steps;
// of every coarse level with PIT_COARSE_SDIRK2: two-stage SDIRK steps of
// dT = m^level dt (the kernel takes the stage step gamma dT); with
// PIT_COARSE_EXTRAP: extrapolated backward-Euler steps of dT (the kernel
// takes the half step dT / 2).
void coarse_call(Mg &M, StepCall &c, int level)
{
    if (level == 1 && M.o->coarse == PIT_COARSE_EXACT) {
        c.dt = M.dtf;
        c.nsteps *= M.mf;
    } else {
        double dtl = M.dt;
        for (int q = 0; q < level; ++q) dtl *= M.o->m;
        c.dt = dtl;
        if (M.o->coarse == PIT_COARSE_SDIRK2) {
            c.dt = (1.0 - 1.0 / std::sqrt(2.0)) * dtl;
            c.sdirk = 1;
        } else if (M.o->coarse == PIT_COARSE_EXTRAP) {
            c.dt = 0.5 * dtl;
            c.ext = 1;
        }
    }
}

// Runs one call with the coarse propagator of `level` (1: Phi_c, 2: Phi_cc).
pit_status run_coarse(Mg &M, StepCall c, int level)
{
    if (level == 1 && M.learned) {
        c.dt = M.dt * M.o->m;
        return run_net(M.P, c, M.active);  // (the learned form runs without lanes)
    }
    coarse_call(M, c, level);
    return run_steps(M.P, M.o->crs, c, M.active, M.L);
}

// Two-level cycle of level 1 in a three-level hierarchy: level-1 points are V
// (read; stride vstride, 0 for a constant initial guess) -> W (written),
// Nc1 = N1/m intervals, forcing of level-1 point k is F[k-1]; the level-2
// problem is solved by a sequential sweep.  W[0] must equal V[0] on entry
// when the cycle runs on a lane (the copy below covers every grid).
pit_status mg_level1_cycle(Mg &M, const double *V, long long vstride, double *W, int N1, const double *F)
{
    pit_problem *P = M.P;
    const int m = M.o->m, Nc = N1 / m;
    const long long nt = M.nt, sm = (long long)m * nt;
    double *UT1 = P->m_UT1.d(), *GC1 = P->m_GC1.d();
    if (W != V && !M.L) CU(cudaMemcpyAsync(W, V, sizeof(double) * nt, cudaMemcpyDeviceToDevice, M.s));
    // FC: F-points and C-point of every interval from the old C-points
    StepCall fc;
    fc.nb = Nc;
    fc.nsteps = m;
    fc.in = V;
    fc.is = vstride * m;
    fc.g = F;
    fc.gs = sm;
    fc.gst = nt;
    fc.out_steps = W + nt;
    fc.oss = sm;
    fc.osst = nt;
    fc.out_last = W + sm;
    fc.ols = sm;
    // (PIT_RELAX_F_ALL: F-relaxation on this level too, from the old C-points)
    const bool f_only = M.o->relax == PIT_RELAX_F_ALL;
    if (!f_only) TRY(run_coarse(M, fc, 1));
    // F-relaxation from the new C-points (F-points in place) and utilde
    StepCall fr = fc;
    fr.in = f_only ? V : W;
    fr.is = f_only ? vstride * m : sm;
    fr.out_last = UT1;
    fr.ols = nt;
    TRY(run_coarse(M, fr, 1));
    // coarse right-hand side and the level-2 sweep into the C-points of W
    StepCall gc;
    gc.nb = Nc;
    gc.nsteps = 1;
    gc.in = f_only ? V : W;
    gc.is = f_only ? vstride * m : sm;
    gc.out_last = GC1;
    gc.ols = nt;
    gc.scale = -1.0;
    gc.h = UT1;
    gc.hs = nt;
    TRY(run_coarse(M, gc, 2));
    StepCall sw;
    sw.nb = 1;
    sw.nsteps = Nc;
    sw.in = W;
    sw.is = nt;
    sw.g = GC1;
    sw.gst = nt;
    sw.guess = UT1;  // Phi_2 of the relaxed level-1 C-points, as in the two-level sweep
    sw.gust = nt;
    sw.out_steps = W + sm;
    sw.osst = sm;
    sw.out_last = W + (long long)Nc * sm;
    sw.ols = nt;
    TRY(run_coarse(M, sw, 2));
    return PIT_OK;
}

// Enqueues one MGRIT cycle of the active grids (of the lane) on M.s:
// relaxation, C-point residual norms (copied to h_res, G x Nc), coarse
// correction of the C-points.  corr: linear coarse problem solved for the
// correction; otherwise the FAS form of Alg. 2.
pit_status mg_cycle(Mg &M, int Nc, bool corr, double *h_res)
{
    pit_problem *P = M.P;
    const pit_mgrit_opts *o = M.o;
    const int G = P->G, m = o->m;
    const long long nt = M.nt;
    const size_t vb = sizeof(double) * nt;
    double *U = P->m_U.d(), *R = P->m_R.d(), *UT = P->m_UT.d(), *GC = P->m_GC.d(), *res = P->m_res.d();
    // F-relaxation alone leaves the C-points as they are: the relaxed C-points
    // are U itself, and the correction updates U in place
    const bool relax_f = o->relax == PIT_RELAX_F || o->relax == PIT_RELAX_F_ALL;
    double *Rx = relax_f ? U : R;
    if (o->residual) {
        // residual mode: the m - 1 F-points of every interval by the fine
        // solves as configured (a fixed number of iterations: inexact), then
        // the space-time residual of the backward-Euler equation at the
        // C-point, rho_{j+1} = u_{(j+1)m-1} + dt f_{(j+1)m} - A u_{(j+1)m};
        // the coarse problem A_c e_{j+1} = e_j + rho_{j+1} (e_0 = 0) is solved
        // by the sweep with forcing rho / dT, and u_{j+1} += e_{j+1}
        StepCall fr;
        fr.dt = M.dtf;
        fr.nb = Nc;
        fr.nsteps = m - 1;
        fr.in = U;
        fr.is = nt;
        if (M.F) {
            fr.f = M.F;
            fr.fs = (long long)m * nt;
            fr.fst = nt;
        }
        fr.out_last = R + nt;
        fr.ols = nt;
        fr.inexact = 1;
        TRY(run_steps(P, o->fine, fr, M.active, M.L));
        const double dT = M.dt * m;
        CU(launch_st_resid(P->d_grids, G, nt, Nc, M.dtf, R + nt, nt, M.F ? M.F + (long long)(m - 1) * nt : nullptr,
                           (long long)m * nt, U + nt, nt, 1.0 / dT, GC, nt, res, M.active, P->d_faces, P->op, M.s));
        count_kernels(P, 3);
        CU(cudaMemcpyAsync(h_res, res, sizeof(double) * G * Nc, cudaMemcpyDeviceToHost, M.s));
        StepCall sw;
        sw.nb = 1;
        sw.nsteps = Nc;
        sw.in = P->m_Z.d();
        sw.is = nt;
        sw.f = GC;
        sw.fst = nt;
        sw.hstep = U + nt;  // u_{j+1} + e_{j+1}, read and written by the same thread
        sw.hsst = nt;
        sw.out_steps = U + nt;
        sw.osst = nt;
        sw.out_last = U + (long long)Nc * nt;
        sw.ols = nt;
        TRY(run_coarse(M, sw, 1));
        return PIT_OK;
    }
    StepCall fc;  // FC relaxation
    fc.dt = M.dtf;
    fc.nb = Nc;
    fc.nsteps = M.mf;
    if (M.F) {  // forcing of common step j m + (s - 1) / tm for step s of interval j
        fc.f = M.F;
        fc.fs = (long long)m * nt;
        fc.fst = nt;
        fc.fdiv = M.tm;
    }
    fc.in = U;
    fc.is = nt;
    fc.out_last = R + nt;
    fc.ols = nt;
    if (!relax_f) TRY(run_steps(P, o->fine, fc, M.active, M.L));
    StepCall fr = fc;  // F relaxation, utilde and the C-point residuals
    fr.in = Rx;
    fr.cmp = Rx + nt;
    fr.cs = nt;
    fr.norms = res;
    if (corr) {
        fr.out_last = GC;  // r_{j+1} = utilde_{j+1} - u_{(j+1)m}
        fr.h = Rx + nt;
        fr.hs = nt;
        fr.hscale = -1.0;
    } else {
        fr.out_last = UT;
    }
    TRY(run_steps(P, o->fine, fr, M.active, M.L));
    CU(cudaMemcpyAsync(h_res, res, sizeof(double) * G * Nc, cudaMemcpyDeviceToHost, M.s));
    if (corr) {
        if (o->levels == 3) {
            // level-1 problem e_k = Phi_c(e_{k-1}) + r_k, e_0 = 0, by one
            // two-level cycle from e = 0; then u_{jm} = relaxed + e_j
            TRY(mg_level1_cycle(M, P->m_Z.d(), 0, P->m_E.d(), Nc, GC));
            CU(launch_add_states(P->d_grids, G, nt, Nc, Rx + nt, P->m_E.d() + nt, U + nt, M.active, M.s));
            count_kernels(P, 3);
        } else {
            StepCall sw;  // e_{j+1} = Phi_c(e_j) + r_{j+1}; stored as u = relaxed + e
            sw.nb = 1;
            sw.nsteps = Nc;
            sw.in = P->m_Z.d();
            sw.is = nt;
            sw.g = GC;
            sw.gst = nt;
            sw.hstep = Rx + nt;  // read and written by the same thread when Rx = U
            sw.hsst = nt;
            sw.out_steps = U + nt;
            sw.osst = nt;
            sw.out_last = U + (long long)Nc * nt;
            sw.ols = nt;
            TRY(run_coarse(M, sw, 1));
        }
        return PIT_OK;
    }
    StepCall gc;  // coarse right-hand side
    gc.nb = Nc;
    gc.nsteps = 1;
    gc.in = Rx;
    gc.is = nt;
    gc.out_last = GC;
    gc.ols = nt;
    gc.scale = -1.0;
    gc.h = UT;
    gc.hs = nt;
    TRY(run_coarse(M, gc, 1));
    if (o->levels == 3) {
        // the level-1 cycle reads the relaxed C-points while it writes U:
        // with F-relaxation they are U itself, so take a copy
        if (relax_f) CU(cudaMemcpyAsync(R + nt, U + nt, vb * Nc, cudaMemcpyDeviceToDevice, M.s));
        TRY(mg_level1_cycle(M, R, nt, U, Nc, GC));
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
            TRY(run_steps(P, o->crs, sw, M.active, M.L));
        }
    } else {
        StepCall sw;  // sequential coarse sweep, one CTA per grid
        sw.nb = 1;
        sw.nsteps = Nc;
        sw.in = U;
        sw.is = nt;
        sw.g = GC;
        sw.gst = nt;
        // Krylov initial guess of Phi_c(u_j): Phi_c(r_j) = UT[j] - GC[j],
        // computed by the FAS launch (r_j = relaxed C-point; equal to u_j
        // once MGRIT has converged there)
        sw.guess = UT;
        sw.gust = nt;
        sw.out_steps = U + nt;
        sw.osst = nt;
        sw.out_last = U + (long long)Nc * nt;
        sw.ols = nt;
        if (M.learned) sw.guess = nullptr;  // explicit: no Krylov guess
        TRY(run_coarse(M, sw, 1));
    }
    return PIT_OK;
}

// Stopping rule of Sec. 4.1 per grid on one cycle's residual norms (h_res,
// G x Nc): a grid whose largest C-point residual is <= tol leaves the active
// set.  Returns the largest norm over the listed grids (NaN propagates).
double mg_evaluate(const double *h_res, int G, int Nc, const int *grids, int n_grids, int *h_act, double tol,
                   int &n_active)
{
    double rmax = 0.0;
    n_active = 0;
    for (int q = 0; q < n_grids; ++q) {
        const int g = grids ? grids[q] : q;
        if (!h_act[g]) continue;
        double r = 0.0;
        for (int j = 0; j < Nc; ++j) {
            const double v = h_res[(size_t)j * G + g];
            if (!(v <= r)) r = v;  // NaN propagates
        }
        if (!(r <= rmax)) rmax = r;
        if (r <= tol) h_act[g] = 0;
        else ++n_active;
    }
    return rmax;
}

// K lanes over the grids, balanced by nodes (largest grid first to the lane
// with the fewest nodes); each lane keeps the class lists of both precision
// forms in the problem's decreasing-size order.
pit_status lanes_prepare(pit_problem *P, int K, int Nc, const std::vector<int> *lane_of_in = nullptr,
                         const std::vector<int> *lane_tm = nullptr)
{
    // lanes balanced by nodes, or the given assignment (grids with their own
    // time partition: one lane per partition)
    std::vector<int> want;
    if (lane_of_in) want = *lane_of_in;
    if ((int)P->lanes.size() != K || want != P->lane_assign) {
        for (pit_lane &L : P->lanes) {
            cudaStreamSynchronize(L.s);
            for (auto sq : L.sides) cudaStreamSynchronize(sq);
            for (int p = 0; p < NPREC; ++p)
                for (int c = 0; c < 2; ++c) cudaFree(L.d_order_cls[p][c]);
            cudaFree(L.d_act);
            cudaFreeHost(L.h_act);
            cudaFreeHost(L.h_res);
            cudaStreamDestroy(L.s);
            for (auto sq : L.sides) cudaStreamDestroy(sq);
            cudaEventDestroy(L.fork);
            cudaEventDestroy(L.join);
            cudaEventDestroy(L.done);
        }
        P->lanes.assign(K, pit_lane());
        P->lane_assign = want;
        std::vector<int> order(P->G);
        for (int g = 0; g < P->G; ++g) order[g] = g;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return P->info[a].n > P->info[b].n; });
        std::vector<long long> load(K, 0);
        for (int g : order) {
            int best = 0;
            if (lane_of_in) {
                best = (*lane_of_in)[g];
            } else {
                for (int k = 1; k < K; ++k)
                    if (load[k] < load[best]) best = k;
            }
            load[best] += P->info[g].n;
            P->lanes[best].grids.push_back(g);
        }
        for (pit_lane &L : P->lanes) {
            CU(cudaStreamCreateWithFlags(&L.s, cudaStreamNonBlocking));
            for (auto &sq : L.sides) CU(cudaStreamCreateWithFlags(&sq, cudaStreamNonBlocking));
            CU(cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming));
            CU(cudaEventCreateWithFlags(&L.join, cudaEventDisableTiming));
            CU(cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming));
            CU(dev_malloc(&L.d_act, sizeof(int) * P->G));
            CU(cudaMallocHost(&L.h_act, sizeof(int) * P->G));
        }
    }
    for (int prec = 0; prec < NPREC; ++prec) {
        if (!P->planned[prec]) continue;
        for (int k = 0; k < K; ++k) {
            pit_lane &L = P->lanes[k];
            if (L.planned[prec]) continue;
            std::vector<char> mine(P->G, 0);
            std::vector<int> bkt(P->G, 0);
            for (int g : L.grids) mine[g] = 1;
            for (int q = 0; q < NBKT; ++q)
                for (int k = P->split[prec][q]; k < P->split[prec][q + 1]; ++k) bkt[P->h_order_cls[prec][0][k]] = q;
            // the lane's class-0 list keeps the problem's order, so its buckets
            // are consecutive too
            int cnt[NBKT] = {};
            for (int g : P->h_order_cls[prec][0])
                if (mine[g]) ++cnt[bkt[g]];
            L.split[prec][0] = 0;
            for (int q = 0; q < NBKT; ++q) L.split[prec][q + 1] = L.split[prec][q] + cnt[q];
            for (int c = 0; c < 2; ++c) {
                std::vector<int> lst;
                for (int g : P->h_order_cls[prec][c])
                    if (mine[g]) lst.push_back(g);
                L.n_cls[prec][c] = (int)lst.size();
                if (!lst.empty()) {
                    CU(dev_malloc(&L.d_order_cls[prec][c], sizeof(int) * lst.size()));
                    CU(cudaMemcpy(L.d_order_cls[prec][c], lst.data(), sizeof(int) * lst.size(),
                                  cudaMemcpyHostToDevice));
                }
            }
            L.planned[prec] = true;
        }
    }
    for (int k = 0; k < K; ++k) P->lanes[k].tm = lane_tm ? (*lane_tm)[k] : 1;
    for (pit_lane &L : P->lanes) {
        const size_t want = (size_t)P->G * Nc;
        if (L.h_res_cap < want) {
            if (L.h_res) cudaFreeHost(L.h_res);
            L.h_res = nullptr;
            L.h_res_cap = 0;
            CU(cudaMallocHost(&L.h_res, sizeof(double) * want));
            L.h_res_cap = want;
        }
    }
    return PIT_OK;
}

// Workspaces and CTA sizes of every launch class a lane cycle uses, prepared
// on the problem's stream before the lanes start (the autotuner times its
// trial launches on that stream).
pit_status lanes_prime(Mg &M, int Nc)
{
    pit_problem *P = M.P;
    const pit_mgrit_opts *o = M.o;
    const long long nt = M.nt;
    struct Rep { const pit_solve_opts *so; int nb; double dt; int nsteps; };
    Rep reps[3] = {{&o->fine, Nc, M.dt, o->m}, {&o->crs, 1, M.dt * o->m, Nc},
                   {&o->crs, Nc / o->m, M.dt * o->m, o->m}};
    const int n_reps = o->levels == 3 ? 3 : 2;
    for (int r = 0; r < n_reps; ++r) {
        const int prec = prec_form(reps[r].so->prec);
        TRY(plan(P, prec));
        if (reps[r].nb <= 0) continue;
        StepCall c;
        c.dt = reps[r].dt;
        c.nb = reps[r].nb;
        c.nsteps = reps[r].nsteps;
        c.in = P->m_U.d();  // u0 at every C-point
        c.is = nt;
        if (P->n_cls[prec][1] > 0) CU(P->w_xg.ensure(sizeof(double) * nt * (size_t)Nc * xg_slabs(prec, P->desc.op, P->desc.d)));
        // (lane launches of extrapolated FP32 steps: the sweeps (one state per
        // grid) and, with three levels, the level-1 relaxations (Nc / m states)
        if (prec == SINGLE && (o->coarse == PIT_COARSE_EXTRAP || o->init == 2))
            CU(P->w_scr.ensure(sizeof(float) * nt * (size_t)(o->levels == 3 && Nc / o->m > 1 ? Nc / o->m : 1)));
        for (int part = 0; part < NPART; ++part) TRY(tune(P, prec, c.nb >= 8, part, *reps[r].so, c, M.active));
    }
    return PIT_OK;
}

}  // namespace

namespace {
pit_status mgrit_run(pit_problem_t P, const double *u0, const pit_mgrit_opts *o, double *uT, pit_mgrit_stats *stats)
{
    auto t_start = std::chrono::steady_clock::now();
    if (!P || !u0 || !uT || !o) return fail(PIT_ERR_INVALID_ARG, "NULL argument");
    TRY(check_solve_opts(&o->fine));
    TRY(check_solve_opts(&o->crs));
    if (o->m < 2 || o->levels < 2 || o->levels > 3 || o->nsteps < 1 || o->maxit < 1 || !(o->tol >= 0.0) ||
        !(o->t1 > o->t0))
        return fail(PIT_ERR_INVALID_ARG, "need m >= 2, levels in {2,3}, nsteps >= 1, maxit >= 1, tol >= 0, t1 > t0");
    if (o->coarse != PIT_COARSE_IMPLICIT && o->coarse != PIT_COARSE_EXACT && o->coarse != PIT_COARSE_LEARNED &&
        o->coarse != PIT_COARSE_SDIRK2 && o->coarse != PIT_COARSE_EXTRAP)
        return fail(PIT_ERR_INVALID_ARG, "unknown coarse propagator %d", o->coarse);
    const bool ext_op = P->desc.op == PIT_OP_HEAT || P->desc.op == PIT_OP_VARHEAT;
    if (o->coarse == PIT_COARSE_EXTRAP && ((o->crs.prec != PIT_PREC_MIXED && o->crs.prec != PIT_PREC_FP32) || !ext_op))
        return fail(PIT_ERR_UNSUPPORTED, "the extrapolated coarse propagator is built for the heat operators (constant "
                                         "and variable coefficient) with PIT_PREC_MIXED or PIT_PREC_FP32 coarse solves");
    if (o->coarse == PIT_COARSE_SDIRK2 && o->crs.prec != PIT_PREC_MIXED && o->crs.prec != PIT_PREC_FP32)
        return fail(PIT_ERR_UNSUPPORTED, "the SDIRK coarse propagator needs PIT_PREC_MIXED or PIT_PREC_FP32 coarse "
                                         "solves");
    if (o->coarse == PIT_COARSE_LEARNED && !P->have_net)
        return fail(PIT_ERR_INVALID_ARG, "the learned coarse propagator has no parameters (pit_train_coarse or "
                                         "pit_net_set_params)");
    long long div = o->m;
    if (o->levels == 3) div *= o->m;
    if (o->nsteps % div != 0) return fail(PIT_ERR_INVALID_ARG, "nsteps must be a multiple of m^(levels-1)");
    if (o->levels == 3 && o->coarse == PIT_COARSE_EXACT)
        return fail(PIT_ERR_UNSUPPORTED, "the exact coarse propagator is a two-level option");
    if (o->relax != PIT_RELAX_FCF && o->relax != PIT_RELAX_F && o->relax != PIT_RELAX_F_ALL)
        return fail(PIT_ERR_INVALID_ARG, "unknown relaxation %d", o->relax);
    if (o->lanes < 0) return fail(PIT_ERR_INVALID_ARG, "lanes must be >= 0");
    if (o->init < 0 || o->init > 2) return fail(PIT_ERR_INVALID_ARG, "init must be 0, 1 or 2");
    if (o->init == 2 && ((o->crs.prec != PIT_PREC_MIXED && o->crs.prec != PIT_PREC_FP32) || !ext_op ||
                         o->coarse == PIT_COARSE_EXACT))
        return fail(PIT_ERR_UNSUPPORTED, "the extrapolated initial sweep is built for the heat operators (constant and "
                                         "variable coefficient) with PIT_PREC_MIXED or PIT_PREC_FP32 coarse solves, "
                                         "without the exact coarse propagator");
    if (o->forcing && !ptr_is_device(o->forcing)) return fail(PIT_ERR_INVALID_ARG, "forcing must be device memory");
    if (o->residual != 0 && o->residual != 1) return fail(PIT_ERR_INVALID_ARG, "residual must be 0 or 1");
    if (o->residual && (o->levels != 2 || o->relax != PIT_RELAX_F || o->fas || o->coarse != PIT_COARSE_IMPLICIT ||
                        o->tmul))
        return fail(PIT_ERR_UNSUPPORTED, "residual mode runs two levels, F-relaxation and the implicit coarse step in "
                                         "the correction form, without per-grid partitions");
    const int G = P->G, m = o->m, Nc = o->nsteps / m;
    const long long nt = P->ntot;
    const size_t vb = sizeof(double) * nt;
    CU(P->m_U.ensure(vb * (Nc + 1)));
    CU(P->m_R.ensure(vb * (Nc + 1)));
    CU(P->m_UT.ensure(vb * Nc));
    CU(P->m_GC.ensure(vb * Nc));
    CU(P->m_res.ensure(sizeof(double) * G * Nc));
    CU(P->m_act.ensure(sizeof(int) * G));
    CU(P->m_Z.ensure(vb));
    CU(cudaMemsetAsync(P->m_Z.p, 0, vb, P->stream));
    if (o->levels == 3) {
        CU(P->m_E.ensure(vb * (Nc + 1)));
        CU(cudaMemsetAsync(P->m_E.p, 0, vb, P->stream));  // e_0 = 0 of the level-1 correction problem
        const int Nc1 = Nc / m;
        CU(P->m_UT1.ensure(sizeof(double) * nt * Nc1));
        CU(P->m_GC1.ensure(sizeof(double) * nt * Nc1));
    }
    P->h_res.resize((size_t)G * Nc);
    double *U = P->m_U.d(), *R = P->m_R.d();
    int *act = (int *)P->m_act.p;
    const double *src;
    TRY(stage_in(P, P->w_in, u0, nt, &src));
    for (int j = 0; j <= Nc; ++j)
        CU(cudaMemcpyAsync(U + (long long)j * nt, src, vb, cudaMemcpyDeviceToDevice, P->stream));
    CU(cudaMemcpyAsync(R, src, vb, cudaMemcpyDeviceToDevice, P->stream));
    for (int g = 0; g < G; ++g) P->h_act[g] = 1;
    CU(cudaMemcpyAsync(act, P->h_act, sizeof(int) * G, cudaMemcpyHostToDevice, P->stream));
    TRY(reset_stats(P));

    Mg M{P, o, (o->t1 - o->t0) / o->nsteps, nt, act, o->coarse == PIT_COARSE_LEARNED && P->net_accepted, nullptr,
         P->stream};
    M.dtf = M.dt;
    M.mf = m;
    M.F = o->forcing;
    // per-grid time partitions: grids with the same number of steps per common
    // step form one lane; a single partition for all grids needs no lanes
    std::vector<int> tm_vals, lane_of;
    if (o->tmul) {
        lane_of.assign(G, 0);
        for (int g = 0; g < G; ++g) {
            const int t = o->tmul[g];
            if (t < 1 || t > 4096) return fail(PIT_ERR_INVALID_ARG, "tmul[%d] = %d outside 1..4096", g, t);
            auto pos = std::find(tm_vals.begin(), tm_vals.end(), t);
            if (pos == tm_vals.end()) {
                tm_vals.push_back(t);
                lane_of[g] = (int)tm_vals.size() - 1;
            } else {
                lane_of[g] = (int)(pos - tm_vals.begin());
            }
        }
        if (tm_vals.size() == 1) {
            M.tm = tm_vals[0];
            M.dtf = M.dt / M.tm;
            M.mf = m * M.tm;
        }
    }
    pit_mgrit_stats st;
    memset(&st, 0, sizeof(st));
    st.learned_used = M.learned ? 1 : 0;
    st.fallback = (o->coarse == PIT_COARSE_LEARNED && !M.learned) ? 1 : 0;
    // linear coarse propagator: solve the coarse problem for the correction
    // (Sec. 3.3.1: Alg. 2's coarse system is linear here), so the coarse
    // tolerance is relative to the correction, which vanishes as MGRIT
    // converges; the learned one is nonlinear and keeps the FAS form
    auto corr_form = [&]() { return !M.learned && o->coarse != PIT_COARSE_EXACT && !o->fas; };
    if (o->init) {
        // initial C-points from one sweep of the level-1 propagator (the
        // F-points follow from the first relaxation)
        if (o->coarse == PIT_COARSE_EXACT) {
            for (int j = 0; j < Nc; ++j) {
                StepCall sw;
                sw.nb = 1;
                sw.nsteps = 1;
                sw.in = U + (long long)j * nt;
                sw.is = nt;
                sw.out_last = U + (long long)(j + 1) * nt;
                sw.ols = nt;
                TRY(run_coarse(M, sw, 1));
            }
        } else {
            StepCall sw;
            sw.nb = 1;
            sw.nsteps = Nc;
            sw.in = U;
            sw.is = nt;
            sw.out_steps = U + nt;
            sw.osst = nt;
            sw.out_last = U + (long long)Nc * nt;
            sw.ols = nt;
            // init 2: this sweep alone with the extrapolated backward Euler
            // (a closer initial guess; the cycles keep the coarse propagator)
            // (also when the cycles use the learned propagator)
            pit_mgrit_opts o_init = *o;
            const bool learned_cyc = M.learned;
            if (o->init == 2) {
                o_init.coarse = PIT_COARSE_EXTRAP;
                M.learned = false;
            }
            const pit_mgrit_opts *o_cyc = M.o;
            M.o = &o_init;
            const pit_status st_init = run_coarse(M, sw, 1);
            M.o = o_cyc;
            M.learned = learned_cyc;
            TRY(st_init);
        }
    }
    // lanes: the correction form with the implicit coarse step for the whole
    // solve (also when a learned propagator was requested but not accepted:
    // the runtime judge only ever switches from the network to the implicit
    // step), default five (measured best or within 1 % of it on four of the five workloads)
    int K = o->lanes == 0 ? 5 : o->lanes;
    if (!corr_form()) K = 1;
    if (K > G) K = G;
    const bool by_tm = tm_vals.size() > 1;
    if (by_tm) {
        if (!corr_form())
            return fail(PIT_ERR_UNSUPPORTED, "per-grid time partitions need the correction form with the implicit "
                                             "coarse step (fas = 0)");
        K = (int)tm_vals.size();
    }
    int it = 0, n_active = G;
    if (K > 1) {
        TRY(lanes_prime(M, Nc));
        TRY(lanes_prepare(P, K, Nc, by_tm ? &lane_of : nullptr, by_tm ? &tm_vals : nullptr));
        CU(cudaEventRecord(P->ev_fork, P->stream));
        for (pit_lane &L : P->lanes) {
            CU(cudaStreamWaitEvent(L.s, P->ev_fork, 0));
            memset(L.h_act, 0, sizeof(int) * G);
            for (int g : L.grids) L.h_act[g] = 1;
            CU(cudaMemcpyAsync(L.d_act, L.h_act, sizeof(int) * G, cudaMemcpyHostToDevice, L.s));
            L.it = 0;
            L.n_active = (int)L.grids.size();
            L.busy = true;
        }
        auto enqueue = [&](pit_lane &L) -> pit_status {
            Mg ML = M;
            ML.active = L.d_act;
            ML.L = &L;
            ML.s = L.s;
            ML.tm = L.tm;
            ML.dtf = M.dt / L.tm;
            ML.mf = m * L.tm;
            TRY(mg_cycle(ML, Nc, true, L.h_res));
            CU(cudaEventRecord(L.done, L.s));
            return PIT_OK;
        };
        for (pit_lane &L : P->lanes) TRY(enqueue(L));
        // the host serves whichever lane finished its cycle first (a blocking
        // wait on the lanes in turn would leave a finished lane idle behind a
        // slower one)
        int n_busy = (int)P->lanes.size();
        while (n_busy > 0) {
            bool served = false;
            for (pit_lane &L : P->lanes) {
                if (!L.busy) continue;
                const cudaError_t q = cudaEventQuery(L.done);
                if (q == cudaErrorNotReady) continue;
                CU(q);
                served = true;
                int na = 0;
                const double rmax = mg_evaluate(L.h_res, G, Nc, L.grids.data(), (int)L.grids.size(), L.h_act,
                                                o->tol, na);
                if (L.it < PIT_MAX_HIST && !(rmax <= st.res_hist[L.it])) st.res_hist[L.it] = rmax;
                ++L.it;
                L.n_active = na;
                if (na > 0 && L.it < o->maxit && rmax == rmax) {
                    CU(cudaMemcpyAsync(L.d_act, L.h_act, sizeof(int) * G, cudaMemcpyHostToDevice, L.s));
                    TRY(enqueue(L));
                } else {
                    L.busy = false;
                    --n_busy;
                }
            }
            if (!served) std::this_thread::yield();
        }
        n_active = 0;
        for (pit_lane &L : P->lanes) {
            CU(cudaEventRecord(L.done, L.s));
            CU(cudaStreamWaitEvent(P->stream, L.done, 0));
            it = L.it > it ? L.it : it;
            n_active += L.n_active;
        }
    } else {
        double r_prev = -1.0;
        while (n_active > 0 && it < o->maxit) {
            TRY(mg_cycle(M, Nc, corr_form(), P->h_res.data()));
            CU(cudaStreamSynchronize(P->stream));
            const double rmax = mg_evaluate(P->h_res.data(), G, Nc, nullptr, G, P->h_act, o->tol, n_active);
            if (it < PIT_MAX_HIST) st.res_hist[it] = rmax;
            ++it;
            // runtime judge of the learned coarse propagator: fall back to the
            // implicit step when a cycle does not reduce the residual enough
            if (M.learned && n_active > 0 && (!(rmax == rmax) || (r_prev > 0.0 && rmax > 0.9 * r_prev))) {
                M.learned = false;
                st.fallback = 1;
            }
            r_prev = rmax;
            if (n_active > 0) CU(cudaMemcpyAsync(act, P->h_act, sizeof(int) * G, cudaMemcpyHostToDevice, P->stream));
            if (!(rmax == rmax)) break;  // NaN: stop at once
        }
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
}  // namespace

// Global MGRIT (Sec. 3.4: MGRIT applied to the whole combination-technique
// problem instead of each subproblem): the propagator of one block of r fine
// steps is Psi = Phi^r o Q, the recombination Q (Eq. "overall_combination_
// operator") followed by r backward-Euler steps on every grid, so that the
// grids are coupled every r steps and iterate together.  Two levels, F-
// relaxation, coarse problem for the correction with Psi_c = Phi_c o Q, one
// stopping rule over all grids (the largest C-point residual).  Its fixed
// point is the time-sequential combination method (Alg. 1) with a
// recombination step every r fine steps.
namespace {
pit_status mgrit_global(pit_problem_t P, const double *u0, const pit_mgrit_opts *o, double *uT,
                        pit_mgrit_stats *stats)
{
    auto t_start = std::chrono::steady_clock::now();
    const int r = o->global_every, m = o->m;
    if (o->levels != 2 || o->relax != PIT_RELAX_F || o->fas || o->coarse != PIT_COARSE_IMPLICIT || o->tmul ||
        o->recomb)
        return fail(PIT_ERR_UNSUPPORTED, "global MGRIT runs two levels, F-relaxation, the implicit coarse step in the "
                                         "correction form, without per-grid partitions or recombination intervals");
    if (r < 1 || m % r != 0) return fail(PIT_ERR_INVALID_ARG, "global_every must divide m");
    if (o->nsteps % m != 0) return fail(PIT_ERR_INVALID_ARG, "nsteps must be a multiple of m");
    const int G = P->G, Nc = o->nsteps / m;
    const long long nt = P->ntot;
    const size_t vb = sizeof(double) * nt;
    const double dt = (o->t1 - o->t0) / o->nsteps;
    CU(P->m_U.ensure(vb * (Nc + 1)));
    CU(P->m_R.ensure(vb * (size_t)Nc * 2));  // relaxation work states (ping-pong)
    CU(P->m_GC.ensure(vb * Nc));
    CU(P->m_E.ensure(vb * (Nc + 1)));
    CU(P->m_res.ensure(sizeof(double) * G * Nc));
    CU(P->m_Z.ensure(vb));
    double *U = P->m_U.d(), *W0 = P->m_R.d(), *W1 = W0 + (long long)Nc * nt, *GC = P->m_GC.d(), *E = P->m_E.d();
    double *res = P->m_res.d(), *Z = P->m_Z.d();
    P->h_res.resize((size_t)G * Nc);
    const double *src;
    TRY(stage_in(P, P->w_in, u0, nt, &src));
    TRY(reset_stats(P));
    // initial guess: u_0 at every C-point, or one sweep of Psi_c
    for (int j = 0; j <= Nc; ++j)
        CU(cudaMemcpyAsync(U + (long long)j * nt, src, vb, cudaMemcpyDeviceToDevice, P->stream));
    auto coarse_step = [&](const double *in, const double *g, double *out) -> pit_status {
        TRY(recombine(P, in, Z));
        StepCall c;
        c.dt = dt * m;
        c.nb = 1;
        c.nsteps = 1;
        c.in = Z;
        c.is = nt;
        c.g = g;
        c.out_last = out;
        c.ols = nt;
        return run_steps(P, o->crs, c, nullptr);
    };
    if (o->init)
        for (int j = 0; j < Nc; ++j) TRY(coarse_step(U + (long long)j * nt, nullptr, U + (long long)(j + 1) * nt));
    CU(cudaMemsetAsync(E, 0, vb, P->stream));  // e_0 = 0
    pit_mgrit_stats st;
    memset(&st, 0, sizeof(st));
    int it = 0;
    bool conv = false;
    while (it < o->maxit) {
        // F-relaxation with Psi: per block, recombine all intervals' states,
        // then r fine steps; the last block writes r_{j+1} = Psi^{m/r}(u_j) - u_{j+1}
        const int nblk = m / r;
        const double *in = U;
        for (int q = 0; q < nblk; ++q) {
            double *w = (q % 2 == 0) ? W0 : W1;
            TRY(recombine(P, in, w, Nc));
            StepCall c;
            c.dt = dt;
            c.nb = Nc;
            c.nsteps = r;
            c.in = w;
            c.is = nt;
            if (o->forcing) {
                c.f = o->forcing + (long long)q * r * nt;
                c.fs = (long long)m * nt;
                c.fst = nt;
            }
            if (q + 1 < nblk) {
                double *wo = (q % 2 == 0) ? W1 : W0;
                c.out_last = wo;
                c.ols = nt;
                TRY(run_steps(P, o->fine, c, nullptr));
                // the next block recombines the block's outputs in place
                in = wo;
                // (recombine reads wo into its own scratch, then writes w of the next block)
            } else {
                c.out_last = GC;
                c.ols = nt;
                c.h = U + nt;
                c.hs = nt;
                c.hscale = -1.0;
                c.cmp = U + nt;
                c.cs = nt;
                c.norms = res;
                TRY(run_steps(P, o->fine, c, nullptr));
            }
        }
        CU(cudaMemcpyAsync(P->h_res.data(), res, sizeof(double) * G * Nc, cudaMemcpyDeviceToHost, P->stream));
        // coarse correction: e_{j+1} = Phi_c(Q e_j) + r_{j+1}; u_{j+1} += e_{j+1}
        for (int j = 0; j < Nc; ++j)
            TRY(coarse_step(E + (long long)j * nt, GC + (long long)j * nt, E + (long long)(j + 1) * nt));
        CU(launch_add_states(P->d_grids, G, nt, Nc, U + nt, E + nt, U + nt, nullptr, P->stream));
        count_kernels(P, 3);
        CU(cudaStreamSynchronize(P->stream));
        double rmax = 0.0;
        for (double v : P->h_res)
            if (!(v <= rmax)) rmax = v;
        if (it < PIT_MAX_HIST) st.res_hist[it] = rmax;
        ++it;
        if (!(rmax == rmax)) break;
        if (rmax <= o->tol) {
            conv = true;
            break;
        }
    }
    CU(cudaMemcpyAsync(uT, U + (long long)Nc * nt, vb, ptr_is_device(uT) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       P->stream));
    DevStats ds;
    TRY(read_stats(P, ds));
    st.max_cycles = it;
    st.n_converged = conv ? G : 0;
    st.phi_items = (long long)ds.items;
    st.krylov_iters = (long long)ds.sum_iters;
    st.point_iters = (long long)ds.point_iters;
    st.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    if (stats) *stats = st;
    TRY(status_of(ds));
    if (!conv) return fail(PIT_ERR_NOCONV, "global MGRIT did not meet tol within %d cycles", it);
    return PIT_OK;
}
}  // namespace

// CTMGRIT^loc (Alg. 3).  recomb = 0: one MGRIT solve over [t0, t1], the
// combination left to pit_combine.  recomb = s >= 1: the interval is split at
// the recombination steps tau_k = t0 + k (t1 - t0) / s; before each of the s
// intervals every grid's state is replaced by the projection of the combined
// solution onto its grid (Q of Eq. "overall_combination_operator"), then every
// grid runs MGRIT on the interval independently.
extern "C" pit_status pit_mgrit_solve(pit_problem_t P, const double *u0, const pit_mgrit_opts *o, double *uT,
                                      pit_mgrit_stats *stats)
{
    if (!P || !u0 || !uT || !o) return fail(PIT_ERR_INVALID_ARG, "NULL argument");
    if (o->recomb < 0) return fail(PIT_ERR_INVALID_ARG, "recomb must be >= 0");
    if (o->global_every < 0) return fail(PIT_ERR_INVALID_ARG, "global_every must be >= 0");
    if (o->global_every > 0) {
        TRY(check_solve_opts(&o->fine));
        TRY(check_solve_opts(&o->crs));
        if (o->m < 2 || o->nsteps < 1 || o->maxit < 1 || !(o->tol >= 0.0) || !(o->t1 > o->t0))
            return fail(PIT_ERR_INVALID_ARG, "need m >= 2, nsteps >= 1, maxit >= 1, tol >= 0, t1 > t0");
        if (o->forcing && !ptr_is_device(o->forcing)) return fail(PIT_ERR_INVALID_ARG, "forcing must be device memory");
        return mgrit_global(P, u0, o, uT, stats);
    }
    if (o->recomb == 0) return mgrit_run(P, u0, o, uT, stats);
    auto t_start = std::chrono::steady_clock::now();
    const int s = o->recomb;
    long long div = (long long)s * o->m * (o->levels == 3 ? o->m : 1);
    if (o->m < 2 || o->nsteps < 1 || o->nsteps % div != 0)
        return fail(PIT_ERR_INVALID_ARG, "nsteps must be a multiple of recomb x m^(levels-1)");
    const long long nt = P->ntot;
    const size_t vb = sizeof(double) * nt;
    const double *src;
    TRY(stage_in(P, P->w_in, u0, nt, &src));
    CU(P->rc_cur.ensure(2 * vb));
    double *cur = P->rc_cur.d(), *nxt = cur + nt;
    pit_mgrit_opts oi = *o;
    oi.recomb = 0;
    oi.nsteps = o->nsteps / s;
    pit_mgrit_stats tot;
    memset(&tot, 0, sizeof(tot));
    tot.n_converged = P->G;
    pit_status worst = PIT_OK;
    for (int k = 0; k < s; ++k) {
        if (o->forcing) oi.forcing = o->forcing + (long long)k * oi.nsteps * nt;
        oi.t0 = o->t0 + (o->t1 - o->t0) * k / s;
        oi.t1 = (k + 1 == s) ? o->t1 : o->t0 + (o->t1 - o->t0) * (k + 1) / s;
        TRY(recombine(P, k == 0 ? src : cur, cur));
        pit_mgrit_stats sk;
        memset(&sk, 0, sizeof(sk));
        const pit_status rs = mgrit_run(P, cur, &oi, nxt, &sk);
        if (rs != PIT_OK && rs != PIT_ERR_NOCONV) return rs;
        if (rs != PIT_OK) worst = rs;
        std::swap(cur, nxt);
        tot.max_cycles = sk.max_cycles > tot.max_cycles ? sk.max_cycles : tot.max_cycles;
        tot.n_converged = sk.n_converged < tot.n_converged ? sk.n_converged : tot.n_converged;
        for (int q = 0; q < PIT_MAX_HIST; ++q)
            if (!(sk.res_hist[q] <= tot.res_hist[q])) tot.res_hist[q] = sk.res_hist[q];
        tot.phi_items += sk.phi_items;
        tot.krylov_iters += sk.krylov_iters;
        tot.point_iters += sk.point_iters;
        tot.learned_used |= sk.learned_used;
        tot.fallback |= sk.fallback;
    }
    CU(cudaMemcpyAsync(uT, cur, vb, ptr_is_device(uT) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, P->stream));
    CU(cudaStreamSynchronize(P->stream));
    tot.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    if (stats) *stats = tot;
    if (worst != PIT_OK) return fail(worst, "a grid did not meet tol within maxit cycles on a recombination interval");
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
    const int chunks = combine_chunks(P->G, n_pts, P->n_sm);
    if (chunks > 1) CU(P->w_part.ensure(sizeof(double) * (size_t)chunks * n_pts));
    {
        ProfScope ps(P, 2);
        CU(launch_combine(P->d_grids, P->d_coef, P->d_levels, P->G, P->op, du, n_pts, dp, target, chunks,
                          chunks > 1 ? P->w_part.d() : nullptr, P->stream));
        count_kernels(P, 2, chunks > 1 ? 2 : 1);
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
    P->prof_allocs0 = g_dev_allocs.load();
    P->ev_used = 0;
    P->prof_recs.clear();
    P->prof_items = P->prof_point_iters = P->prof_point_passes = P->prof_point_steps = 0;
    for (long long &k : P->prof_kernels) k = 0;
    for (int f = 0; f < 2; ++f) P->prof_fam_iters[f] = P->prof_fam_passes[f] = P->prof_fam_steps[f] = 0;
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
    for (int f = 0; f < 4; ++f) out->kernels[f] = P->prof_kernels[f];
    for (int f = 0; f < 2; ++f) {
        out->point_iters_f[f] = P->prof_fam_iters[f];
        out->point_passes_f[f] = P->prof_fam_passes[f];
        out->point_steps_f[f] = P->prof_fam_steps[f];
    }
    out->device_allocs = g_dev_allocs.load() - P->prof_allocs0;
    out->phi_items = P->prof_items;
    out->point_iters = P->prof_point_iters;
    out->point_passes = P->prof_point_passes;
    out->point_steps = P->prof_point_steps;
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
    const int prec = prec_form(opts->prec);
    // the launch plan was made when the problem was created; planning here
    // would allocate, so a form without a plan is refused
    if (!P->planned[prec])
        return fail(PIT_ERR_UNSUPPORTED, "precision form %d is not supported on this problem (operator or grid "
                                         "sizes); pit_phi_batch gives the reason",
                    opts->prec);
    if (P->n_cls[prec][1] > 0)
        return fail(PIT_ERR_UNSUPPORTED, "this problem has grids whose solver state needs global scratch; "
                                         "pit_phi_batch_inplace_static cannot serve it");
    const bool wide = n_batch >= 8;
    const int family = wide ? 0 : 1;
    const int threads = P->threads[prec][family == 0 ? 1 : 0][0] ? P->threads[prec][family == 0 ? 1 : 0][0] : 128;
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
    a.order = P->d_order_cls[prec][0];
    a.n_order = P->n_cls[prec][0];
    // counters as in pit_phi_batch: the family of the batch width, both reset
    const bool want = stats || P->prof_on;
    if (want) TRY(reset_stats(P));
    a.stats = want ? P->d_stats + family : nullptr;
    {
        ProfScope ps(P, family);
        CU(launch_steps(prec, a, threads, P->smem_need[prec], P->stream));
        count_kernels(P, family);
    }
    CU(cudaMemcpyAsync(u, scratch, sizeof(double) * count, cudaMemcpyDeviceToDevice, P->stream));
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

// ---------------------------------------------------------------------------
// Learned coarse propagator: parameters, forward, loss gradient, training.
namespace {

float bf16_round_host(float v)
{
    uint32_t b;
    memcpy(&b, &v, 4);
    if ((b & 0x7f800000u) == 0x7f800000u) return v;
    b += 0x7fffu + ((b >> 16) & 1u);
    b &= 0xffff0000u;
    float r;
    memcpy(&r, &b, 4);
    return r;
}

// SplitMix64 (Steele, Lea, Flood 2014) and Box-Muller normals for the seeded
// training data.
struct Rng {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
    double normal()
    {
        const double u1 = 1.0 - uniform(), u2 = uniform();
        return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
    }
};

pit_status net_loss_grad_dev(pit_problem *P, double dT, int n_batch, const double *u, const double *y,
                             const NetTrainItem *items_host, int n_items, const float *w_dev, float *grad_dev,
                             double *loss_host)
{
    int nmax = 0;
    for (const GridInfo &I : P->info) nmax = I.n > nmax ? I.n : nmax;
    (void)n_batch;
    const long long slab = (long long)net_act_floats(nmax, true);
    CU(P->n_act.ensure(sizeof(float) * (size_t)(slab * n_items)));
    CU(P->n_rows.ensure(sizeof(float) * (size_t)PIT_NET_PARAMS * n_items));
    CU(P->n_loss.ensure(sizeof(double) * n_items));
    CU(P->n_items.ensure(sizeof(NetTrainItem) * n_items));
    CU(cudaMemcpyAsync(P->n_items.p, items_host, sizeof(NetTrainItem) * n_items, cudaMemcpyHostToDevice, P->stream));
    {
        ProfScope ps(P, 3);
        CU(launch_net_train(P->d_grids, (const NetTrainItem *)P->n_items.p, n_items, u, y, dT, w_dev,
                            (float *)P->n_act.p, slab, (float *)P->n_rows.p, P->n_loss.d(), P->op, P->stream));
        count_kernels(P, 3);
    }
    if (grad_dev)
        CU(launch_net_adam((const float *)P->n_rows.p, n_items, 1.0f, nullptr, nullptr, nullptr, nullptr, 0, 0, 0, 0, 0,
                           grad_dev, P->stream));
        count_kernels(P, 3);
    if (loss_host) {
        std::vector<double> l(n_items);
        CU(cudaMemcpyAsync(l.data(), P->n_loss.p, sizeof(double) * n_items, cudaMemcpyDeviceToHost, P->stream));
        CU(cudaStreamSynchronize(P->stream));
        double s = 0.0;
        for (int k = 0; k < n_items; ++k) s += l[k];
        *loss_host = s;
    }
    return PIT_OK;
}

}  // namespace

extern "C" pit_status pit_net_set_params(pit_problem_t P, const float *w, int n)
{
    if (!P || !w) return fail(PIT_ERR_INVALID_ARG, "NULL argument");
    if (n != PIT_NET_PARAMS) return fail(PIT_ERR_INVALID_ARG, "expected %d parameters, got %d", PIT_NET_PARAMS, n);
    for (int k = 0; k < n; ++k) {
        if (!std::isfinite(w[k])) return fail(PIT_ERR_NONFINITE, "parameter %d is not finite", k);
        P->h_net.w[k] = bf16_round_host(w[k]);
    }
    CU(P->n_master.ensure(sizeof(float) * n));
    CU(P->n_w.ensure(sizeof(float) * n));
    CU(cudaMemcpyAsync(P->n_master.p, w, sizeof(float) * n, cudaMemcpyHostToDevice, P->stream));
    CU(cudaMemcpyAsync(P->n_w.p, P->h_net.w, sizeof(float) * n, cudaMemcpyHostToDevice, P->stream));
    CU(cudaStreamSynchronize(P->stream));
    P->have_net = true;
    P->net_accepted = true;
    return PIT_OK;
}

extern "C" pit_status pit_net_get_params(pit_problem_t P, float *w, int n)
{
    if (!P || !w) return fail(PIT_ERR_INVALID_ARG, "NULL argument");
    if (n != PIT_NET_PARAMS) return fail(PIT_ERR_INVALID_ARG, "expected %d parameters, got %d", PIT_NET_PARAMS, n);
    if (!P->have_net) return fail(PIT_ERR_INVALID_ARG, "the network has no parameters yet");
    memcpy(w, P->h_net.w, sizeof(float) * n);
    return PIT_OK;
}

extern "C" pit_status pit_net_forward(pit_problem_t P, double dT, int n_batch, const double *u, double *out)
{
    if (!P || !u || !out || n_batch < 0) return fail(PIT_ERR_INVALID_ARG, "bad argument");
    if (!P->have_net) return fail(PIT_ERR_INVALID_ARG, "the network has no parameters yet");
    if (!(dT > 0.0) || !std::isfinite(dT)) return fail(PIT_ERR_INVALID_ARG, "dT must be finite and > 0");
    if (!ptr_is_device(u) || !ptr_is_device(out)) return fail(PIT_ERR_INVALID_ARG, "u and out must be device memory");
    StepCall c;
    c.dt = dT;
    c.nb = n_batch;
    c.nsteps = 1;
    c.in = u;
    c.is = P->ntot;
    c.out_last = out;
    c.ols = P->ntot;
    return run_net(P, c, nullptr);
}

extern "C" pit_status pit_net_loss_grad(pit_problem_t P, double dT, int n_batch, const double *u, const double *y,
                                        double *loss, float *grad)
{
    if (!P || !u || !y || !loss || !grad || n_batch < 1) return fail(PIT_ERR_INVALID_ARG, "bad argument");
    if (!P->have_net) return fail(PIT_ERR_INVALID_ARG, "the network has no parameters yet");
    if (!(dT > 0.0) || !std::isfinite(dT)) return fail(PIT_ERR_INVALID_ARG, "dT must be finite and > 0");
    if (!ptr_is_device(u) || !ptr_is_device(y)) return fail(PIT_ERR_INVALID_ARG, "u and y must be device memory");
    std::vector<NetTrainItem> items;
    for (int b = 0; b < n_batch; ++b)
        for (int g = 0; g < P->G; ++g) items.push_back({g, 0, (long long)b * P->ntot + P->off[g]});
    CU(P->n_grad.ensure(sizeof(float) * PIT_NET_PARAMS));
    TRY(net_loss_grad_dev(P, dT, n_batch, u, y, items.data(), (int)items.size(), (const float *)P->n_w.p,
                          (float *)P->n_grad.p, loss));
    CU(cudaMemcpyAsync(grad, P->n_grad.p, sizeof(float) * PIT_NET_PARAMS, cudaMemcpyDeviceToHost, P->stream));
    CU(cudaStreamSynchronize(P->stream));
    return PIT_OK;
}

extern "C" pit_status pit_train_coarse(pit_problem_t P, const pit_train_opts *o, pit_train_stats *stats)
{
    if (!P || !o) return fail(PIT_ERR_INVALID_ARG, "NULL argument");
    TRY(check_solve_opts(&o->fine));
    TRY(check_solve_opts(&o->crs));
    if (!(o->dt_fine > 0.0) || o->m < 1 || o->n_pairs < 1 || o->n_holdout < 1 || o->epochs < 1 || o->batch < 1 ||
        !(o->lr > 0.0) || o->ic_modes < 1 || o->ic_fmax < 1 || o->traj_len < 1 ||
        !(o->accept_ratio > 0.0 && o->accept_ratio <= 1.0))
        return fail(PIT_ERR_INVALID_ARG, "invalid training options");
    auto t0 = std::chrono::steady_clock::now();
    const int G = P->G, d = P->desc.d;
    const long long nt = P->ntot;
    const double dT = o->dt_fine * o->m;
    // --- data: n_states packed pair states (training, then held-out)
    const int n_train_states = (o->n_pairs + G - 1) / G;
    const int n_hold_states = (o->n_holdout + G - 1) / G;
    const int n_states = n_train_states + n_hold_states;
    const int n_traj = (n_states + o->traj_len - 1) / o->traj_len;
    CU(P->n_U.ensure(sizeof(double) * nt * (size_t)n_traj * o->traj_len));
    CU(P->n_Y.ensure(sizeof(double) * nt * (size_t)n_traj * o->traj_len));
    double *Ud = P->n_U.d(), *Yd = P->n_Y.d();
    Rng rng{o->seed};
    std::vector<double> prm(1 + o->ic_modes * (d + 1));
    CU(P->n_prm.ensure(sizeof(double) * prm.size()));
    TRY(reset_stats(P));
    for (int tr = 0; tr < n_traj; ++tr) {
        // seeded random initial value: sum of product-sine modes
        prm[0] = o->ic_modes;
        for (int k = 0; k < o->ic_modes; ++k) {
            prm[1 + k * (d + 1)] = rng.normal();
            for (int i = 0; i < d; ++i)
                prm[2 + k * (d + 1) + i] = 1 + (int)(rng.uniform() * o->ic_fmax) % o->ic_fmax;
        }
        CU(cudaMemcpyAsync(P->n_prm.p, prm.data(), sizeof(double) * prm.size(), cudaMemcpyHostToDevice, P->stream));
        double *u0 = Ud + (long long)tr * o->traj_len * nt;
        CU(launch_initial(P->d_grids, G, P->op, P->d_hi, 0, P->n_prm.d(), (int)prm.size(), u0, P->stream));
        count_kernels(P, 3);
        // pair k: (u_k, u_{k+1} = Phi^m u_k), u_{k+1} also the input of pair k+1
        for (int k = 0; k < o->traj_len; ++k) {
            StepCall c;
            c.dt = o->dt_fine;
            c.nb = 1;
            c.nsteps = o->m;
            c.in = u0 + (long long)k * nt;
            c.is = nt;
            c.out_last = Yd + ((long long)tr * o->traj_len + k) * nt;
            c.ols = nt;
            TRY(run_steps(P, o->fine, c, nullptr));
            if (k + 1 < o->traj_len)
                CU(cudaMemcpyAsync(u0 + (long long)(k + 1) * nt, c.out_last, sizeof(double) * nt,
                                   cudaMemcpyDeviceToDevice, P->stream));
        }
    }
    DevStats ds;
    TRY(read_stats(P, ds));
    TRY(status_of(ds));
    auto t1 = std::chrono::steady_clock::now();
    // training and held-out items: state p < n_train_states is training
    std::vector<NetTrainItem> train, hold;
    for (int p = 0; p < n_states; ++p)
        for (int g = 0; g < G; ++g) {
            NetTrainItem it{g, 0, (long long)p * nt + P->off[g]};
            if (p < n_train_states) train.push_back(it);
            else hold.push_back(it);
        }
    if ((int)train.size() > o->n_pairs) train.resize(o->n_pairs);
    if ((int)hold.size() > o->n_holdout) hold.resize(o->n_holdout);
    // --- parameters: FP32 master weights, He-scaled normals, last layer zero
    //     (the network starts as the identity map)
    std::vector<float> w0(PIT_NET_PARAMS, 0.0f);
    {
        int pos = 0;
        const int cin[4] = {3, 17, 17, 17}, cout[4] = {16, 16, 16, 1};
        for (int k = 0; k < 4; ++k) {
            const int nw = cout[k] * cin[k] * 5;
            const double sd = (k == 3) ? 0.0 : sqrt(2.0 / (cin[k] * 5.0 * d));
            for (int q = 0; q < nw; ++q) w0[pos + q] = (float)(sd * rng.normal());
            pos += nw + cout[k];
        }
    }
    CU(P->n_master.ensure(sizeof(float) * PIT_NET_PARAMS));
    CU(P->n_w.ensure(sizeof(float) * PIT_NET_PARAMS));
    CU(P->n_m.ensure(sizeof(float) * PIT_NET_PARAMS));
    CU(P->n_v.ensure(sizeof(float) * PIT_NET_PARAMS));
    std::vector<float> wr(PIT_NET_PARAMS);
    for (int k = 0; k < PIT_NET_PARAMS; ++k) wr[k] = bf16_round_host(w0[k]);
    CU(cudaMemcpyAsync(P->n_master.p, w0.data(), sizeof(float) * PIT_NET_PARAMS, cudaMemcpyHostToDevice, P->stream));
    CU(cudaMemcpyAsync(P->n_w.p, wr.data(), sizeof(float) * PIT_NET_PARAMS, cudaMemcpyHostToDevice, P->stream));
    CU(cudaMemsetAsync(P->n_m.p, 0, sizeof(float) * PIT_NET_PARAMS, P->stream));
    CU(cudaMemsetAsync(P->n_v.p, 0, sizeof(float) * PIT_NET_PARAMS, P->stream));
    int nmax = 0;
    for (const GridInfo &I : P->info) nmax = I.n > nmax ? I.n : nmax;
    const long long slab = (long long)net_act_floats(nmax, true);
    const int B = o->batch < (int)train.size() ? o->batch : (int)train.size();
    CU(P->n_act.ensure(sizeof(float) * (size_t)(slab * B)));
    CU(P->n_rows.ensure(sizeof(float) * (size_t)PIT_NET_PARAMS * B));
    const int steps_per_epoch = ((int)train.size() + B - 1) / B;
    CU(P->n_loss.ensure(sizeof(double) * (size_t)B * steps_per_epoch));
    CU(P->n_items.ensure(sizeof(NetTrainItem) * (size_t)B * steps_per_epoch));
    std::vector<double> losses((size_t)B * steps_per_epoch);
    pit_train_stats st;
    memset(&st, 0, sizeof(st));
    int t = 0;
    std::vector<NetTrainItem> order(train);
    for (int ep = 0; ep < o->epochs; ++ep) {
        for (int k = (int)order.size() - 1; k > 0; --k) std::swap(order[k], order[rng.next() % (uint64_t)(k + 1)]);
        CU(cudaMemcpyAsync(P->n_items.p, order.data(), sizeof(NetTrainItem) * order.size(), cudaMemcpyHostToDevice,
                           P->stream));
        int n_loss = 0;
        for (int s0 = 0; s0 < (int)order.size(); s0 += B) {
            const int nb = ((int)order.size() - s0) < B ? ((int)order.size() - s0) : B;
            {
                ProfScope ps(P, 3);
                CU(launch_net_train(P->d_grids, (const NetTrainItem *)P->n_items.p + s0, nb, Ud, Yd, dT,
                                    (const float *)P->n_w.p, (float *)P->n_act.p, slab, (float *)P->n_rows.p,
                                    P->n_loss.d() + s0, P->op, P->stream));
                count_kernels(P, 3);
            }
            ++t;
            CU(launch_net_adam((const float *)P->n_rows.p, nb, 1.0f / nb, (float *)P->n_master.p, (float *)P->n_m.p,
                               (float *)P->n_v.p, (float *)P->n_w.p, (float)o->lr, 0.9f, 0.999f, 1e-8f, t, nullptr,
                               P->stream));
            count_kernels(P, 3);
            n_loss += nb;
        }
        if (ep == 0 || ep == o->epochs - 1) {
            CU(cudaMemcpyAsync(losses.data(), P->n_loss.p, sizeof(double) * n_loss, cudaMemcpyDeviceToHost, P->stream));
            CU(cudaStreamSynchronize(P->stream));
            double sum = 0.0;
            for (int k = 0; k < n_loss; ++k) sum += losses[k];
            const double mean = sum / n_loss;
            if (!std::isfinite(mean)) return fail(PIT_ERR_NONFINITE, "training loss is not finite (epoch %d)", ep);
            if (ep == 0) st.loss_first_epoch = mean;
            st.loss_last_epoch = mean;
        }
    }
    CU(cudaMemcpyAsync(P->h_net.w, P->n_w.p, sizeof(float) * PIT_NET_PARAMS, cudaMemcpyDeviceToHost, P->stream));
    CU(cudaStreamSynchronize(P->stream));
    P->have_net = true;
    st.adam_steps = t;
    auto t2 = std::chrono::steady_clock::now();
    // --- judge on the held-out pairs: learned vs implicit coarse step
    const int n_hold_states_used = n_hold_states;
    const double *Uh = Ud + (long long)n_train_states * nt, *Yh = Yd + (long long)n_train_states * nt;
    CU(P->n_tmp.ensure(sizeof(double) * nt * (size_t)n_hold_states_used * 2));
    double *Ln = P->n_tmp.d(), *Li = Ln + (long long)n_hold_states_used * nt;
    StepCall c;
    c.dt = dT;
    c.nb = n_hold_states_used;
    c.nsteps = 1;
    c.in = Uh;
    c.is = nt;
    c.out_last = Ln;
    c.ols = nt;
    TRY(run_net(P, c, nullptr));
    c.out_last = Li;
    TRY(reset_stats(P));
    TRY(run_steps(P, o->crs, c, nullptr));
    TRY(read_stats(P, ds));
    TRY(status_of(ds));
    std::vector<double> hy((size_t)nt * n_hold_states_used), hn(hy.size()), hi(hy.size());
    CU(cudaMemcpyAsync(hy.data(), Yh, sizeof(double) * hy.size(), cudaMemcpyDeviceToHost, P->stream));
    CU(cudaMemcpyAsync(hn.data(), Ln, sizeof(double) * hn.size(), cudaMemcpyDeviceToHost, P->stream));
    CU(cudaMemcpyAsync(hi.data(), Li, sizeof(double) * hi.size(), cudaMemcpyDeviceToHost, P->stream));
    CU(cudaStreamSynchronize(P->stream));
    double el = 0.0, ei = 0.0;
    for (const NetTrainItem &it : hold) {
        const long long off = it.off - (long long)n_train_states * nt;
        const int n = P->info[it.g].n;
        double yy = 0.0, dl = 0.0, di = 0.0;
        for (int j = 0; j < n; ++j) {
            const double yv = hy[off + j];
            yy += yv * yv;
            dl += (hn[off + j] - yv) * (hn[off + j] - yv);
            di += (hi[off + j] - yv) * (hi[off + j] - yv);
        }
        if (yy > 0.0) {
            el += sqrt(dl / yy);
            ei += sqrt(di / yy);
        }
    }
    st.holdout_err_learned = el / hold.size();
    st.holdout_err_implicit = ei / hold.size();
    st.accepted = (st.holdout_err_learned <= o->accept_ratio * st.holdout_err_implicit) ? 1 : 0;
    P->net_accepted = st.accepted != 0;
    st.ms_data = std::chrono::duration<double, std::milli>(t1 - t0).count();
    st.ms_train = std::chrono::duration<double, std::milli>(t2 - t1).count();
    if (stats) *stats = st;
    return PIT_OK;
}
