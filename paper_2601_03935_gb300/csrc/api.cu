// Host side of the GSIS C ABI: validation, geometry preprocessing, device buffers and
// the orchestration of one outer iteration (Section 3) on the context stream.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <array>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "../../include/gsis.h"
#include "gsis_impl.cuh"

using namespace gsis;

namespace {

enum KernelId {
    K_COEF, K_WALL, K_SLOPE_GAS, K_SWEEP_GAS, K_SLOPE_PHOTON, K_SWEEP_PHOTON, K_FINISH, K_EPS, K_EQUIL, K_MOMENTS,
    K_KBFLUX, K_HOT, K_MGRAD, K_MBFLUX, K_MRES, K_MNORM, K_MJACOBI, K_MCONV, K_SYNC, K_MLP, K_COUNT
};
const char *kKernelNames[K_COUNT] = {"coefficients", "wall_density",  "slopes_gas",    "sweep_gas",
                                     "slopes_photon", "sweep_photon", "finish",        "eps_reduce",
                                     "equilibrium",  "moments_only",  "kinetic_bflux", "macro_hot",
                                     "macro_grad",   "macro_bflux",   "macro_residual", "macro_norm",
                                     "macro_jacobi", "macro_convert", "sync",          "mlp"};

}  // namespace

struct gsis_ctx {
    int dim = 0, precision = 0, order = 2, block = 16;
    int64_t nc = 0;
    int V = 0, Vp = 0, NO = 0, Op = 0, nch = 0, och = 0, n_bf = 0;
    size_t real_size = 4;
    cudaStream_t stream = nullptr;
    ModelDev model{};
    gsis_solver_params solver{};

    // device buffers; Real-typed ones are void* and cast by precision
    void *f[2] = {nullptr, nullptr}, *I[2] = {nullptr, nullptr};
    int cur = 0;
    // staged uploads (created on first use): a buffer pair with the layout of f[cur] and
    // I[cur] filled on a copy stream while the context stream computes; stage_ready marks
    // the copy done, stage_free the point after which the context stream no longer reads
    // the pair's previous contents
    void *f_stage = nullptr, *I_stage = nullptr;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t stage_ready = nullptr, stage_free = nullptr;
    // the photon slope pass and sweep run on side_stream, between fork_ev (recorded on the
    // context stream after the wall densities) and join_ev (waited on before the moments
    // are finished), concurrently with the gas kernels; created on first use
    cudaStream_t side_stream = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    bool staged = false;
    void *coef = nullptr, *bcoef = nullptr, *partial = nullptr, *opartial = nullptr;
    // defect correction (solver.defect_correction): coefficients of M^{k+1/2}, the moment
    // rows of the kinetic residual at f^{k+1/2} and the synthetic residual's offset
    void *coef_h = nullptr;
    double *rrow = nullptr, *moff = nullptr;
    void *sync_kc = nullptr;                    // FP32: per-cell synchronisation constants [nc][SYNC_KC] floats
    void *fface = nullptr, *oface = nullptr;    // upwind face values [n_fi][Vp][4], [n_fi][Op] (order 2)
    double *fields = nullptr, *fields_old = nullptr, *eps_terms = nullptr, *eps_sums = nullptr;
    int *err = nullptr;
    double *vol = nullptr, *cell_dx = nullptr;
    int *bf_cell = nullptr, *bf_patch = nullptr, *g_stn = nullptr;
    int4 *g_info = nullptr;
    int2 *g_fnb = nullptr;
    void *g_fgeo = nullptr, *g_lsq = nullptr, *g_eps2 = nullptr, *bf_nrm = nullptr;
    void *vq_x = nullptr, *vq_w = nullptr, *oq_x = nullptr, *oq_w = nullptr;
    double *patch_T = nullptr, *patch_u = nullptr, *bf_inc = nullptr, *eps_part = nullptr;
    unsigned int *eps_ticket = nullptr;
    int *patch_kind = nullptr;
    double *h_pinned = nullptr;  // NEPS sums + error word

    // synthetic equations (FP64): geometry, quadratures in FP64, state and work arrays
    MacroGeom mg{};
    bool closed = true;          // walls only: the synthetic solution keeps the mass
    MlpDev mlp;                  // learned closure (allocated on first use)
    std::vector<void *> mlp_alloc;
    float *mlp_X = nullptr, *mlp_Y = nullptr;   // per-cell features / predictions [nc][16], [nc][12]
    int *mlp_idx = nullptr;
    float *mlp_data = nullptr;   // training data on the device
    int64_t mlp_data_cap = 0;
    int mfp32 = 0;               // FP32 path: residual side of the synthetic equations and the
                                 // relaxation's flux increments in FP32 (1), or that except the
                                 // last MACRO_TAIL inner iterations (2)
    int tcm = 0;                 // FP32 path: gas moments on tensor cores (1: standalone passes, 2: also the sweep)
    int tc_wait = 1 << 22;       // polls of the first tensor-core completion wait (gsis_set_wait_limit)
    int *m_fi_i = nullptr, *m_fi_j = nullptr, *m_cface = nullptr, *m_pkind = nullptr;
    double *m_fi_n = nullptr, *m_fi_S = nullptr, *m_fi_dn = nullptr, *m_fi_dist = nullptr, *m_fi_t = nullptr,
           *m_fi_dx = nullptr, *m_lsq = nullptr, *m_eps2 = nullptr, *m_bf_n = nullptr,
           *m_bf_S = nullptr, *m_bf_dn = nullptr, *m_pstate = nullptr;
    double *vqd_x = nullptr, *vqd_w = nullptr, *oqd_x = nullptr, *oqd_w = nullptr;
    double *W[2] = {nullptr, nullptr}, *mq = nullptr, *mgrad = nullptr, *mphi = nullptr, *Rg = nullptr,
           *Dinv = nullptr, *gam = nullptr, *dG[2] = {nullptr, nullptr}, *rpart = nullptr, *hot = nullptr,
           *hot_b = nullptr, *kbf = nullptr, *mbf = nullptr, *fields_h = nullptr, *fields_n = nullptr,
           *mhist = nullptr;
    MacroState *mstate = nullptr;
    MacroState *h_mstate = nullptr;   // pinned: initial state and the polled stop flag
    int last_inner = 0;
    cudaGraphExec_t macro_exec = nullptr;   // POLL inner iterations, captured once
    cudaGraphExec_t macro_exec64 = nullptr; // the same with the FP64 residual side (mixed schedule's tail)
    int macro_nodes = 0, macro_nodes64 = 0;

    // velocity sharding (gsis_shard_setup): this context holds one contiguous range of the
    // velocities and photon directions; per-cell moment sums, wall outflow and kinetic
    // boundary-flux sums go through xbuf [n_cells][NXC] | [n_bf] | [n_bf][KBR], which the
    // caller sums over the ranks between the phase calls; wout_g keeps the summed wall
    // outflow of the current f for the next wall density
    bool sharded = false;
    double *xbuf = nullptr, *wout_g = nullptr;
    int64_t xcount = 0;
    int shard_state = 0;         // 0 idle, 1 after begin (CIS) / mid, 2 after begin (GSIS), 3 after refresh
    int shard_nxt = 0;
    int Vd = 0, Vdp = 0, NOd = 0, Odp = 0;   // sizes of the FP64 quadratures of the synthetic equations
    std::vector<double> h_wall;  // per boundary face: wall flag, normal[3], wall T, wall u[3]
    int *bf_tab = nullptr, *refl_v = nullptr, *refl_o = nullptr;   // mirror-plane reflection tables
    bool mirrors = false;

    bool have_eps = false;
    double last_eps = 0.0;
    // outer iterations since the distributions were last set (the CIS preconditioning of
    // gsis_solve counts from here) and the convergence measure of each one that was read
    int64_t iter = 0;
    bool eps_pending = false;
    std::vector<double> eps_hist;
    bool prof = false;
    double prof_ms[K_COUNT] = {0};
    int64_t prof_n[K_COUNT] = {0};
    struct Pending { int id; cudaEvent_t e0, e1; };
    std::vector<Pending> pending;          // recorded, not yet resolved
    std::vector<cudaEvent_t> event_pool;   // free events
    int64_t launches = 0;
    std::vector<void *> allocations;
    std::string last_error;
};

namespace {

int fail(gsis_ctx *c, int code, const std::string &msg) {
    if (c) c->last_error = msg;
    return code;
}

#define CUDA_TRY(c, expr)                                                                         \
    do {                                                                                          \
        cudaError_t _e = (expr);                                                                  \
        if (_e != cudaSuccess)                                                                    \
            return fail((c), GSIS_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

template <typename T>
int dalloc(gsis_ctx *c, T **p, size_t n) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
    if (e != cudaSuccess) return fail(c, GSIS_ERR_OUT_OF_MEMORY, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    c->allocations.push_back(q);
    *p = static_cast<T *>(q);
    return GSIS_OK;
}

int dalloc_real(gsis_ctx *c, void **p, size_t n) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, n * c->real_size > 0 ? n * c->real_size : 16);
    if (e != cudaSuccess) return fail(c, GSIS_ERR_OUT_OF_MEMORY, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    c->allocations.push_back(q);
    *p = q;
    return GSIS_OK;
}

// upload a host double array as Real
int upload_real(gsis_ctx *c, void *dst, const std::vector<double> &src) {
    if (c->precision == GSIS_FP64) {
        CUDA_TRY(c, cudaMemcpy(dst, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice));
    } else {
        std::vector<float> t(src.begin(), src.end());
        CUDA_TRY(c, cudaMemcpy(dst, t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    return GSIS_OK;
}

template <typename T>
int upload(gsis_ctx *c, T *dst, const std::vector<T> &src) {
    CUDA_TRY(c, cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return GSIS_OK;
}

template <typename Real>
Geom<Real> geom(const gsis_ctx *c) {
    Geom<Real> g;
    g.n_cells = (int)c->nc;
    g.dim = c->dim;
    g.block = c->block;
    g.tc = c->tcm >= 2 && MT % c->block == 0;
    g.info = c->g_info;
    g.fnb = c->g_fnb;
    g.cface = c->m_cface;
    g.fgeo = (const Real *)c->g_fgeo;
    g.stn = c->g_stn;
    g.lsq = (const Real *)c->g_lsq;
    g.eps2 = (const Real *)c->g_eps2;
    g.n_bf = c->n_bf;
    g.bf_cell = c->bf_cell;
    g.bf_patch = c->bf_patch;
    g.bf_nrm = (const Real *)c->bf_nrm;
    g.tc_wait = c->tc_wait;
    g.pos_theta = (Real)c->solver.positivity;
    g.err = c->err;
    g.bf_tab = c->bf_tab;
    g.refl_v = c->refl_v;
    g.refl_o = c->refl_o;
    g.resid = 0;
    return g;
}

template <typename Real>
Quad<Real> vquad(const gsis_ctx *c) {
    return Quad<Real>{c->V, c->Vp, (const Real *)c->vq_x, (const Real *)c->vq_w};
}
template <typename Real>
Quad<Real> oquad(const gsis_ctx *c) {
    return Quad<Real>{c->NO, c->Op, (const Real *)c->oq_x, (const Real *)c->oq_w};
}

int take_event(gsis_ctx *c, cudaEvent_t *e) {
    if (!c->event_pool.empty()) {
        *e = c->event_pool.back();
        c->event_pool.pop_back();
        return GSIS_OK;
    }
    CUDA_TRY(c, cudaEventCreate(e));
    return GSIS_OK;
}

// Resolve recorded launch timings (synchronises on the last recorded event).
int resolve_profile(gsis_ctx *c) {
    for (auto &p : c->pending) {
        CUDA_TRY(c, cudaEventSynchronize(p.e1));
        float ms = 0.f;
        CUDA_TRY(c, cudaEventElapsedTime(&ms, p.e0, p.e1));
        c->prof_ms[p.id] += ms;
        c->prof_n[p.id] += 1;
        c->event_pool.push_back(p.e0);
        c->event_pool.push_back(p.e1);
    }
    c->pending.clear();
    return GSIS_OK;
}

// Launch bracket: counts launches and, when profiling, brackets the launch with two
// events on the stream it is launched on (`st`, the context stream unless given; resolved
// later, so the stream never stalls).
template <typename F>
int launch(gsis_ctx *c, int id, F &&fn, cudaStream_t st = nullptr) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!st) st = c->stream;
    if (c->prof) {
        if (take_event(c, &e0) != GSIS_OK || take_event(c, &e1) != GSIS_OK) return GSIS_ERR_CUDA;
        CUDA_TRY(c, cudaEventRecord(e0, st));
    }
    cudaError_t e = fn();
    if (e != cudaSuccess)
        return fail(c, GSIS_ERR_CUDA, std::string("launch of ") + kKernelNames[id] + ": " + cudaGetErrorString(e));
    c->launches++;
    if (c->prof) {
        CUDA_TRY(c, cudaEventRecord(e1, st));
        c->pending.push_back({id, e0, e1});
    }
    return GSIS_OK;
}

#define TRY(expr)                 \
    do {                          \
        int _r = (expr);          \
        if (_r != GSIS_OK) return _r; \
    } while (0)

// moments of the current distributions -> fields (FP64): a first pass about zero
// velocity, a second about the velocity it found
template <typename Real>
int refresh_fields(gsis_ctx *c) {
    const Geom<Real> g = geom<Real>(c);
    CUDA_TRY(c, cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
    // the first pass takes moments about zero velocity, independent of earlier state
    CUDA_TRY(c, cudaMemsetAsync(c->coef, 0, (size_t)c->nc * cf::NC * c->real_size, c->stream));
    for (int pass = 0; pass < 2; ++pass) {
        TRY(launch(c, K_MOMENTS, [&] {
            return launch_moments_only<Real>(c->stream, c->dim, (int)c->nc, c->tcm >= 1, vquad<Real>(c), oquad<Real>(c),
                                             (const Real *)c->coef, (const Real *)c->f[c->cur],
                                             (const Real *)c->I[c->cur], (Real *)c->partial, (Real *)c->opartial,
                                             c->tc_wait, c->err);
        }));
        TRY(launch(c, K_FINISH, [&] {
            return launch_finish<Real>(c->stream, c->dim, (int)c->nc, c->nch, c->och, c->model, (const Real *)c->coef,
                                       (const Real *)c->partial, (const Real *)c->opartial, c->vol, nullptr,
                                       c->fields, c->eps_terms, c->err, 0);
        }));
        TRY(launch(c, K_COEF, [&] {
            return launch_coefficients<Real>(c->stream, c->dim, g, c->model, c->fields, c->cell_dx, (Real *)c->coef);
        }));
    }
    c->have_eps = false;
    c->eps_pending = false;
    c->iter = 0;
    c->eps_hist.clear();
    return GSIS_OK;
}

int refresh(gsis_ctx *c) { return c->precision == GSIS_FP64 ? refresh_fields<double>(c) : refresh_fields<float>(c); }

// The kinetic step of Eq. (dis_micro) from f^k (buffers cur) into buffers nxt, with the
// moment partials of f^{k+1/2}; coefficients are current (built from the fields of f^k).
template <typename Real>
int kinetic_step(gsis_ctx *c, int nxt) {
    const Geom<Real> g = geom<Real>(c);
    TRY(launch(c, K_WALL, [&] {
        return launch_wall_density<Real>(c->stream, c->dim, g, vquad<Real>(c), c->patch_T, c->bf_inc, c->patch_kind,
                                         (const Real *)c->f[c->cur], c->sharded ? c->wout_g : nullptr,
                                         (Real *)c->bcoef);
    }));
    // photon transport is independent of the gas planes: it runs on the side stream
    if (!c->side_stream) {   // the events first: a side stream implies both events exist
        cudaEvent_t e = nullptr;
        if (!c->fork_ev) {
            CUDA_TRY(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            c->fork_ev = e;
        }
        if (!c->join_ev) {
            CUDA_TRY(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            c->join_ev = e;
        }
        cudaStream_t st = nullptr;
        CUDA_TRY(c, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        c->side_stream = st;
    }
    CUDA_TRY(c, cudaEventRecord(c->fork_ev, c->stream));
    CUDA_TRY(c, cudaStreamWaitEvent(c->side_stream, c->fork_ev, 0));
    const cudaStream_t ps = c->side_stream;
    if (c->order == 2) {
        TRY(launch(c, K_SLOPE_PHOTON, [&] {
            return launch_slopes<Real>(ps, c->dim, 1, g, oquad<Real>(c), (const Real *)c->I[c->cur],
                                       (Real *)c->oface);
        }, ps));
    }
    TRY(launch(c, K_SWEEP_PHOTON, [&] {
        return launch_sweep_photon<Real>(ps, c->dim, c->order, g, oquad<Real>(c), (const Real *)c->coef,
                                         (const Real *)c->bcoef, (const Real *)c->I[c->cur], (const Real *)c->oface,
                                         (Real *)c->I[nxt], (Real *)c->opartial);
    }, ps));
    CUDA_TRY(c, cudaEventRecord(c->join_ev, ps));
    if (c->order == 2) {
        TRY(launch(c, K_SLOPE_GAS, [&] {
            return launch_slopes<Real>(c->stream, c->dim, 4, g, vquad<Real>(c), (const Real *)c->f[c->cur],
                                       (Real *)c->fface);
        }));
    }
    TRY(launch(c, K_SWEEP_GAS, [&] {
        return launch_sweep_gas<Real>(c->stream, c->dim, c->order, g, vquad<Real>(c), (const Real *)c->coef,
                                      (const Real *)c->bcoef, (const Real *)c->f[c->cur], (const Real *)c->fface,
                                      (Real *)c->f[nxt], (Real *)c->partial);
    }));
    CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->join_ev, 0));
    return GSIS_OK;
}

// fields of the new distribution from the partials, epsilon against the fields of f^k,
// coefficients for the next iteration, and the asynchronous read-back of epsilon
template <typename Real>
int close_iteration(gsis_ctx *c, int nxt) {
    const Geom<Real> g = geom<Real>(c);
    std::swap(c->fields, c->fields_old);
    TRY(launch(c, K_FINISH, [&] {
        return launch_finish<Real>(c->stream, c->dim, (int)c->nc, c->nch, c->och, c->model, (const Real *)c->coef,
                                   (const Real *)c->partial, (const Real *)c->opartial, c->vol, c->fields_old,
                                   c->fields, c->eps_terms, c->err, 1, c->eps_part, c->eps_ticket, c->eps_sums);
    }));
    TRY(launch(c, K_COEF, [&] {
        return launch_coefficients<Real>(c->stream, c->dim, g, c->model, c->fields, c->cell_dx, (Real *)c->coef);
    }));
    CUDA_TRY(c, cudaMemcpyAsync(c->h_pinned, c->eps_sums, NEPS * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->h_pinned + NEPS, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    c->cur = nxt;
    c->have_eps = true;
    c->eps_pending = true;
    ++c->iter;
    return GSIS_OK;
}

// One CIS iteration: f^{k+1} = f^{k+1/2}.
template <typename Real>
int cis_iteration(gsis_ctx *c) {
    const int nxt = 1 - c->cur;
    CUDA_TRY(c, cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
    TRY(kinetic_step<Real>(c, nxt));
    return close_iteration<Real>(c, nxt);
}

QuadD vquad_d(const gsis_ctx *c) { return QuadD{c->Vd, c->Vdp, c->vqd_x, c->vqd_w}; }
QuadD oquad_d(const gsis_ctx *c) { return QuadD{c->NOd, c->Odp, c->oqd_x, c->oqd_w}; }

// Pseudo-time iterations of the synthetic equations from W[0] until ||R|| <= tol_inner
// ||R_0|| or max_inner; returns the index of the buffer that holds the result.  The
// device stop flag is polled every POLL iterations (one stream synchronisation each).
// enqueue one inner iteration reading W[w] and writing W[1 - w]; returns a CUDA status
// fp32: the residual side of this iteration in FP32.
cudaError_t enqueue_inner(gsis_ctx *c, int w, int fp32, int *kernels) {
    const MacroGeom &g = c->mg;
    const gsis_solver_params &sp = c->solver;
    const int nparts = macro_rpart_count((int)c->nc);
    const int sweeps = std::max(sp.macro_sweeps, 1);
    cudaError_t e;
    if ((e = launch_macro_grad(c->stream, g, c->order, fp32, c->model, c->mstate, c->W[w], c->mq, c->mgrad, c->mphi)))
        return e;
    if ((e = launch_macro_bflux(c->stream, g, fp32, c->model, vquad_d(c), oquad_d(c), c->mstate, c->mq, c->mbf))) return e;
    if ((e = launch_macro_residual(c->stream, g, c->order, fp32, c->model, sp.cfl_macro, c->mstate, c->W[w], c->mq,
                                   c->mgrad, c->mphi, c->hot, c->mbf, c->hot_b, c->Rg, c->Dinv, c->gam, c->rpart)))
        return e;
    if ((e = launch_macro_norm(c->stream, nparts, c->rpart, c->mstate, c->mhist))) return e;
    for (int sw = 0; sw < sweeps; ++sw)
        if ((e = launch_macro_jacobi(c->stream, g, fp32, c->model, c->mstate, sw == 0, sw == sweeps - 1, c->W[w],
                                     c->mq, c->Rg, c->Dinv, c->gam, c->dG[sw & 1], c->dG[(sw + 1) & 1],
                                     c->W[1 - w])))
            return e;
    *kernels += 4 + sweeps - (g.n_bf == 0 ? 1 : 0);
    return cudaSuccess;
}

// Pseudo-time iterations of the synthetic equations from W[0] until ||R|| <= tol_inner
// ||R_0|| or max_inner; returns the index of the buffer that holds the result.  Every
// kernel returns at once after the device stop flag is set, so the host polls the flag
// only every POLL iterations (one stream synchronisation each).  Without kernel
// profiling, and on a non-default stream, the POLL iterations are a CUDA graph captured
// once per context.
// Captures POLL inner iterations (residual side in FP32 when fp32) as one graph.
int capture_inner(gsis_ctx *c, int fp32, cudaGraphExec_t *exec, int *nodes_out) {
    constexpr int POLL = 8;
    cudaGraph_t gr = nullptr;
    int nodes = 0;
    CUDA_TRY(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < POLL && e == cudaSuccess; ++k) e = enqueue_inner(c, k & 1, fp32, &nodes);
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &gr);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        return fail(c, GSIS_ERR_CUDA, std::string("capture of the synthetic solve: ") +
                                          cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(exec, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
        *exec = nullptr;
        return fail(c, GSIS_ERR_CUDA, std::string("graph instantiation: ") + cudaGetErrorString(e));
    }
    *nodes_out = nodes;
    return GSIS_OK;
}

int macro_solve(gsis_ctx *c, int *w_out) {
    constexpr int POLL = 8;
    constexpr int MACRO_TAIL = 16;   // FP64 inner iterations that end a mixed-precision solve
    const gsis_solver_params &sp = c->solver;
    const bool mixed = c->mfp32 == 2;
    const int fp_main = c->mfp32 != 0 ? 1 : 0;
    const int tail = mixed ? std::min(MACRO_TAIL, sp.max_inner) : 0;
    c->h_mstate->it = 0;
    c->h_mstate->done = 0;
    c->h_mstate->max_inner = sp.max_inner - tail;
    c->h_mstate->r0 = 0.0;
    c->h_mstate->rn = 0.0;
    c->h_mstate->tol = sp.tol_inner;
    CUDA_TRY(c, cudaMemcpyAsync(c->mstate, c->h_mstate, sizeof(MacroState), cudaMemcpyHostToDevice, c->stream));
    const bool graph = !c->prof && c->stream != nullptr;
    if (graph && !c->macro_exec) TRY(capture_inner(c, fp_main, &c->macro_exec, &c->macro_nodes));
    if (graph && mixed && !c->macro_exec64) TRY(capture_inner(c, 0, &c->macro_exec64, &c->macro_nodes64));
    // one chunk of POLL inner iterations (the main phase's precision, or the FP64 tail),
    // then (unless it is the last) a look at the stop flag
    auto chunk = [&](bool tail_phase, bool poll) -> int {
        const int fp32 = tail_phase ? 0 : fp_main;
        if (graph) {
            CUDA_TRY(c, cudaGraphLaunch(tail_phase ? c->macro_exec64 : c->macro_exec, c->stream));
            c->launches += tail_phase ? c->macro_nodes64 : c->macro_nodes;
        } else {
            for (int k = 0; k < POLL; ++k) {
                const int wk = k & 1;
                TRY(launch(c, K_MGRAD, [&] {
                    return launch_macro_grad(c->stream, c->mg, c->order, fp32, c->model, c->mstate, c->W[wk], c->mq,
                                             c->mgrad, c->mphi);
                }));
                TRY(launch(c, K_MBFLUX, [&] {
                    return launch_macro_bflux(c->stream, c->mg, fp32, c->model, vquad_d(c), oquad_d(c), c->mstate,
                                              c->mq, c->mbf);
                }));
                TRY(launch(c, K_MRES, [&] {
                    return launch_macro_residual(c->stream, c->mg, c->order, fp32, c->model, sp.cfl_macro, c->mstate,
                                                 c->W[wk], c->mq, c->mgrad, c->mphi, c->hot, c->mbf, c->hot_b, c->Rg,
                                                 c->Dinv, c->gam, c->rpart);
                }));
                TRY(launch(c, K_MNORM, [&] {
                    return launch_macro_norm(c->stream, macro_rpart_count((int)c->nc), c->rpart, c->mstate,
                                             c->mhist);
                }));
                const int sweeps = std::max(sp.macro_sweeps, 1);
                for (int sw = 0; sw < sweeps; ++sw)
                    TRY(launch(c, K_MJACOBI, [&] {
                        return launch_macro_jacobi(c->stream, c->mg, fp32, c->model, c->mstate, sw == 0,
                                                   sw == sweeps - 1, c->W[wk], c->mq, c->Rg, c->Dinv, c->gam,
                                                   c->dG[sw & 1], c->dG[(sw + 1) & 1], c->W[1 - wk]);
                    }));
            }
        }
        if (poll) {
            CUDA_TRY(c, cudaMemcpyAsync(c->h_mstate, c->mstate, sizeof(MacroState), cudaMemcpyDeviceToHost,
                                        c->stream));
            CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        }
        return GSIS_OK;
    };
    const int main_iters = sp.max_inner - tail;
    for (int it = 0; it < main_iters; it += POLL) {
        TRY(chunk(false, it + POLL < main_iters || tail > 0));
        if ((it + POLL < main_iters || tail > 0) && c->h_mstate->done) break;
    }
    if (tail > 0) {
        // the FP64 residual side for up to `tail` more iterations, from where the FP32 ones stopped
        c->h_mstate->done = 0;
        c->h_mstate->max_inner = c->h_mstate->it + tail;
        CUDA_TRY(c, cudaMemcpyAsync(c->mstate, c->h_mstate, sizeof(MacroState), cudaMemcpyHostToDevice, c->stream));
        for (int it = 0; it < tail; it += POLL) {
            TRY(chunk(true, it + POLL < tail));
            if (it + POLL < tail && c->h_mstate->done) break;
        }
    }
    int w = 0;
    *w_out = w;   // POLL is even: every chunk ends where it started
    return GSIS_OK;
}

// Defect correction (an extension): the offset r_h - R(W_h) that the synthetic solve adds
// to its residual, so that it solves R(W) - R(W_h) + r_h = 0 with r_h the moments of the
// kinetic residual (Eq. dis_micro's right-hand side) at f^{k+1/2}, coefficients of M^{k+1/2}:
// the wall densities, slopes and residuals of f^{k+1/2} (into the buffers the next kinetic
// step overwrites anyway), their moment rows, and R(W_h) in FP64 without the offset.
template <typename Real>
int defect_offset(gsis_ctx *c, int nxt) {
    const Geom<Real> g = geom<Real>(c);
    TRY(launch(c, K_COEF, [&] {
        return launch_coefficients<Real>(c->stream, c->dim, g, c->model, c->fields_h, c->cell_dx, (Real *)c->coef_h);
    }));
    TRY(launch(c, K_WALL, [&] {
        return launch_wall_density<Real>(c->stream, c->dim, g, vquad<Real>(c), c->patch_T, c->bf_inc, c->patch_kind,
                                         (const Real *)c->f[nxt], nullptr, (Real *)c->bcoef);
    }));
    if (c->order == 2) {
        TRY(launch(c, K_SLOPE_GAS, [&] {
            return launch_slopes<Real>(c->stream, c->dim, 4, g, vquad<Real>(c), (const Real *)c->f[nxt],
                                       (Real *)c->fface);
        }));
        TRY(launch(c, K_SLOPE_PHOTON, [&] {
            return launch_slopes<Real>(c->stream, c->dim, 1, g, oquad<Real>(c), (const Real *)c->I[nxt],
                                       (Real *)c->oface);
        }));
    }
    Geom<Real> gr = g;
    gr.resid = 1;
    gr.tc = 0;
    TRY(launch(c, K_SWEEP_GAS, [&] {   // residual moments only: f_out is not written
        return launch_sweep_gas<Real>(c->stream, c->dim, c->order, gr, vquad<Real>(c), (const Real *)c->coef_h,
                                      (const Real *)c->bcoef, (const Real *)c->f[nxt], (const Real *)c->fface,
                                      (Real *)c->f[nxt], (Real *)c->partial);
    }));
    TRY(launch(c, K_SWEEP_PHOTON, [&] {
        return launch_sweep_photon<Real>(c->stream, c->dim, c->order, gr, oquad<Real>(c), (const Real *)c->coef_h,
                                         (const Real *)c->bcoef, (const Real *)c->I[nxt], (const Real *)c->oface,
                                         (Real *)c->I[nxt], (Real *)c->opartial);
    }));
    TRY(launch(c, K_MCONV, [&] {
        return launch_resid_rows<Real>(c->stream, c->dim, (int)c->nc, c->nch, c->och, (const Real *)c->coef_h,
                                       (const Real *)c->partial, (const Real *)c->opartial, c->rrow);
    }));
    MacroGeom g0 = c->mg;
    g0.moff = nullptr;
    TRY(launch(c, K_MGRAD, [&] {
        return launch_macro_grad(c->stream, g0, c->order, 0, c->model, nullptr, c->W[0], c->mq, c->mgrad, c->mphi);
    }));
    TRY(launch(c, K_MBFLUX, [&] {
        return launch_macro_bflux(c->stream, g0, 0, c->model, vquad_d(c), oquad_d(c), nullptr, c->mq, c->mbf);
    }));
    TRY(launch(c, K_MRES, [&] {
        return launch_macro_residual(c->stream, g0, c->order, 0, c->model, c->solver.cfl_macro, nullptr, c->W[0],
                                     c->mq, c->mgrad, c->mphi, c->hot, c->mbf, c->hot_b, c->Rg, c->Dinv, c->gam,
                                     c->rpart);
    }));
    TRY(launch(c, K_MCONV, [&] {
        return launch_macro_offset(c->stream, c->dim, (int)c->nc, c->Rg, c->rrow, c->moff);
    }));
    return GSIS_OK;
}

// One GSIS iteration (Section 3): kinetic step, high-order terms from f^{k+1/2}, the
// synthetic equations, f^{k+1} = f^{k+1/2} + w [f_eq(M^{k+1}) - f_eq(M^{k+1/2})].
template <typename Real>
int gsis_iteration(gsis_ctx *c) {
    const int nxt = 1 - c->cur;
    const MacroGeom &g = c->mg;
    CUDA_TRY(c, cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
    TRY(kinetic_step<Real>(c, nxt));
    TRY(launch(c, K_FINISH, [&] {       // M^{k+1/2}
        return launch_finish<Real>(c->stream, c->dim, (int)c->nc, c->nch, c->och, c->model, (const Real *)c->coef,
                                   (const Real *)c->partial, (const Real *)c->opartial, c->vol, nullptr,
                                   c->fields_h, c->eps_terms, c->err, 0);
    }));
    TRY(launch(c, K_KBFLUX, [&] {
        return launch_kinetic_bflux<Real>(c->stream, g, c->model, vquad<Real>(c), oquad<Real>(c),
                                          (const Real *)c->f[nxt], (const Real *)c->I[nxt], c->kbf);
    }));
    TRY(launch(c, K_MCONV, [&] {
        return launch_macro_from_fields(c->stream, c->dim, (int)c->nc, c->model, c->fields_h, c->W[0]);
    }));
    TRY(launch(c, K_MGRAD, [&] {
        return launch_macro_grad(c->stream, g, 1, c->mfp32 == 1, c->model, nullptr, c->W[0], c->mq, c->mgrad, c->mphi);
    }));
    TRY(launch(c, K_MBFLUX, [&] {
        return launch_macro_bflux(c->stream, g, c->mfp32 == 1, c->model, vquad_d(c), oquad_d(c), nullptr, c->mq, c->mbf);
    }));
    TRY(launch(c, K_HOT, [&] {
        return launch_macro_hot(c->stream, g, c->mfp32 == 1, c->model, c->fields_h, c->mq, c->mgrad, c->kbf, c->mbf, c->hot,
                                c->hot_b);
    }));
    if (c->moff) TRY(defect_offset<Real>(c, nxt));
    int w = 0;
    TRY(macro_solve(c, &w));
    if (c->closed) {
        TRY(launch(c, K_MCONV, [&] {
            return launch_macro_mass_rescale(c->stream, c->dim, (int)c->nc, c->vol, c->fields, c->W[w]);
        }));
    }
    TRY(launch(c, K_MCONV, [&] {
        return launch_macro_fields_from_W(c->stream, c->dim, (int)c->nc, c->model, c->W[w], c->fields_n);
    }));
    TRY(launch(c, K_SYNC, [&] {
        return launch_sync<Real>(c->stream, c->dim, (int)c->nc, c->tcm >= 1, vquad<Real>(c), oquad<Real>(c), c->model,
                                 c->solver.sync_relax, c->fields_n, c->fields_h, (const Real *)c->coef,
                                 (Real *)c->f[nxt], (Real *)c->I[nxt], (Real *)c->partial, (Real *)c->opartial,
                                 c->sync_kc, c->tc_wait, c->err);
    }));
    return close_iteration<Real>(c, nxt);
}

int read_eps(gsis_ctx *c, double *eps) {
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const double *s = c->h_pinned;
    int errw = 0;
    std::memcpy(&errw, c->h_pinned + NEPS, sizeof(int));
    if (errw & ERR_TIMEOUT_BIT)
        return fail(c, GSIS_ERR_TIMEOUT, "a tensor-core completion wait ran out of its poll budget");
    if (errw) return fail(c, GSIS_ERR_DIVERGED, "non-finite or non-positive density or temperature");
    // Section 6: max over rho, u, T of the volume-weighted relative change; the
    // velocity denominator is floored at 1% of the thermal-speed norm
    const double e_rho = std::sqrt(s[0]) / std::sqrt(s[1]);
    const double e_T = std::sqrt(s[4]) / std::sqrt(s[5]);
    const double den_u = std::fmax(std::sqrt(s[3]), 0.01 * std::sqrt(s[6]));
    const double e_u = std::sqrt(s[2]) / den_u;
    double e = std::fmax(e_rho, std::fmax(e_T, e_u));
    c->last_eps = e;
    if (c->eps_pending) {
        c->eps_hist.push_back(e);
        c->eps_pending = false;
    }
    if (eps) *eps = e;
    return GSIS_OK;
}

// Reads the device error word after the queued work (refresh passes report a tensor-core
// completion wait that ran out, or non-finite moments, here).
int check_err(gsis_ctx *c) {
    CUDA_TRY(c, cudaMemcpyAsync(c->h_pinned + NEPS, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    int errw = 0;
    std::memcpy(&errw, c->h_pinned + NEPS, sizeof(int));
    if (errw & ERR_TIMEOUT_BIT)
        return fail(c, GSIS_ERR_TIMEOUT, "a tensor-core completion wait ran out of its poll budget");
    return GSIS_OK;
}

int validate(const gsis_mesh *m, const gsis_velocity_quad *vq, const gsis_photon_quad *pq,
             const gsis_model_params *mp, const gsis_solver_params *sp, std::string &why) {
    if (!m || !vq || !pq || !mp || !sp) return why = "null argument", GSIS_ERR_INVALID_ARG;
    if (m->dim < 1 || m->dim > 3) return why = "dim must be 1, 2 or 3", GSIS_ERR_INVALID_ARG;
    if (m->dim == 3 && sp->precision == GSIS_FP32 && sp->tc_moments != 0)
        return why = "tensor-core moments are built for 1-D and 2-D: set tc_moments = 0 on a 3-D mesh",
               GSIS_ERR_UNSUPPORTED;
    if (m->n_cells <= 0 || m->n_faces <= 0 || m->n_cells > (1LL << 30)) return why = "bad mesh sizes", GSIS_ERR_INVALID_ARG;
    if (!m->face_owner || !m->face_nbr || !m->face_normal || !m->face_area || !m->face_centroid || !m->cell_volume ||
        !m->cell_centroid)
        return why = "null mesh array", GSIS_ERR_INVALID_ARG;
    if (m->n_patches < 0 || (m->n_patches > 0 && !m->patches)) return why = "bad patches", GSIS_ERR_INVALID_ARG;
    if (m->period)
        for (int a = 0; a < m->dim; ++a)
            if (!(m->period[a] >= 0.0) || !std::isfinite(m->period[a]))
                return why = "periods must be finite and non-negative", GSIS_ERR_INVALID_ARG;
    if (vq->n <= 0 || !vq->xi || !vq->w) return why = "bad velocity quadrature", GSIS_ERR_INVALID_ARG;
    if (pq->n <= 0 || !pq->omega || !pq->w) return why = "bad photon quadrature", GSIS_ERR_INVALID_ARG;
    if (sp->precision != GSIS_FP32 && sp->precision != GSIS_FP64) return why = "bad precision", GSIS_ERR_INVALID_ARG;
    if (sp->order != 1 && sp->order != 2) return why = "order must be 1 or 2", GSIS_ERR_INVALID_ARG;
    if (sp->relax_block < 1 || sp->relax_block > MAXB) return why = "relax_block must be in 1..64", GSIS_ERR_INVALID_ARG;
    {   // the gas sweep keeps a block's residuals and diagonals in shared memory
        const size_t rs = sp->precision == GSIS_FP64 ? 8 : 4;
        const bool tc = rs == 4 && sp->tc_moments >= 2 && MT % sp->relax_block == 0;
        if (sweep_smem_bytes(sp->relax_block, 4, m->dim, rs, tc) > 227 * 1024)
            return why = "relax_block too large for the shared memory of one CTA", GSIS_ERR_INVALID_ARG;
    }
    if (!(sp->cfl_meso > 0) || !(sp->venkat_K > 0)) return why = "bad CFL or limiter constant", GSIS_ERR_INVALID_ARG;
    if (!(sp->cfl_macro > 0) || sp->max_inner < 1 || sp->macro_sweeps < 1 || !(sp->tol_inner >= 0))
        return why = "bad synthetic-equation parameters", GSIS_ERR_INVALID_ARG;
    if (!(sp->sync_relax > 0) || !(sp->sync_relax <= 1)) return why = "sync_relax must be in (0, 1]", GSIS_ERR_INVALID_ARG;
    if (sp->tc_moments < 0 || sp->tc_moments > 2) return why = "tc_moments must be 0, 1 or 2", GSIS_ERR_INVALID_ARG;
    if (!(sp->positivity >= 0.0) || !(sp->positivity < 1.0)) return why = "positivity must be in [0, 1)", GSIS_ERR_INVALID_ARG;
    if (sp->defect_correction != 0 && sp->defect_correction != 1)
        return why = "defect_correction must be 0 or 1", GSIS_ERR_INVALID_ARG;
    if (sp->macro_fp32 < 0 || sp->macro_fp32 > 2) return why = "macro_fp32 must be 0, 1 or 2", GSIS_ERR_INVALID_ARG;
    if (!(mp->Kn > 0) || !(mp->Kn_p > 0) || !(mp->sigma_R >= 0) || !(mp->Z_r > 0) || !(mp->Z_v > 0) ||
        !(mp->d_r >= 0) || !(mp->d_v > 0) || !(mp->d_r > 0))
        return why = "bad model parameters", GSIS_ERR_INVALID_ARG;
    if (!(mp->sigma_R > 0)) return why = "sigma_R must be positive (photons always on)", GSIS_ERR_INVALID_ARG;
    if (mp->dv_temperature_dependent && !(mp->Tv_ref > 0))
        return why = "a temperature-dependent d_v needs Tv_ref > 0", GSIS_ERR_INVALID_ARG;
    for (int p = 0; p < m->n_patches; ++p) {
        const gsis_patch &P = m->patches[p];
        if (P.kind != GSIS_PATCH_WALL && P.kind != GSIS_PATCH_FARFIELD && P.kind != GSIS_PATCH_SYMMETRY)
            return why = "bad patch kind", GSIS_ERR_INVALID_ARG;
        if (P.kind == GSIS_PATCH_SYMMETRY) continue;     // a mirror plane has no state
        if (!(P.T_t > 0) || (P.kind == GSIS_PATCH_FARFIELD && (!(P.rho > 0) || !(P.T_r > 0) || !(P.T_v > 0) || !(P.T_R >= 0))))
            return why = "bad patch state", GSIS_ERR_INVALID_ARG;
    }
    return GSIS_OK;
}

void mason_monchick(const gsis_model_params *mp, double A[9]) {
    const double dr = mp->d_r, dv = mp->d_v, Zr = mp->Z_r, Zv = mp->Z_v, Sc = mp->Sc;
    for (int k = 0; k < 9; ++k) A[k] = 0.0;
    A[0] = 2.0 / 3.0 + 5.0 / 6.0 * (dr / ((3 + dr) * Zr) + dv / ((3 + dv) * Zv));
    A[1] = -5.0 / (2.0 * (3 + dr) * Zr);
    A[2] = -5.0 / (2.0 * (3 + dv) * Zv);
    A[3] = -dr / ((3 + dr) * Zr);
    A[4] = Sc + 3.0 / (2.0 * (3 + dr) * Zr);
    A[6] = -dv / ((3 + dv) * Zv);
    A[8] = Sc + 3.0 / (2.0 * (3 + dv) * Zv);
}

template <typename Real>
int init_uniform(gsis_ctx *c) {
    std::vector<double> M((size_t)c->nc * NF, 0.0);
    for (int64_t i = 0; i < c->nc; ++i) {
        M[i * NF + 0] = 1.0;
        for (int k = 4; k < 8; ++k) M[i * NF + k] = 1.0;
    }
    CUDA_TRY(c, cudaMemcpy(c->fields, M.data(), M.size() * sizeof(double), cudaMemcpyHostToDevice));
    TRY(launch(c, K_EQUIL, [&] {
        return launch_equilibrium<Real>(c->stream, c->dim, (int)c->nc, vquad<Real>(c), oquad<Real>(c), c->model,
                                        c->fields, (Real *)c->f[c->cur], (Real *)c->I[c->cur]);
    }));
    return GSIS_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char *gsis_strerror(int code) {
    switch (code) {
        case GSIS_OK: return "ok";
        case GSIS_ERR_INVALID_ARG: return "invalid argument";
        case GSIS_ERR_OUT_OF_MEMORY: return "out of memory";
        case GSIS_ERR_CUDA: return "CUDA error";
        case GSIS_ERR_DIVERGED: return "iteration diverged";
        case GSIS_ERR_NOT_CONVERGED: return "not converged";
        case GSIS_ERR_TIMEOUT: return "device wait timed out";
        case GSIS_ERR_BAD_MESH: return "bad mesh";
        case GSIS_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

const char *gsis_last_error(const gsis_ctx *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

void gsis_destroy(gsis_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto &p : ctx->pending) {
        cudaEventDestroy(p.e0);
        cudaEventDestroy(p.e1);
    }
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamDestroy(ctx->copy_stream);
    }
    if (ctx->side_stream) {
        cudaStreamSynchronize(ctx->side_stream);
        cudaStreamDestroy(ctx->side_stream);
    }
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
    if (ctx->stage_ready) cudaEventDestroy(ctx->stage_ready);
    if (ctx->stage_free) cudaEventDestroy(ctx->stage_free);
    if (ctx->macro_exec) cudaGraphExecDestroy(ctx->macro_exec);
    if (ctx->macro_exec64) cudaGraphExecDestroy(ctx->macro_exec64);
    for (void *p : ctx->mlp_alloc) cudaFree(p);
    for (void *p : ctx->allocations) cudaFree(p);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    if (ctx->h_mstate) cudaFreeHost(ctx->h_mstate);
    delete ctx;
}

int gsis_create(const gsis_mesh *m, const gsis_velocity_quad *vq, const gsis_photon_quad *pq,
                const gsis_model_params *mp, const gsis_solver_params *sp, void *cuda_stream, gsis_ctx **out) {
    if (!out) return GSIS_ERR_INVALID_ARG;
    *out = nullptr;
    std::string why;
    int rc = validate(m, vq, pq, mp, sp, why);
    if (rc != GSIS_OK) return rc;
    gsis_ctx *c = new (std::nothrow) gsis_ctx();
    if (!c) return GSIS_ERR_OUT_OF_MEMORY;
    auto bail = [&](int code) {
        gsis_destroy(c);
        return code;
    };
    const int dim = m->dim;
    c->dim = dim;
    c->precision = sp->precision;
    c->real_size = sp->precision == GSIS_FP64 ? 8 : 4;
    c->mfp32 = sp->precision == GSIS_FP32 ? sp->macro_fp32 : 0;
    c->tcm = sp->precision == GSIS_FP32 ? sp->tc_moments : 0;
    c->order = sp->order;
    c->block = sp->relax_block;
    c->solver = *sp;
    c->nc = m->n_cells;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->V = vq->n;
    c->Vp = (vq->n + VCH - 1) / VCH * VCH;
    c->NO = pq->n;
    c->Op = (pq->n + OCH - 1) / OCH * OCH;
    c->Vd = c->V;
    c->Vdp = c->Vp;
    c->NOd = c->NO;
    c->Odp = c->Op;
    c->nch = c->Vp / VCH;
    c->och = c->Op / OCH;

    ModelDev &md = c->model;
    md.d_r = mp->d_r;
    md.d_v = mp->d_v;
    md.Z_r = mp->Z_r;
    md.Z_v = mp->Z_v;
    md.omega = mp->omega;
    md.Sc = mp->Sc;
    md.Kn = mp->Kn;
    md.Kn_p = mp->Kn_p;
    md.sigma_R = mp->sigma_R;
    md.k_eff_density_scaled = mp->k_eff_density_scaled;
    md.cfl_meso = sp->cfl_meso;
    md.dv_T = mp->dv_temperature_dependent ? 1 : 0;
    md.Tv_ref = mp->Tv_ref;
    md.userA = mp->A ? 1 : 0;
    if (mp->A) std::memcpy(md.A, mp->A, 9 * sizeof(double));
    else mason_monchick(mp, md.A);
    {   // auxiliary heat-flux matrix of Section 2.1
        const double Zi = 1.0 / (1.0 / mp->Z_r + 1.0 / mp->Z_v);
        const double *A = md.A;
        const double Mx[9] = {(2.0 - 3.0 * A[0]) * Zi + 1.0, -3.0 * A[1] * Zi, -3.0 * A[2] * Zi,
                              -A[3] * Zi, 1.0 - A[4] * Zi, -A[5] * Zi,
                              -A[6] * Zi, -A[7] * Zi, 1.0 - A[8] * Zi};
        std::memcpy(md.Mix, Mx, sizeof(Mx));
    }

    // periodic axes: a centroid difference across a seam is the minimal image
    double per[3] = {0.0, 0.0, 0.0};
    if (m->period)
        for (int a = 0; a < dim; ++a) per[a] = m->period[a];
    auto wrap = [&](double d, int a) { return per[a] > 0.0 ? d - per[a] * std::nearbyint(d / per[a]) : d; };

    // ---- connectivity: per cell up to MAXF faces (outward normal, neighbour)
    const int64_t nc = m->n_cells, nfc = m->n_faces;
    std::vector<int> nf(nc, 0), nbr(nc * MAXF, 0), bf_cell, bf_patch;
    std::vector<double> nrm(nc * MAXF * 3, 0.0), sv(nc * MAXF, 0.0), dxf(nc * MAXF * 3, 0.0),
        dxn(nc * MAXF * 3, 0.0), bfn;
    std::vector<int64_t> face_of(nc * MAXF, -1);
    for (int64_t f = 0; f < nfc; ++f) {
        const int o = m->face_owner[f], nb = m->face_nbr[f];
        if (o < 0 || o >= nc) return bail(GSIS_ERR_BAD_MESH);
        if (nb >= nc || (nb < 0 && -1 - nb >= m->n_patches) || nb == o) return bail(GSIS_ERR_BAD_MESH);
        const double S = m->face_area[f];
        double nn = 0.0;
        for (int a = 0; a < dim; ++a) nn += m->face_normal[f * dim + a] * m->face_normal[f * dim + a];
        if (!(S > 0) || std::fabs(nn - 1.0) > 1e-6) return bail(GSIS_ERR_BAD_MESH);
        const int sides[2] = {o, nb};
        for (int s = 0; s < (nb >= 0 ? 2 : 1); ++s) {
            const int cell = sides[s];
            if (nf[cell] >= MAXF) return bail(GSIS_ERR_UNSUPPORTED);
            const int k = nf[cell]++;
            const double sg = s == 0 ? 1.0 : -1.0;
            const double V = m->cell_volume[cell];
            if (!(V > 0)) return bail(GSIS_ERR_BAD_MESH);
            for (int a = 0; a < dim; ++a) {
                nrm[(cell * MAXF + k) * 3 + a] = sg * m->face_normal[f * dim + a];
                dxf[(cell * MAXF + k) * 3 + a] = wrap(m->face_centroid[f * dim + a] - m->cell_centroid[cell * dim + a], a);
            }
            sv[cell * MAXF + k] = S / V;
            face_of[cell * MAXF + k] = f;
            if (nb >= 0) {
                const int other = sides[1 - s];
                nbr[cell * MAXF + k] = other;
                for (int a = 0; a < dim; ++a)
                    dxn[(cell * MAXF + k) * 3 + a] =
                        wrap(m->face_centroid[f * dim + a] - m->cell_centroid[other * dim + a], a);
            } else {
                const int b = (int)bf_cell.size();
                nbr[cell * MAXF + k] = -1 - b;
                bf_cell.push_back(o);
                bf_patch.push_back(-1 - nb);
                for (int a = 0; a < 3; ++a) bfn.push_back(a < dim ? m->face_normal[f * dim + a] : 0.0);
            }
        }
    }
    c->n_bf = (int)bf_cell.size();
    // least-squares weights C_ij = (sum_k d_k d_k^T)^-1 d_j over the stencil of face
    // neighbours and their face neighbours (interior face neighbours first); a zero
    // gradient where the normal matrix is singular (det <= 1e-10 (tr/dim)^dim)
    // (layouts per dimension: stencil length MS, LW weights per entry, FRS Reals per face)
    const int MS = lay_maxs(dim), LW = lay_lw(dim), FRS = lay_frs(dim);
    std::vector<double> lsq(nc * MS * LW, 0.0), eps2(nc), cdx(nc), vol(nc), fgeo(nc * MAXF * FRS, 0.0);
    std::vector<int> stn(nc * MS, 0), info(nc * 4, 0), fnb(nc * MAXF * 2, -1);
    for (int64_t i = 0; i < nc; ++i) {
        vol[i] = m->cell_volume[i];
        cdx[i] = std::pow(vol[i], 1.0 / dim);
        const double Kdx = sp->venkat_K * cdx[i];
        eps2[i] = Kdx * Kdx * Kdx;
        std::vector<int> first, rest;
        for (int k = 0; k < nf[i]; ++k) {
            const int j = nbr[i * MAXF + k];
            double *F = &fgeo[((size_t)i * MAXF + k) * FRS];
            const double *nk = &nrm[(i * MAXF + k) * 3], *fk = &dxf[(i * MAXF + k) * 3], *gk = &dxn[(i * MAXF + k) * 3];
            const double svn = j >= 0 ? m->face_area[face_of[i * MAXF + k]] / m->cell_volume[j] : 0.0;
            if (dim < 3) {
                F[fr::NX] = nk[0];
                F[fr::NY] = dim > 1 ? nk[1] : 0.0;
                F[fr::SV] = sv[i * MAXF + k];
                F[fr::DFX] = fk[0];
                F[fr::DFY] = dim > 1 ? fk[1] : 0.0;
                F[fr::SVN] = svn;
                F[fr::DNX] = j >= 0 ? gk[0] : 0.0;
                F[fr::DNY] = j >= 0 && dim > 1 ? gk[1] : 0.0;
            } else {   // n (3), S/V, S/V of the neighbour, face - cell (3), face - neighbour (3), pad
                for (int a = 0; a < 3; ++a) {
                    F[a] = nk[a];
                    F[5 + a] = fk[a];
                    F[8 + a] = j >= 0 ? gk[a] : 0.0;
                }
                F[3] = sv[i * MAXF + k];
                F[4] = svn;
            }
            fnb[(i * MAXF + k) * 2 + 0] = j;
            if (j < 0) continue;
            if (j / c->block == i / c->block) fnb[(i * MAXF + k) * 2 + 1] = (int)(j - (i / c->block) * c->block);
            if (std::find(first.begin(), first.end(), j) == first.end()) first.push_back(j);
        }
        for (int j : first)
            for (int k2 = 0; k2 < nf[j]; ++k2) {
                const int j2 = nbr[j * MAXF + k2];
                if (j2 >= 0 && j2 != i && std::find(first.begin(), first.end(), j2) == first.end()) rest.push_back(j2);
            }
        std::sort(rest.begin(), rest.end());
        rest.erase(std::unique(rest.begin(), rest.end()), rest.end());
        std::vector<int> st(first);
        st.insert(st.end(), rest.begin(), rest.end());
        if ((int)st.size() > MS) {
            fprintf(stderr, "gsis: least-squares stencil of %d cells, more than %d\n", (int)st.size(), MS);
            return bail(GSIS_ERR_UNSUPPORTED);
        }
        info[i * 4 + 0] = nf[i];
        info[i * 4 + 1] = (int)st.size();
        info[i * 4 + 2] = (int)first.size();
        for (size_t k = 0; k < st.size(); ++k) stn[i * MS + k] = st[k];
        if ((int)st.size() < dim) continue;
        double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int j : st) {
            double d[3] = {0, 0, 0};
            for (int a = 0; a < dim; ++a) d[a] = wrap(m->cell_centroid[j * dim + a] - m->cell_centroid[i * dim + a], a);
            for (int a = 0; a < dim; ++a)
                for (int b = 0; b < dim; ++b) G[a][b] += d[a] * d[b];
        }
        // inverse of the normal matrix; singular when det <= 1e-10 (trace / dim)^dim
        double Gi[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        if (dim == 1) {
            if (!(G[0][0] > 0.0)) continue;
            Gi[0][0] = 1.0 / G[0][0];
        } else if (dim == 2) {
            const double det = G[0][0] * G[1][1] - G[0][1] * G[1][0];
            const double sc = 0.5 * (G[0][0] + G[1][1]);
            if (!(det > 1e-10 * sc * sc)) continue;
            Gi[0][0] = G[1][1] / det;
            Gi[1][1] = G[0][0] / det;
            Gi[0][1] = -G[0][1] / det;
            Gi[1][0] = -G[1][0] / det;
        } else {
            // adjugate / determinant
            const double c00 = G[1][1] * G[2][2] - G[1][2] * G[2][1], c01 = G[1][2] * G[2][0] - G[1][0] * G[2][2],
                         c02 = G[1][0] * G[2][1] - G[1][1] * G[2][0];
            const double det = G[0][0] * c00 + G[0][1] * c01 + G[0][2] * c02;
            const double sc = (G[0][0] + G[1][1] + G[2][2]) / 3.0;
            if (!(det > 1e-10 * sc * sc * sc)) continue;
            Gi[0][0] = c00 / det;
            Gi[1][0] = c01 / det;
            Gi[2][0] = c02 / det;
            Gi[0][1] = (G[0][2] * G[2][1] - G[0][1] * G[2][2]) / det;
            Gi[1][1] = (G[0][0] * G[2][2] - G[0][2] * G[2][0]) / det;
            Gi[2][1] = (G[0][1] * G[2][0] - G[0][0] * G[2][1]) / det;
            Gi[0][2] = (G[0][1] * G[1][2] - G[0][2] * G[1][1]) / det;
            Gi[1][2] = (G[0][2] * G[1][0] - G[0][0] * G[1][2]) / det;
            Gi[2][2] = (G[0][0] * G[1][1] - G[0][1] * G[1][0]) / det;
        }
        for (size_t k = 0; k < st.size(); ++k) {
            const int j = st[k];
            double d[3] = {0, 0, 0};
            for (int a = 0; a < dim; ++a) d[a] = wrap(m->cell_centroid[j * dim + a] - m->cell_centroid[i * dim + a], a);
            for (int a = 0; a < dim; ++a) {
                double s = 0.0;
                for (int b = 0; b < dim; ++b) s += Gi[a][b] * d[b];
                lsq[(i * MS + k) * LW + a] = s;
            }
        }
    }

    // ---- quadratures, padded with zero-weight points at the origin
    std::vector<double> vx(3 * (size_t)c->Vp, 0.0), vw(c->Vp, 0.0), ox(3 * (size_t)c->Op, 0.0), ow(c->Op, 0.0);
    for (int v = 0; v < vq->n; ++v) {
        for (int a = 0; a < dim; ++a) vx[a * (size_t)c->Vp + v] = vq->xi[v * dim + a];
        vw[v] = vq->w[v];
    }
    for (int o = 0; o < pq->n; ++o) {
        for (int a = 0; a < 3; ++a) ox[a * (size_t)c->Op + o] = pq->omega[o * 3 + a];
        ow[o] = pq->w[o];
    }

    // ---- boundary records: constant parts (wall density is refreshed every step)
    const int MH = 3 - dim;
    std::vector<double> bco((size_t)std::max(c->n_bf, 1) * bc::NB, 0.0), pT(std::max(m->n_patches, 1)),
        pu(3 * std::max(m->n_patches, 1)), tmp;
    std::vector<int> pk(std::max(m->n_patches, 1), 0);
    for (int p = 0; p < m->n_patches; ++p) {
        pT[p] = m->patches[p].T_t;
        pk[p] = m->patches[p].kind;
        for (int a = 0; a < 3; ++a) pu[p * 3 + a] = m->patches[p].u[a];
    }
    for (int b = 0; b < c->n_bf; ++b) {
        const gsis_patch &P = m->patches[bf_patch[b]];
        double *B = &bco[(size_t)b * bc::NB];
        const bool wall = P.kind == GSIS_PATCH_WALL;
        const double T = P.T_t, Tr = wall ? P.T_t : P.T_r, Tv = wall ? P.T_t : P.T_v, TR = wall ? P.T_t : P.T_R;
        B[bc::A] = (wall ? 1.0 : P.rho) * std::pow(2.0 * M_PI * T, -0.5 * dim);
        B[bc::B] = 0.5 / T;
        for (int a = 0; a < 3; ++a) B[bc::U + a] = P.u[a];
        B[bc::M0] = 1.0;
        B[bc::MH] = MH * T;
        B[bc::M1] = 0.5 * mp->d_r * Tr;
        B[bc::M2] = vib_energy<double>(c->model, Tv);       // d_v(T) T / 2 of the entering gas
        B[bc::IIN] = mp->sigma_R * TR * TR * TR * TR / M_PI;
    }

    // ---- synthetic-equation geometry: interior faces (owner -> neighbour), the cell -> face
    // map in the cell's face order, boundary faces, FP64 quadratures and patch states
    std::vector<int> fi_i, fi_j, cface(nc * MAXF, 0), mpk(std::max(m->n_patches, 1), 0);
    std::vector<double> fi_n, fi_S, fi_dn, fi_dist, fi_t, fi_dx, mbn, mbS, mbdn,
        mps(8 * std::max(m->n_patches, 1), 0.0);
    {
        std::vector<int> id_of(nfc, -1);
        for (int64_t f = 0; f < nfc; ++f) {
            const int o = m->face_owner[f], nb = m->face_nbr[f];
            if (nb < 0) continue;
            id_of[f] = (int)fi_i.size();
            fi_i.push_back(o);
            fi_j.push_back(nb);
            double d[3] = {0, 0, 0}, dn = 0.0, dd = 0.0;
            for (int a = 0; a < dim; ++a) {
                d[a] = wrap(m->cell_centroid[nb * dim + a] - m->cell_centroid[o * dim + a], a);
                dn += m->face_normal[f * dim + a] * d[a];
                dd += d[a] * d[a];
            }
            dd = std::sqrt(dd);
            for (int a = 0; a < MGS; ++a) {
                fi_n.push_back(a < dim ? m->face_normal[f * dim + a] : 0.0);
                fi_t.push_back(d[a] / dd);
            }
            for (int s = 0; s < 2; ++s)
                for (int a = 0; a < MGS; ++a)
                    fi_dx.push_back(a < dim ? wrap(m->face_centroid[f * dim + a] -
                                                   m->cell_centroid[(s == 0 ? o : nb) * dim + a], a)
                                            : 0.0);
            fi_S.push_back(m->face_area[f]);
            fi_dn.push_back(std::fabs(dn));
            fi_dist.push_back(dd);
        }
        for (int64_t i = 0; i < nc; ++i) {
            for (int k = 0; k < MAXF; ++k) {
                if (k >= nf[i]) { cface[i * MAXF + k] = -1 - std::max(c->n_bf, 1); continue; }
                const int j = nbr[i * MAXF + k];
                cface[i * MAXF + k] = j >= 0 ? id_of[face_of[i * MAXF + k]] : j;
            }
        }
        // boundary faces in the order the kinetic connectivity numbered them
        mbn.assign(MGS * std::max(c->n_bf, 1), 0.0);
        mbS.assign(std::max(c->n_bf, 1), 0.0);
        mbdn.assign(std::max(c->n_bf, 1), 0.0);
        for (int64_t i = 0; i < nc; ++i)
            for (int k = 0; k < nf[i]; ++k) {
                const int j = nbr[i * MAXF + k];
                if (j >= 0) continue;
                const int b = -1 - j;
                const int64_t f = face_of[i * MAXF + k];
                double dn = 0.0;
                for (int a = 0; a < dim; ++a) {
                    mbn[b * MGS + a] = m->face_normal[f * dim + a];
                    dn += m->face_normal[f * dim + a] * wrap(m->face_centroid[f * dim + a] - m->cell_centroid[i * dim + a], a);
                }
                mbS[b] = m->face_area[f];
                mbdn[b] = std::fabs(dn);
            }
        for (int p = 0; p < m->n_patches; ++p) {
            const gsis_patch &P = m->patches[p];
            mpk[p] = P.kind;
            if (P.kind != GSIS_PATCH_WALL && P.kind != GSIS_PATCH_SYMMETRY) c->closed = false;
            const double st[8] = {P.rho, P.u[0], P.u[1], P.u[2], P.T_t, P.T_r, P.T_v, P.T_R};
            for (int k = 0; k < 8; ++k) mps[p * 8 + k] = st[k];
        }
        if (fi_i.empty()) {   // keep every device array non-empty
            fi_i.push_back(0); fi_j.push_back(0); fi_S.push_back(0.0); fi_dn.push_back(1.0); fi_dist.push_back(1.0);
            for (int a = 0; a < MGS; ++a) { fi_n.push_back(0.0); fi_t.push_back(0.0); fi_dx.push_back(0.0); fi_dx.push_back(0.0); }
        }
    }
    const int n_fi = (int)std::count_if(fi_S.begin(), fi_S.end(), [](double x) { return x > 0.0; });

    // ---- device allocations
    const size_t fsz = (size_t)nc * c->Vp * 4, isz = (size_t)nc * c->Op;
    rc = GSIS_OK;
#define A_(x) do { rc = (x); if (rc != GSIS_OK) { int _r = rc; if (!c->last_error.empty()) fprintf(stderr, "gsis: %s\n", c->last_error.c_str()); return bail(_r); } } while (0)
    A_(dalloc_real(c, &c->f[0], fsz));
    A_(dalloc_real(c, &c->f[1], fsz));
    A_(dalloc_real(c, &c->I[0], isz));
    A_(dalloc_real(c, &c->I[1], isz));
    A_(dalloc_real(c, &c->coef, (size_t)nc * cf::NC));
    A_(dalloc_real(c, &c->bcoef, bco.size()));
    A_(dalloc_real(c, &c->partial, (size_t)nc * c->nch * lay_nmp(dim)));
    A_(dalloc_real(c, &c->opartial, (size_t)nc * c->och * NMO));
    if (c->precision == GSIS_FP32) A_(dalloc_real(c, &c->sync_kc, (size_t)nc * SYNC_KC));
    if (c->order == 2) {
        A_(dalloc_real(c, &c->fface, fi_i.size() * c->Vp * 4));
        A_(dalloc_real(c, &c->oface, fi_i.size() * c->Op));
    }
    A_(dalloc(c, &c->fields, (size_t)nc * NF));
    A_(dalloc(c, &c->fields_old, (size_t)nc * NF));
    A_(dalloc(c, &c->eps_terms, (size_t)nc * NEPS));
    A_(dalloc(c, &c->eps_sums, NEPS));
    A_(dalloc(c, &c->err, 1));
    A_(dalloc(c, &c->vol, nc));
    A_(dalloc(c, &c->cell_dx, nc));
    A_(dalloc(c, &c->g_info, nc));
    A_(dalloc(c, &c->g_fnb, nc * MAXF));
    A_(dalloc(c, &c->bf_cell, std::max(c->n_bf, 1)));
    A_(dalloc(c, &c->bf_patch, std::max(c->n_bf, 1)));
    A_(dalloc_real(c, &c->g_fgeo, fgeo.size()));
    A_(dalloc_real(c, &c->g_lsq, lsq.size()));
    A_(dalloc(c, &c->g_stn, stn.size()));
    A_(dalloc_real(c, &c->g_eps2, nc));
    A_(dalloc_real(c, &c->bf_nrm, 3 * std::max(c->n_bf, 1)));
    A_(dalloc_real(c, &c->vq_x, vx.size()));
    A_(dalloc_real(c, &c->vq_w, vw.size()));
    A_(dalloc_real(c, &c->oq_x, ox.size()));
    A_(dalloc_real(c, &c->oq_w, ow.size()));
    A_(dalloc(c, &c->patch_T, pT.size()));
    A_(dalloc(c, &c->patch_u, pu.size()));
    A_(dalloc(c, &c->bf_inc, (size_t)std::max(c->n_bf, 1)));
    A_(dalloc(c, &c->eps_part, (size_t)std::max<int64_t>(64, (nc + 31) / 32) * NEPS));
    A_(dalloc(c, &c->eps_ticket, 1));
    A_(dalloc(c, &c->patch_kind, pk.size()));
    if (cudaMallocHost(&c->h_pinned, (NEPS + 1) * sizeof(double)) != cudaSuccess) return bail(GSIS_ERR_OUT_OF_MEMORY);
    if (cudaMallocHost(&c->h_mstate, sizeof(MacroState)) != cudaSuccess) return bail(GSIS_ERR_OUT_OF_MEMORY);
    {
        const size_t nbf1 = std::max(c->n_bf, 1), nfi1 = fi_i.size();
        A_(dalloc(c, &c->m_fi_i, nfi1));
        A_(dalloc(c, &c->m_fi_j, nfi1));
        A_(dalloc(c, &c->m_cface, (size_t)nc * MAXF));
        A_(dalloc(c, &c->m_pkind, mpk.size()));
        A_(dalloc(c, &c->m_fi_n, nfi1 * MGS));
        A_(dalloc(c, &c->m_fi_S, nfi1));
        A_(dalloc(c, &c->m_fi_dn, nfi1));
        A_(dalloc(c, &c->m_fi_dist, nfi1));
        A_(dalloc(c, &c->m_fi_t, nfi1 * MGS));
        A_(dalloc(c, &c->m_fi_dx, nfi1 * 2 * MGS));
        A_(dalloc(c, &c->m_lsq, lsq.size()));
        A_(dalloc(c, &c->m_eps2, (size_t)nc));
        A_(dalloc(c, &c->m_bf_n, nbf1 * MGS));
        A_(dalloc(c, &c->m_bf_S, nbf1));
        A_(dalloc(c, &c->m_bf_dn, nbf1));
        A_(dalloc(c, &c->m_pstate, mps.size()));
        A_(dalloc(c, &c->vqd_x, vx.size()));
        A_(dalloc(c, &c->vqd_w, vw.size()));
        A_(dalloc(c, &c->oqd_x, ox.size()));
        A_(dalloc(c, &c->oqd_w, ow.size()));
        for (int k = 0; k < 2; ++k) {
            A_(dalloc(c, &c->W[k], (size_t)nc * NVM));
            A_(dalloc(c, &c->dG[k], (size_t)nc * NVM));
        }
        A_(dalloc(c, &c->mq, (size_t)nc * NVM));
        A_(dalloc(c, &c->mgrad, (size_t)nc * MGS * NVM));
        A_(dalloc(c, &c->mphi, (size_t)nc * NVM));
        A_(dalloc(c, &c->Rg, (size_t)nc * NVM));
        if (sp->defect_correction) {
            A_(dalloc_real(c, &c->coef_h, (size_t)nc * cf::NC));
            A_(dalloc(c, &c->rrow, (size_t)nc * NVM));
            A_(dalloc(c, &c->moff, (size_t)nc * NVM));
            if (cudaMemset(c->moff, 0, (size_t)nc * NVM * sizeof(double)) != cudaSuccess) return bail(GSIS_ERR_CUDA);
        }
        A_(dalloc(c, &c->Dinv, (size_t)nc * 24));
        A_(dalloc(c, &c->gam, (size_t)nc * MAXF * 2));
        A_(dalloc(c, &c->rpart, (size_t)macro_rpart_count((int)nc)));
        A_(dalloc(c, &c->hot, nfi1 * NHOT));
        A_(dalloc(c, &c->hot_b, nbf1 * NVM));
        A_(dalloc(c, &c->kbf, nbf1 * NVM));
        A_(dalloc(c, &c->mbf, nbf1 * NVM));
        A_(dalloc(c, &c->fields_h, (size_t)nc * NF));
        A_(dalloc(c, &c->fields_n, (size_t)nc * NF));
        A_(dalloc(c, &c->mhist, (size_t)std::max(sp->max_inner, 1)));
        A_(dalloc(c, &c->mstate, 1));
        A_(upload(c, c->m_fi_i, fi_i));
        A_(upload(c, c->m_fi_j, fi_j));
        A_(upload(c, c->m_cface, cface));
        A_(upload(c, c->m_pkind, mpk));
        A_(upload(c, c->m_fi_n, fi_n));
        A_(upload(c, c->m_fi_S, fi_S));
        A_(upload(c, c->m_fi_dn, fi_dn));
        A_(upload(c, c->m_fi_dist, fi_dist));
        A_(upload(c, c->m_fi_t, fi_t));
        A_(upload(c, c->m_fi_dx, fi_dx));
        A_(upload(c, c->m_lsq, lsq));
        A_(upload(c, c->m_eps2, eps2));
        A_(upload(c, c->m_bf_n, mbn));
        A_(upload(c, c->m_bf_S, mbS));
        A_(upload(c, c->m_bf_dn, mbdn));
        A_(upload(c, c->m_pstate, mps));
        A_(upload(c, c->vqd_x, vx));
        A_(upload(c, c->vqd_w, vw));
        A_(upload(c, c->oqd_x, ox));
        A_(upload(c, c->oqd_w, ow));
        MacroGeom &G = c->mg;
        G.n_cells = (int)nc;
        G.dim = dim;
        G.n_fi = n_fi;
        G.n_bf = c->n_bf;
        G.fi_i = c->m_fi_i;
        G.fi_j = c->m_fi_j;
        G.fi_n = c->m_fi_n;
        G.fi_S = c->m_fi_S;
        G.fi_dn = c->m_fi_dn;
        G.fi_dist = c->m_fi_dist;
        G.fi_t = c->m_fi_t;
        G.fi_dx = c->m_fi_dx;
        G.cface = c->m_cface;
        G.info = c->g_info;
        G.stn = c->g_stn;
        G.lsq = c->m_lsq;
        G.eps2 = c->m_eps2;
        G.vol = c->vol;
        G.dx = c->cell_dx;
        G.moff = c->moff;              // null unless the defect correction is on
        G.bf_cell = c->bf_cell;
        G.bf_patch = c->bf_patch;
        G.bf_n = c->m_bf_n;
        G.bf_S = c->m_bf_S;
        G.bf_dn = c->m_bf_dn;
        G.patch_kind = c->m_pkind;
        G.patch_state = c->m_pstate;
    }

    if (bfn.empty()) bfn.assign(3, 0.0);
    if (bf_cell.empty()) { bf_cell.push_back(0); bf_patch.push_back(0); }
    A_(upload(c, c->vol, vol));
    A_(upload(c, c->cell_dx, cdx));
    CUDA_TRY(c, cudaMemcpy(c->g_info, info.data(), info.size() * sizeof(int), cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(c->g_fnb, fnb.data(), fnb.size() * sizeof(int), cudaMemcpyHostToDevice));
    A_(upload(c, c->g_stn, stn));
    A_(upload(c, c->bf_cell, bf_cell));
    A_(upload(c, c->bf_patch, bf_patch));
    A_(upload_real(c, c->g_fgeo, fgeo));
    A_(upload_real(c, c->g_lsq, lsq));
    A_(upload_real(c, c->g_eps2, eps2));
    A_(upload_real(c, c->bf_nrm, bfn));
    A_(upload_real(c, c->vq_x, vx));
    A_(upload_real(c, c->vq_w, vw));
    A_(upload_real(c, c->oq_x, ox));
    A_(upload_real(c, c->oq_w, ow));
    A_(upload_real(c, c->bcoef, bco));
    A_(upload(c, c->patch_T, pT));
    A_(upload(c, c->patch_u, pu));
    {   // mirror planes: for each distinct face normal of a SYMMETRY patch, the index of the
        // mirror image x - 2 (x.n) n of every velocity and photon direction (the sets must be
        // symmetric under it; images matched to 1e-9 of the set's scale)
        std::vector<int> tab((size_t)std::max(c->n_bf, 1), -1), rv, ro;
        std::vector<std::array<double, 3>> normals;
        auto mirror = [&](int n_pts, int pad, int d, const double *pts, const double *nn, std::vector<int> &out) {
            double scale = 1.0;
            for (int v = 0; v < n_pts * d; ++v) scale = std::max(scale, std::fabs(pts[v]));
            const size_t base = out.size();
            out.resize(base + (size_t)pad);
            for (int v = 0; v < pad; ++v) out[base + v] = v;     // padding maps to itself
            for (int v = 0; v < n_pts; ++v) {
                double img[3] = {0, 0, 0}, dot = 0.0;
                for (int a = 0; a < d; ++a) dot += pts[(size_t)v * d + a] * (a < dim ? nn[a] : 0.0);
                for (int a = 0; a < d; ++a) img[a] = pts[(size_t)v * d + a] - 2.0 * dot * (a < dim ? nn[a] : 0.0);
                int best = -1;
                double bd = 1e300;
                for (int w = 0; w < n_pts; ++w) {
                    double e = 0.0;
                    for (int a = 0; a < d; ++a) e = std::max(e, std::fabs(pts[(size_t)w * d + a] - img[a]));
                    if (e < bd) bd = e, best = w;
                }
                if (bd > 1e-9 * scale) return false;
                out[base + v] = best;
            }
            return true;
        };
        for (int b = 0; b < c->n_bf; ++b) {
            if (m->patches[bf_patch[b]].kind != GSIS_PATCH_SYMMETRY) continue;
            const std::array<double, 3> nb = {bfn[b * 3], bfn[b * 3 + 1], bfn[b * 3 + 2]};
            int t = -1;
            for (size_t k = 0; k < normals.size(); ++k)
                if (std::fabs(normals[k][0] - nb[0]) + std::fabs(normals[k][1] - nb[1]) + std::fabs(normals[k][2] - nb[2]) < 1e-12)
                    t = (int)k;
            if (t < 0) {
                t = (int)normals.size();
                normals.push_back(nb);
                if (!mirror(vq->n, c->Vp, dim, vq->xi, nb.data(), rv) || !mirror(pq->n, c->Op, 3, pq->omega, nb.data(), ro)) {
                    fprintf(stderr, "gsis: a mirror plane needs velocity and photon sets symmetric under its reflection\n");
                    return bail(GSIS_ERR_INVALID_ARG);
                }
            }
            tab[b] = t;
        }
        if (rv.empty()) rv.assign(1, 0), ro.assign(1, 0);
        A_(dalloc(c, &c->bf_tab, tab.size()));
        A_(dalloc(c, &c->refl_v, rv.size()));
        A_(dalloc(c, &c->refl_o, ro.size()));
        A_(upload(c, c->bf_tab, tab));
        A_(upload(c, c->refl_v, rv));
        A_(upload(c, c->refl_o, ro));
        c->mirrors = !normals.empty();
        c->mg.bf_tab = c->bf_tab;       // the synthetic equations' geometry was filled above
        c->mg.refl_v = c->refl_v;
        c->mg.refl_o = c->refl_o;
    }
    c->h_wall.assign((size_t)std::max(c->n_bf, 1) * 8, 0.0);
    for (int b = 0; b < c->n_bf; ++b) {     // per boundary face: wall flag, normal, wall T and u
        const gsis_patch &P = m->patches[bf_patch[b]];
        double *hw = c->h_wall.data() + (size_t)b * 8;
        hw[0] = P.kind == GSIS_PATCH_WALL ? 1.0 : 0.0;
        for (int a = 0; a < 3; ++a) {
            hw[1 + a] = bfn[b * 3 + a];
            hw[5 + a] = P.u[a];
        }
        hw[4] = P.T_t;
    }
    {   // incoming mass flux of the unit-density wall Maxwellian at every wall face
        std::vector<double> inc(std::max(c->n_bf, 1), 0.0);
        for (int b = 0; b < c->n_bf; ++b) {
            const gsis_patch &P = m->patches[bf_patch[b]];
            if (P.kind != GSIS_PATCH_WALL) continue;
            const double norm = std::pow(2.0 * M_PI * P.T_t, -0.5 * dim);
            double acc = 0.0;
            for (int v = 0; v < vq->n; ++v) {
                double xn = 0.0, c2 = 0.0;
                for (int a = 0; a < dim; ++a) {
                    const double x = vq->xi[v * dim + a];
                    xn += x * bfn[b * 3 + a];
                    c2 += (x - P.u[a]) * (x - P.u[a]);
                }
                if (xn < 0.0) acc += vq->w[v] * xn * norm * std::exp(-c2 / (2.0 * P.T_t));
            }
            inc[b] = acc;
        }
        A_(upload(c, c->bf_inc, inc));
    }
    if (cudaMemset(c->eps_ticket, 0, sizeof(unsigned int)) != cudaSuccess) return bail(GSIS_ERR_CUDA);
    A_(upload(c, c->patch_kind, pk));
    if (cudaMemset(c->err, 0, sizeof(int)) != cudaSuccess) return bail(GSIS_ERR_CUDA);
    if (cudaMemset(c->coef, 0, (size_t)nc * cf::NC * c->real_size) != cudaSuccess) return bail(GSIS_ERR_CUDA);
    A_(c->precision == GSIS_FP64 ? init_uniform<double>(c) : init_uniform<float>(c));
    A_(refresh(c));
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bail(GSIS_ERR_CUDA);
#undef A_
    *out = c;
    return GSIS_OK;
}

int gsis_init_fields(gsis_ctx *c, const double *M, int64_t len) {
    if (!c || !M || len < c->nc * NF) return fail(c, GSIS_ERR_INVALID_ARG, "fields buffer too short");
    CUDA_TRY(c, cudaMemcpyAsync(c->fields, M, (size_t)c->nc * NF * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    int rc = c->precision == GSIS_FP64
                 ? launch(c, K_EQUIL, [&] {
                       return launch_equilibrium<double>(c->stream, c->dim, (int)c->nc, vquad<double>(c),
                                                         oquad<double>(c), c->model, c->fields, (double *)c->f[c->cur],
                                                         (double *)c->I[c->cur]);
                   })
                 : launch(c, K_EQUIL, [&] {
                       return launch_equilibrium<float>(c->stream, c->dim, (int)c->nc, vquad<float>(c),
                                                        oquad<float>(c), c->model, c->fields, (float *)c->f[c->cur],
                                                        (float *)c->I[c->cur]);
                   });
    TRY(rc);
    TRY(refresh(c));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return GSIS_OK;
}

int gsis_upload_distributions(gsis_ctx *c, const void *f, const void *I) {
    if (!c || !f || !I) return fail(c, GSIS_ERR_INVALID_ARG, "null buffer");
    const size_t rs = c->real_size;
    CUDA_TRY(c, cudaMemcpy2DAsync(c->f[c->cur], (size_t)c->Vp * 4 * rs, f, (size_t)c->V * 4 * rs, (size_t)c->V * 4 * rs,
                                  (size_t)c->nc, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpy2DAsync(c->I[c->cur], (size_t)c->Op * rs, I, (size_t)c->NO * rs, (size_t)c->NO * rs,
                                  (size_t)c->nc, cudaMemcpyHostToDevice, c->stream));
    TRY(refresh(c));
    return GSIS_OK;
}

int gsis_stage_distributions(gsis_ctx *c, const void *f, const void *I) {
    if (!c || !f || !I) return fail(c, GSIS_ERR_INVALID_ARG, "null buffer");
    const size_t rs = c->real_size;
    if (!c->f_stage) {
        TRY(dalloc_real(c, &c->f_stage, (size_t)c->nc * c->Vp * 4));
        TRY(dalloc_real(c, &c->I_stage, (size_t)c->nc * c->Op));
        CUDA_TRY(c, cudaMemsetAsync(c->f_stage, 0, (size_t)c->nc * c->Vp * 4 * rs, c->stream));
        CUDA_TRY(c, cudaMemsetAsync(c->I_stage, 0, (size_t)c->nc * c->Op * rs, c->stream));
        CUDA_TRY(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        CUDA_TRY(c, cudaEventCreateWithFlags(&c->stage_ready, cudaEventDisableTiming));
        CUDA_TRY(c, cudaEventCreateWithFlags(&c->stage_free, cudaEventDisableTiming));
        CUDA_TRY(c, cudaEventRecord(c->stage_free, c->stream));
    }
    if (c->staged) return fail(c, GSIS_ERR_INVALID_ARG, "a staged upload is pending: commit it first");
    CUDA_TRY(c, cudaStreamWaitEvent(c->copy_stream, c->stage_free, 0));
    CUDA_TRY(c, cudaMemcpy2DAsync(c->f_stage, (size_t)c->Vp * 4 * rs, f, (size_t)c->V * 4 * rs, (size_t)c->V * 4 * rs,
                                  (size_t)c->nc, cudaMemcpyHostToDevice, c->copy_stream));
    CUDA_TRY(c, cudaMemcpy2DAsync(c->I_stage, (size_t)c->Op * rs, I, (size_t)c->NO * rs, (size_t)c->NO * rs,
                                  (size_t)c->nc, cudaMemcpyHostToDevice, c->copy_stream));
    CUDA_TRY(c, cudaEventRecord(c->stage_ready, c->copy_stream));
    c->staged = true;
    return GSIS_OK;
}

int gsis_commit_staged(gsis_ctx *c) {
    if (!c) return GSIS_ERR_INVALID_ARG;
    if (!c->staged) return fail(c, GSIS_ERR_INVALID_ARG, "nothing staged");
    CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->stage_ready, 0));
    std::swap(c->f[c->cur], c->f_stage);
    std::swap(c->I[c->cur], c->I_stage);
    CUDA_TRY(c, cudaEventRecord(c->stage_free, c->stream));
    c->staged = false;
    return refresh(c);
}

int gsis_refresh_fields(gsis_ctx *c) {
    if (!c) return GSIS_ERR_INVALID_ARG;
    TRY(refresh(c));
    return check_err(c);
}

int gsis_set_wait_limit(gsis_ctx *c, int32_t polls) {
    if (!c || polls < 0) return fail(c, GSIS_ERR_INVALID_ARG, "negative poll budget");
    c->tc_wait = polls;
    return GSIS_OK;
}

// ---- checkpoint / resume: a little-endian host image of the iteration state
namespace {
struct StateHeader {
    char magic[8];
    int32_t version, dim, precision, V, NO, pad;
    int64_t nc, iter, n_hist;
    double last_eps;
};
constexpr char kStateMagic[8] = {'G', 'S', 'I', 'S', 'S', 'T', 'A', 'T'};
constexpr int32_t kStateVersion = 1;

int64_t state_bytes(const gsis_ctx *c) {
    return (int64_t)sizeof(StateHeader) + (int64_t)c->eps_hist.size() * 8 + c->nc * NF * 8 +
           (c->nc * c->V * 4 + c->nc * c->NO) * (int64_t)c->real_size;
}
}  // namespace

int gsis_state_size(const gsis_ctx *c, int64_t *bytes) {
    if (!c || !bytes) return GSIS_ERR_INVALID_ARG;
    *bytes = state_bytes(c);
    return GSIS_OK;
}

int gsis_export_state(gsis_ctx *c, void *buf, int64_t len) {
    if (!c || !buf) return fail(c, GSIS_ERR_INVALID_ARG, "null buffer");
    if (len < state_bytes(c)) return fail(c, GSIS_ERR_INVALID_ARG, "state buffer too short");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    unsigned char *p = static_cast<unsigned char *>(buf);
    StateHeader h{};
    std::memcpy(h.magic, kStateMagic, 8);
    h.version = kStateVersion;
    h.dim = c->dim;
    h.precision = c->precision;
    h.V = c->V;
    h.NO = c->NO;
    h.nc = c->nc;
    h.iter = c->iter;
    h.n_hist = (int64_t)c->eps_hist.size();
    h.last_eps = c->last_eps;
    std::memcpy(p, &h, sizeof h);
    p += sizeof h;
    if (h.n_hist) std::memcpy(p, c->eps_hist.data(), (size_t)h.n_hist * 8);
    p += (size_t)h.n_hist * 8;
    CUDA_TRY(c, cudaMemcpy(p, c->fields, (size_t)c->nc * NF * 8, cudaMemcpyDeviceToHost));
    p += (size_t)c->nc * NF * 8;
    const size_t rs = c->real_size;
    CUDA_TRY(c, cudaMemcpy2D(p, (size_t)c->V * 4 * rs, c->f[c->cur], (size_t)c->Vp * 4 * rs, (size_t)c->V * 4 * rs,
                             (size_t)c->nc, cudaMemcpyDeviceToHost));
    p += (size_t)c->nc * c->V * 4 * rs;
    CUDA_TRY(c, cudaMemcpy2D(p, (size_t)c->NO * rs, c->I[c->cur], (size_t)c->Op * rs, (size_t)c->NO * rs,
                             (size_t)c->nc, cudaMemcpyDeviceToHost));
    return GSIS_OK;
}

int gsis_import_state(gsis_ctx *c, const void *buf, int64_t len) {
    if (!c || !buf) return fail(c, GSIS_ERR_INVALID_ARG, "null buffer");
    if (len < (int64_t)sizeof(StateHeader)) return fail(c, GSIS_ERR_INVALID_ARG, "state buffer too short");
    const unsigned char *p = static_cast<const unsigned char *>(buf);
    StateHeader h;
    std::memcpy(&h, p, sizeof h);
    if (std::memcmp(h.magic, kStateMagic, 8) != 0 || h.version != kStateVersion)
        return fail(c, GSIS_ERR_INVALID_ARG, "not a state image of this library version");
    if (h.dim != c->dim || h.precision != c->precision || h.V != c->V || h.NO != c->NO || h.nc != c->nc)
        return fail(c, GSIS_ERR_INVALID_ARG, "state image of a different problem (dim, precision or sizes)");
    if (h.n_hist < 0 || h.iter < 0) return fail(c, GSIS_ERR_INVALID_ARG, "corrupt state header");
    const int64_t need = (int64_t)sizeof(StateHeader) + h.n_hist * 8 + c->nc * NF * 8 +
                         (c->nc * c->V * 4 + c->nc * c->NO) * (int64_t)c->real_size;
    if (len < need) return fail(c, GSIS_ERR_INVALID_ARG, "state buffer too short");
    p += sizeof h;
    std::vector<double> hist((size_t)h.n_hist);
    if (h.n_hist) std::memcpy(hist.data(), p, (size_t)h.n_hist * 8);
    p += (size_t)h.n_hist * 8;
    const size_t rs = c->real_size;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    CUDA_TRY(c, cudaMemcpy(c->fields, p, (size_t)c->nc * NF * 8, cudaMemcpyHostToDevice));
    p += (size_t)c->nc * NF * 8;
    CUDA_TRY(c, cudaMemset(c->f[c->cur], 0, (size_t)c->nc * c->Vp * 4 * rs));
    CUDA_TRY(c, cudaMemset(c->I[c->cur], 0, (size_t)c->nc * c->Op * rs));
    CUDA_TRY(c, cudaMemcpy2D(c->f[c->cur], (size_t)c->Vp * 4 * rs, p, (size_t)c->V * 4 * rs, (size_t)c->V * 4 * rs,
                             (size_t)c->nc, cudaMemcpyHostToDevice));
    p += (size_t)c->nc * c->V * 4 * rs;
    CUDA_TRY(c, cudaMemcpy2D(c->I[c->cur], (size_t)c->Op * rs, p, (size_t)c->NO * rs, (size_t)c->NO * rs,
                             (size_t)c->nc, cudaMemcpyHostToDevice));
    // the next iteration reads the coefficient record built from the fields, exactly as
    // after the iteration that produced them
    int rc = c->precision == GSIS_FP64 ? launch(c, K_COEF, [&] {
        return launch_coefficients<double>(c->stream, c->dim, geom<double>(c), c->model, c->fields, c->cell_dx,
                                           (double *)c->coef);
    })
                                       : launch(c, K_COEF, [&] {
        return launch_coefficients<float>(c->stream, c->dim, geom<float>(c), c->model, c->fields, c->cell_dx,
                                          (float *)c->coef);
    });
    TRY(rc);
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->iter = h.iter;
    c->eps_hist = std::move(hist);
    c->last_eps = h.last_eps;
    c->have_eps = false;
    c->eps_pending = false;
    return GSIS_OK;
}

int gsis_get_history(const gsis_ctx *c, int64_t *iter, double *eps, int64_t len, int64_t *n_out) {
    if (!c) return GSIS_ERR_INVALID_ARG;
    if (iter) *iter = c->iter;
    const int64_t n = (int64_t)c->eps_hist.size();
    if (n_out) *n_out = n;
    if (eps)
        for (int64_t k = 0; k < std::min(n, len); ++k) eps[k] = c->eps_hist[(size_t)k];
    return GSIS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- velocity sharding
namespace {

double *xbuf_wall(gsis_ctx *c) { return c->xbuf + (size_t)c->nc * NXC; }
double *xbuf_kbf(gsis_ctx *c) { return xbuf_wall(c) + std::max(c->n_bf, 1); }

// this shard's moment sums of the partials into xbuf, and of f's wall outflow (gas) or
// its kinetic boundary-flux sums (kbf) into their sections, the other section zeroed
template <typename Real>
int shard_pack(gsis_ctx *c, int fidx, bool kbf) {
    const Geom<Real> g = geom<Real>(c);
    TRY(launch(c, K_FINISH, [&] {
        return launch_cell_sums<Real>(c->stream, c->dim, (int)c->nc, c->nch, c->och, (const Real *)c->partial,
                                      (const Real *)c->opartial, c->xbuf);
    }));
    const size_t nbf1 = std::max(c->n_bf, 1);
    CUDA_TRY(c, cudaMemsetAsync(xbuf_wall(c), 0, nbf1 * sizeof(double), c->stream));
    CUDA_TRY(c, cudaMemsetAsync(xbuf_kbf(c), 0, nbf1 * KBR * sizeof(double), c->stream));
    if (kbf) {
        TRY(launch(c, K_KBFLUX, [&] {
            return launch_kinetic_bflux<Real>(c->stream, c->mg, c->model, vquad<Real>(c), oquad<Real>(c),
                                              (const Real *)c->f[fidx], (const Real *)c->I[fidx], c->kbf,
                                              xbuf_kbf(c));
        }));
    } else {
        TRY(launch(c, K_WALL, [&] {
            return launch_wall_outflux<Real>(c->stream, c->dim, g, vquad<Real>(c), c->patch_kind,
                                             (const Real *)c->f[fidx], xbuf_wall(c));
        }));
    }
    return GSIS_OK;
}

template <typename Real>
int shard_begin(gsis_ctx *c, int mode) {
    const int nxt = 1 - c->cur;
    CUDA_TRY(c, cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
    TRY(kinetic_step<Real>(c, nxt));
    TRY(shard_pack<Real>(c, nxt, mode == GSIS_MODE_GSIS));
    c->shard_nxt = nxt;
    c->shard_state = mode == GSIS_MODE_GSIS ? 2 : 1;
    return GSIS_OK;
}

// GSIS after the first exchange: M^{k+1/2} and the kinetic boundary fluxes from the
// summed shards, the replicated synthetic solve, the synchronisation of this shard's
// velocities, then the shard's sums of f^{k+1} for the second exchange
template <typename Real>
int shard_mid(gsis_ctx *c) {
    const int nxt = c->shard_nxt;
    const MacroGeom &g = c->mg;
    TRY(launch(c, K_FINISH, [&] {
        return launch_finish<Real>(c->stream, c->dim, (int)c->nc, c->nch, c->och, c->model, (const Real *)c->coef,
                                   (const Real *)c->partial, (const Real *)c->opartial, c->vol, nullptr,
                                   c->fields_h, c->eps_terms, c->err, 0, nullptr, nullptr, nullptr, c->xbuf);
    }));
    TRY(launch(c, K_KBFLUX, [&] { return launch_kbflux_combine(c->stream, g, xbuf_kbf(c), c->kbf); }));
    TRY(launch(c, K_MCONV, [&] {
        return launch_macro_from_fields(c->stream, c->dim, (int)c->nc, c->model, c->fields_h, c->W[0]);
    }));
    TRY(launch(c, K_MGRAD, [&] {
        return launch_macro_grad(c->stream, g, 1, c->mfp32 == 1, c->model, nullptr, c->W[0], c->mq, c->mgrad, c->mphi);
    }));
    TRY(launch(c, K_MBFLUX, [&] {
        return launch_macro_bflux(c->stream, g, c->mfp32 == 1, c->model, vquad_d(c), oquad_d(c), nullptr, c->mq, c->mbf);
    }));
    TRY(launch(c, K_HOT, [&] {
        return launch_macro_hot(c->stream, g, c->mfp32 == 1, c->model, c->fields_h, c->mq, c->mgrad, c->kbf, c->mbf,
                                c->hot, c->hot_b);
    }));
    int w = 0;
    TRY(macro_solve(c, &w));
    if (c->closed) {
        TRY(launch(c, K_MCONV, [&] {
            return launch_macro_mass_rescale(c->stream, c->dim, (int)c->nc, c->vol, c->fields, c->W[w]);
        }));
    }
    TRY(launch(c, K_MCONV, [&] {
        return launch_macro_fields_from_W(c->stream, c->dim, (int)c->nc, c->model, c->W[w], c->fields_n);
    }));
    TRY(launch(c, K_SYNC, [&] {
        return launch_sync<Real>(c->stream, c->dim, (int)c->nc, c->tcm >= 1, vquad<Real>(c), oquad<Real>(c), c->model,
                                 c->solver.sync_relax, c->fields_n, c->fields_h, (const Real *)c->coef,
                                 (Real *)c->f[nxt], (Real *)c->I[nxt], (Real *)c->partial, (Real *)c->opartial,
                                 c->sync_kc, c->tc_wait, c->err);
    }));
    TRY(shard_pack<Real>(c, nxt, false));
    c->shard_state = 1;
    return GSIS_OK;
}

// after the last exchange of an iteration (state 1) or a refresh pass (state 3): fields
// from the summed shards (with eps against M^k for an iteration), the summed wall outflow
// for the next wall density, the coefficients
template <typename Real>
int shard_end(gsis_ctx *c) {
    const Geom<Real> g = geom<Real>(c);
    const bool step = c->shard_state == 1;
    if (step) {
        std::swap(c->fields, c->fields_old);
        TRY(launch(c, K_FINISH, [&] {
            return launch_finish<Real>(c->stream, c->dim, (int)c->nc, c->nch, c->och, c->model, (const Real *)c->coef,
                                       (const Real *)c->partial, (const Real *)c->opartial, c->vol, c->fields_old,
                                       c->fields, c->eps_terms, c->err, 1, c->eps_part, c->eps_ticket, c->eps_sums,
                                       c->xbuf);
        }));
    } else {
        TRY(launch(c, K_FINISH, [&] {
            return launch_finish<Real>(c->stream, c->dim, (int)c->nc, c->nch, c->och, c->model, (const Real *)c->coef,
                                       (const Real *)c->partial, (const Real *)c->opartial, c->vol, nullptr,
                                       c->fields, c->eps_terms, c->err, 0, nullptr, nullptr, nullptr, c->xbuf);
        }));
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->wout_g, xbuf_wall(c), (size_t)std::max(c->n_bf, 1) * sizeof(double),
                                cudaMemcpyDeviceToDevice, c->stream));
    TRY(launch(c, K_COEF, [&] {
        return launch_coefficients<Real>(c->stream, c->dim, g, c->model, c->fields, c->cell_dx, (Real *)c->coef);
    }));
    if (step) {
        CUDA_TRY(c, cudaMemcpyAsync(c->h_pinned, c->eps_sums, NEPS * sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(c->h_pinned + NEPS, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        c->cur = c->shard_nxt;
        c->have_eps = true;
        c->eps_pending = true;
        ++c->iter;
    } else {
        c->have_eps = false;
        c->eps_pending = false;
        c->iter = 0;
        c->eps_hist.clear();
    }
    c->shard_state = 0;
    return GSIS_OK;
}

// moments of the current distributions for a refresh: pass 0 about zero velocity, pass 1
// about the velocity pass 0 found (as refresh_fields does without sharding)
template <typename Real>
int shard_refresh(gsis_ctx *c, int pass) {
    CUDA_TRY(c, cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
    if (pass == 0) CUDA_TRY(c, cudaMemsetAsync(c->coef, 0, (size_t)c->nc * cf::NC * c->real_size, c->stream));
    TRY(launch(c, K_MOMENTS, [&] {
        return launch_moments_only<Real>(c->stream, c->dim, (int)c->nc, c->tcm >= 1, vquad<Real>(c), oquad<Real>(c),
                                         (const Real *)c->coef, (const Real *)c->f[c->cur], (const Real *)c->I[c->cur],
                                         (Real *)c->partial, (Real *)c->opartial, c->tc_wait, c->err);
    }));
    TRY(shard_pack<Real>(c, c->cur, false));
    c->shard_state = 3;
    return GSIS_OK;
}

void pack_quad(int n, int pad, int dim, const double *x, const double *w, std::vector<double> &vx,
               std::vector<double> &vw) {
    vx.assign(3 * (size_t)pad, 0.0);
    vw.assign((size_t)pad, 0.0);
    for (int v = 0; v < n; ++v) {
        for (int a = 0; a < dim; ++a) vx[a * (size_t)pad + v] = x[(size_t)v * dim + a];
        vw[v] = w[v];
    }
}

}  // namespace

extern "C" {

int gsis_shard_setup(gsis_ctx *c, int32_t n_xi_all, const double *xi_all, const double *w_all, int32_t n_omega_all,
                     const double *omega_all, const double *wo_all) {
    if (!c || !xi_all || !w_all || !omega_all || !wo_all) return fail(c, GSIS_ERR_INVALID_ARG, "null pointer");
    if (c->sharded) return fail(c, GSIS_ERR_INVALID_ARG, "the context is already a shard");
    if (c->mirrors)
        return fail(c, GSIS_ERR_UNSUPPORTED, "mirror planes pair velocities across shards; shard a mesh without them");
    if (c->dim == 3) return fail(c, GSIS_ERR_UNSUPPORTED, "velocity shards are built for 1-D and 2-D meshes");
    if (c->moff) return fail(c, GSIS_ERR_UNSUPPORTED, "the defect correction is built for unsharded contexts");
    if (n_xi_all < c->V || n_omega_all < c->NO) return fail(c, GSIS_ERR_INVALID_ARG, "the full sets are smaller than the shard");
    const int dim = c->dim;
    // the incoming unit-density wall flux over every velocity of every shard
    std::vector<double> inc((size_t)std::max(c->n_bf, 1), 0.0);
    for (int b = 0; b < c->n_bf; ++b) {
        const double *hw = c->h_wall.data() + (size_t)b * 8;
        if (hw[0] == 0.0) continue;
        const double T = hw[4], norm = std::pow(2.0 * M_PI * T, -0.5 * dim);
        double acc = 0.0;
        for (int v = 0; v < n_xi_all; ++v) {
            double xn = 0.0, c2 = 0.0;
            for (int a = 0; a < dim; ++a) {
                const double x = xi_all[(size_t)v * dim + a];
                xn += x * hw[1 + a];
                c2 += (x - hw[5 + a]) * (x - hw[5 + a]);
            }
            if (xn < 0.0) acc += w_all[v] * xn * norm * std::exp(-c2 / (2.0 * T));
        }
        inc[b] = acc;
    }
    TRY(upload(c, c->bf_inc, inc));
    // the replicated synthetic equations take their boundary fluxes on the full sets
    const int vdp = (n_xi_all + 63) / 64 * 64, odp = (n_omega_all + 63) / 64 * 64;
    std::vector<double> vx, vw, ox, ow;
    pack_quad(n_xi_all, vdp, dim, xi_all, w_all, vx, vw);
    pack_quad(n_omega_all, odp, 3, omega_all, wo_all, ox, ow);
    TRY(dalloc(c, &c->vqd_x, vx.size()));
    TRY(dalloc(c, &c->vqd_w, vw.size()));
    TRY(dalloc(c, &c->oqd_x, ox.size()));
    TRY(dalloc(c, &c->oqd_w, ow.size()));
    TRY(upload(c, c->vqd_x, vx));
    TRY(upload(c, c->vqd_w, vw));
    TRY(upload(c, c->oqd_x, ox));
    TRY(upload(c, c->oqd_w, ow));
    c->Vd = n_xi_all;
    c->Vdp = vdp;
    c->NOd = n_omega_all;
    c->Odp = odp;
    const size_t nbf1 = std::max(c->n_bf, 1);
    c->xcount = (int64_t)((size_t)c->nc * NXC + nbf1 * (1 + KBR));
    TRY(dalloc(c, &c->xbuf, (size_t)c->xcount));
    TRY(dalloc(c, &c->wout_g, nbf1));
    CUDA_TRY(c, cudaMemset(c->xbuf, 0, (size_t)c->xcount * sizeof(double)));
    CUDA_TRY(c, cudaMemset(c->wout_g, 0, nbf1 * sizeof(double)));
    c->sharded = true;
    c->shard_state = 0;
    return GSIS_OK;
}

int gsis_shard_buffer(gsis_ctx *c, void **dev_ptr, int64_t *count) {
    if (!c || !dev_ptr || !count) return GSIS_ERR_INVALID_ARG;
    if (!c->sharded) return fail(c, GSIS_ERR_INVALID_ARG, "not a shard (gsis_shard_setup)");
    *dev_ptr = c->xbuf;
    *count = c->xcount;
    return GSIS_OK;
}

int gsis_shard_refresh(gsis_ctx *c, int32_t pass) {
    if (!c || (pass != 0 && pass != 1)) return GSIS_ERR_INVALID_ARG;
    if (!c->sharded || c->shard_state != 0) return fail(c, GSIS_ERR_INVALID_ARG, "shard phase out of order");
    return c->precision == GSIS_FP64 ? shard_refresh<double>(c, pass) : shard_refresh<float>(c, pass);
}

int gsis_shard_begin(gsis_ctx *c, int32_t mode) {
    if (!c || (mode != GSIS_MODE_CIS && mode != GSIS_MODE_GSIS)) return GSIS_ERR_INVALID_ARG;
    if (!c->sharded || c->shard_state != 0) return fail(c, GSIS_ERR_INVALID_ARG, "shard phase out of order");
    return c->precision == GSIS_FP64 ? shard_begin<double>(c, mode) : shard_begin<float>(c, mode);
}

int gsis_shard_mid(gsis_ctx *c) {
    if (!c) return GSIS_ERR_INVALID_ARG;
    if (!c->sharded || c->shard_state != 2) return fail(c, GSIS_ERR_INVALID_ARG, "shard phase out of order");
    return c->precision == GSIS_FP64 ? shard_mid<double>(c) : shard_mid<float>(c);
}

int gsis_shard_end(gsis_ctx *c, double *eps_out) {
    if (!c) return GSIS_ERR_INVALID_ARG;
    if (!c->sharded || (c->shard_state != 1 && c->shard_state != 3))
        return fail(c, GSIS_ERR_INVALID_ARG, "shard phase out of order");
    const bool step = c->shard_state == 1;
    TRY(c->precision == GSIS_FP64 ? shard_end<double>(c) : shard_end<float>(c));
    if (!step) return check_err(c);
    return read_eps(c, eps_out);
}


int gsis_set_distributions(gsis_ctx *c, const double *f, int64_t f_len, const double *I, int64_t I_len) {
    if (!c || !f || !I) return fail(c, GSIS_ERR_INVALID_ARG, "null buffer");
    if (f_len < c->nc * c->V * 4 || I_len < c->nc * c->NO) return fail(c, GSIS_ERR_INVALID_ARG, "buffer too short");
    // zero the padding so that padded velocities start from a defined state
    CUDA_TRY(c, cudaMemsetAsync(c->f[c->cur], 0, (size_t)c->nc * c->Vp * 4 * c->real_size, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->I[c->cur], 0, (size_t)c->nc * c->Op * c->real_size, c->stream));
    if (c->precision == GSIS_FP64) {
        TRY(gsis_upload_distributions(c, f, I));
    } else {
        std::vector<float> ff(f, f + (size_t)c->nc * c->V * 4), fi(I, I + (size_t)c->nc * c->NO);
        TRY(gsis_upload_distributions(c, ff.data(), fi.data()));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return GSIS_OK;
}

int gsis_get_distributions(gsis_ctx *c, double *f, int64_t f_len, double *I, int64_t I_len) {
    if (!c || !f || !I) return fail(c, GSIS_ERR_INVALID_ARG, "null buffer");
    if (f_len < c->nc * c->V * 4 || I_len < c->nc * c->NO) return fail(c, GSIS_ERR_INVALID_ARG, "buffer too short");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const size_t rs = c->real_size;
    std::vector<unsigned char> hf((size_t)c->nc * c->V * 4 * rs), hi((size_t)c->nc * c->NO * rs);
    CUDA_TRY(c, cudaMemcpy2D(hf.data(), (size_t)c->V * 4 * rs, c->f[c->cur], (size_t)c->Vp * 4 * rs, (size_t)c->V * 4 * rs,
                             (size_t)c->nc, cudaMemcpyDeviceToHost));
    CUDA_TRY(c, cudaMemcpy2D(hi.data(), (size_t)c->NO * rs, c->I[c->cur], (size_t)c->Op * rs, (size_t)c->NO * rs,
                             (size_t)c->nc, cudaMemcpyDeviceToHost));
    const size_t nf = (size_t)c->nc * c->V * 4, ni = (size_t)c->nc * c->NO;
    if (rs == 8) {
        std::memcpy(f, hf.data(), nf * 8);
        std::memcpy(I, hi.data(), ni * 8);
    } else {
        const float *a = reinterpret_cast<const float *>(hf.data()), *b = reinterpret_cast<const float *>(hi.data());
        for (size_t k = 0; k < nf; ++k) f[k] = a[k];
        for (size_t k = 0; k < ni; ++k) I[k] = b[k];
    }
    return GSIS_OK;
}

int gsis_get_fields(gsis_ctx *c, double *out, int64_t len) {
    if (!c || !out || len < c->nc * NF) return fail(c, GSIS_ERR_INVALID_ARG, "fields buffer too short");
    CUDA_TRY(c, cudaMemcpyAsync(out, c->fields, (size_t)c->nc * NF * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return GSIS_OK;
}

int gsis_download_fields_async(gsis_ctx *c, double *out, int64_t len) {
    if (!c || !out || len < c->nc * NF) return fail(c, GSIS_ERR_INVALID_ARG, "fields buffer too short");
    CUDA_TRY(c, cudaMemcpyAsync(out, c->fields, (size_t)c->nc * NF * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return GSIS_OK;
}

int gsis_step_async(gsis_ctx *c, int32_t mode) {
    if (!c) return GSIS_ERR_INVALID_ARG;
    if (c->sharded) return fail(c, GSIS_ERR_UNSUPPORTED, "a velocity shard steps through gsis_shard_begin/mid/end");
    if (mode == GSIS_MODE_GSIS)
        return c->precision == GSIS_FP64 ? gsis_iteration<double>(c) : gsis_iteration<float>(c);
    if (mode != GSIS_MODE_CIS) return fail(c, GSIS_ERR_INVALID_ARG, "bad mode");
    return c->precision == GSIS_FP64 ? cis_iteration<double>(c) : cis_iteration<float>(c);
}

int gsis_last_eps(gsis_ctx *c, double *eps_out) {
    if (!c) return GSIS_ERR_INVALID_ARG;
    if (!c->have_eps) return fail(c, GSIS_ERR_INVALID_ARG, "no iteration since the distributions were set");
    return read_eps(c, eps_out);
}

int gsis_step(gsis_ctx *c, int32_t mode, double *eps_out) {
    TRY(gsis_step_async(c, mode));
    return read_eps(c, eps_out);
}

int gsis_solve(gsis_ctx *c, int32_t mode, int32_t max_outer, double tol, int32_t *iters_out, double *eps_history) {
    if (!c) return GSIS_ERR_INVALID_ARG;
    if (mode != GSIS_MODE_CIS && mode != GSIS_MODE_GSIS) return fail(c, GSIS_ERR_INVALID_ARG, "bad mode");
    const int n = max_outer > 0 ? max_outer : c->solver.max_outer;
    const double t = tol > 0 ? tol : c->solver.tol_outer;
    if (iters_out) *iters_out = 0;
    for (int k = 0; k < n; ++k) {
        const int md = (mode == GSIS_MODE_GSIS && c->iter >= c->solver.n_cis_precond) ? GSIS_MODE_GSIS : GSIS_MODE_CIS;
        double e = 0.0;
        TRY(gsis_step(c, md, &e));
        if (eps_history) eps_history[k] = e;
        if (iters_out) *iters_out = k + 1;
        if (e < t) return GSIS_OK;
    }
    return fail(c, GSIS_ERR_NOT_CONVERGED, "max_outer reached before tol");
}

}  // extern "C"

// ---------------------------------------------------------------- learned closure
namespace {

int mlp_malloc(gsis_ctx *c, void **p, size_t bytes) {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
        *p = nullptr;
        return fail(c, GSIS_ERR_OUT_OF_MEMORY, "learned-closure buffers");
    }
    c->mlp_alloc.push_back(*p);
    return GSIS_OK;
}

void mlp_free(gsis_ctx *c, void *p) {
    if (!p) return;
    cudaFree(p);
    c->mlp_alloc.erase(std::remove(c->mlp_alloc.begin(), c->mlp_alloc.end(), p), c->mlp_alloc.end());
}

// parameters, moments and per-cell buffers once; work buffers for at least n rows
int mlp_ensure(gsis_ctx *c, int64_t n) {
    MlpDev &d = c->mlp;
    if (!d.p) {
        TRY(mlp_malloc(c, (void **)&d.p, MLP_NPARAM * sizeof(float)));
        TRY(mlp_malloc(c, (void **)&d.g, MLP_NW * sizeof(float)));
        TRY(mlp_malloc(c, (void **)&d.m1, MLP_NW * sizeof(float)));
        TRY(mlp_malloc(c, (void **)&d.m2, MLP_NW * sizeof(float)));
        TRY(mlp_malloc(c, &d.pb, MLP_NW * 2));
        TRY(mlp_malloc(c, (void **)&c->mlp_X, (size_t)c->nc * MLP_IN * sizeof(float)));
        TRY(mlp_malloc(c, (void **)&c->mlp_Y, (size_t)c->nc * MLP_OUT * sizeof(float)));
        CUDA_TRY(c, cudaMemsetAsync(d.p, 0, MLP_NPARAM * sizeof(float), c->stream));
        CUDA_TRY(c, cudaMemsetAsync(d.m1, 0, MLP_NW * sizeof(float), c->stream));
        CUDA_TRY(c, cudaMemsetAsync(d.m2, 0, MLP_NW * sizeof(float), c->stream));
    }
    if (n > d.cap) {
        const int widths[MLP_LAYERS + 1] = {MLP_IN, MLP_H, MLP_H, MLP_H, MLP_OUT};
        for (int l = 0; l <= MLP_LAYERS; ++l) mlp_free(c, d.act[l]);
        for (int l = 0; l < MLP_LAYERS; ++l) mlp_free(c, d.pre[l]);
        mlp_free(c, d.dA[0]);
        mlp_free(c, d.dA[1]);
        mlp_free(c, d.T);
        mlp_free(c, d.lpart);
        mlp_free(c, c->mlp_idx);
        for (int l = 0; l <= MLP_LAYERS; ++l) TRY(mlp_malloc(c, (void **)&d.act[l], n * widths[l] * sizeof(float)));
        for (int l = 0; l < MLP_LAYERS; ++l) TRY(mlp_malloc(c, (void **)&d.pre[l], n * widths[l + 1] * sizeof(float)));
        TRY(mlp_malloc(c, (void **)&d.dA[0], n * MLP_H * sizeof(float)));
        TRY(mlp_malloc(c, (void **)&d.dA[1], n * MLP_H * sizeof(float)));
        TRY(mlp_malloc(c, (void **)&d.T, n * MLP_OUT * sizeof(float)));
        TRY(mlp_malloc(c, (void **)&d.lpart, (size_t)mlp_loss_parts((int)n) * sizeof(double)));
        TRY(mlp_malloc(c, (void **)&c->mlp_idx, n * sizeof(int)));
        d.cap = (int)n;
    }
    return GSIS_OK;
}

const float *x_mean(const gsis_ctx *c) { return c->mlp.p + MLP_NW; }
const float *x_std(const gsis_ctx *c) { return c->mlp.p + MLP_NW + MLP_IN; }
const float *y_mean(const gsis_ctx *c) { return c->mlp.p + MLP_NW + 2 * MLP_IN; }
const float *y_std(const gsis_ctx *c) { return c->mlp.p + MLP_NW + 2 * MLP_IN + MLP_OUT; }

// forward pass of n rows already standardised in act[0]; loss over standardised targets in T
int mlp_loss(gsis_ctx *c, int n, double *loss) {
    MlpDev &d = c->mlp;
    CUDA_TRY(c, launch_mlp_forward(c->stream, d, n));
    CUDA_TRY(c, launch_mlp_loss_backward(c->stream, d, n));
    c->launches += 4 + 1 + 3 + 4 + 3;
    if (loss) {
        const int np = mlp_loss_parts(n);
        std::vector<double> part(np);
        CUDA_TRY(c, cudaMemcpyAsync(part.data(), d.lpart, np * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        double sum = 0.0;
        for (double x : part) sum += x;
        *loss = sum / ((double)n * MLP_OUT);
    }
    return GSIS_OK;
}

}  // namespace

extern "C" {

int gsis_mlp_set_params(gsis_ctx *c, const float *p, int64_t len) {
    if (!c || !p || len < MLP_NPARAM) return fail(c, GSIS_ERR_INVALID_ARG, "parameter buffer too short");
    TRY(mlp_ensure(c, 1));
    CUDA_TRY(c, cudaMemcpyAsync(c->mlp.p, p, MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->mlp.m1, 0, MLP_NW * sizeof(float), c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->mlp.m2, 0, MLP_NW * sizeof(float), c->stream));
    CUDA_TRY(c, launch_mlp_to_bf16(c->stream, c->mlp));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->mlp.step = 0;
    c->mlp.trained = true;
    return GSIS_OK;
}

int gsis_mlp_get_params(gsis_ctx *c, float *p, int64_t len) {
    if (!c || !p || len < MLP_NPARAM) return fail(c, GSIS_ERR_INVALID_ARG, "parameter buffer too short");
    if (!c->mlp.p) return fail(c, GSIS_ERR_INVALID_ARG, "no network parameters yet");
    CUDA_TRY(c, cudaMemcpyAsync(p, c->mlp.p, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return GSIS_OK;
}

int gsis_mlp_init(gsis_ctx *c, uint64_t seed) {
    if (!c) return GSIS_ERR_INVALID_ARG;
    std::vector<float> p(MLP_NPARAM, 0.0f);
    std::mt19937_64 rng(seed);
    size_t o = 0;
    const int ins[MLP_LAYERS] = {MLP_IN, MLP_H, MLP_H, MLP_H}, outs[MLP_LAYERS] = {MLP_H, MLP_H, MLP_H, MLP_OUT};
    for (int l = 0; l < MLP_LAYERS; ++l) {
        std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / ins[l]));
        for (int k = 0; k < outs[l] * ins[l]; ++k) p[o++] = (float)nd(rng);
        o += outs[l];   // zero biases
    }
    for (int k = 0; k < MLP_IN; ++k) p[MLP_NW + MLP_IN + k] = 1.0f;                       // x_std
    for (int k = 0; k < MLP_OUT; ++k) p[MLP_NW + 2 * MLP_IN + MLP_OUT + k] = 1.0f;        // y_std
    TRY(gsis_mlp_set_params(c, p.data(), MLP_NPARAM));
    c->mlp.trained = false;
    return GSIS_OK;
}

int gsis_mlp_loss_grad(gsis_ctx *c, const float *X, const float *Y, int64_t n, double *loss, float *grad) {
    if (!c || !X || !Y || n <= 0) return fail(c, GSIS_ERR_INVALID_ARG, "bad samples");
    if (!c->mlp.p) return fail(c, GSIS_ERR_INVALID_ARG, "no network parameters yet");
    TRY(mlp_ensure(c, n));
    MlpDev &d = c->mlp;
    CUDA_TRY(c, cudaMemcpyAsync(d.act[0], X, n * MLP_IN * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(d.T, Y, n * MLP_OUT * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, launch_mlp_standardise(c->stream, (int)n, MLP_IN, d.act[0], x_mean(c), x_std(c), 0));
    CUDA_TRY(c, launch_mlp_standardise(c->stream, (int)n, MLP_OUT, d.T, y_mean(c), y_std(c), 0));
    TRY(mlp_loss(c, (int)n, loss));
    if (grad) {
        CUDA_TRY(c, cudaMemcpyAsync(grad, d.g, MLP_NW * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    return GSIS_OK;
}

int gsis_mlp_predict(gsis_ctx *c, const float *X, int64_t n, float *Y) {
    if (!c || !X || !Y || n <= 0) return fail(c, GSIS_ERR_INVALID_ARG, "bad samples");
    if (!c->mlp.p) return fail(c, GSIS_ERR_INVALID_ARG, "no network parameters yet");
    TRY(mlp_ensure(c, n));
    MlpDev &d = c->mlp;
    CUDA_TRY(c, cudaMemcpyAsync(d.act[0], X, n * MLP_IN * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, launch_mlp_standardise(c->stream, (int)n, MLP_IN, d.act[0], x_mean(c), x_std(c), 0));
    CUDA_TRY(c, launch_mlp_forward(c->stream, d, (int)n));
    CUDA_TRY(c, launch_mlp_standardise(c->stream, (int)n, MLP_OUT, d.act[MLP_LAYERS], y_mean(c), y_std(c), 1));
    CUDA_TRY(c, cudaMemcpyAsync(Y, d.act[MLP_LAYERS], n * MLP_OUT * sizeof(float), cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->launches += 6;
    return GSIS_OK;
}

int gsis_mlp_train(gsis_ctx *c, const float *X, const float *Y, int64_t n, int32_t epochs, int32_t batch, double lr,
                   uint64_t seed, double *loss_out) {
    if (!c || !X || !Y || n <= 0 || epochs < 0 || batch <= 0 || !(lr > 0))
        return fail(c, GSIS_ERR_INVALID_ARG, "bad training arguments");
    for (int64_t k = 0; k < n * MLP_IN; ++k)
        if (!std::isfinite(X[k])) return fail(c, GSIS_ERR_INVALID_ARG, "non-finite training input");
    for (int64_t k = 0; k < n * MLP_OUT; ++k)
        if (!std::isfinite(Y[k])) return fail(c, GSIS_ERR_INVALID_ARG, "non-finite training target");
    if (!c->mlp.p) TRY(gsis_mlp_init(c, seed));
    const int64_t b = std::min<int64_t>(batch, n);
    TRY(mlp_ensure(c, b));
    MlpDev &d = c->mlp;
    // standardisation from the data (FP64 sums), kept with the parameters
    std::vector<float> stat(MLP_NSTAT);
    auto moments = [&](const float *A, int m, float *mean, float *sd) {
        for (int j = 0; j < m; ++j) {
            double s = 0.0, s2 = 0.0;
            for (int64_t r = 0; r < n; ++r) {
                const double x = A[r * m + j];
                s += x;
                s2 += x * x;
            }
            const double mu = s / n, var = std::max(s2 / n - mu * mu, 0.0);
            mean[j] = (float)mu;
            sd[j] = var > 0 ? (float)std::sqrt(var) : 1.0f;
        }
    };
    moments(X, MLP_IN, stat.data(), stat.data() + MLP_IN);
    moments(Y, MLP_OUT, stat.data() + 2 * MLP_IN, stat.data() + 2 * MLP_IN + MLP_OUT);
    CUDA_TRY(c, cudaMemcpyAsync(d.p + MLP_NW, stat.data(), MLP_NSTAT * sizeof(float), cudaMemcpyHostToDevice,
                                c->stream));
    // the data set on the device, standardised
    const int64_t need = n * (MLP_IN + MLP_OUT);
    if (need > c->mlp_data_cap) {
        mlp_free(c, c->mlp_data);
        TRY(mlp_malloc(c, (void **)&c->mlp_data, need * sizeof(float)));
        c->mlp_data_cap = need;
    }
    float *Xd = c->mlp_data, *Yd = c->mlp_data + n * MLP_IN;
    CUDA_TRY(c, cudaMemcpyAsync(Xd, X, n * MLP_IN * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(Yd, Y, n * MLP_OUT * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, launch_mlp_standardise(c->stream, (int)n, MLP_IN, Xd, x_mean(c), x_std(c), 0));
    CUDA_TRY(c, launch_mlp_standardise(c->stream, (int)n, MLP_OUT, Yd, y_mean(c), y_std(c), 0));
    std::vector<int> perm(n);
    for (int64_t r = 0; r < n; ++r) perm[r] = (int)r;
    std::mt19937_64 rng(seed ^ 0x9E3779B97F4A7C15ull);
    double last = 0.0;
    for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        for (int64_t s0 = 0; s0 + b <= n; s0 += b) {
            CUDA_TRY(c, cudaMemcpyAsync(c->mlp_idx, perm.data() + s0, b * sizeof(int), cudaMemcpyHostToDevice,
                                        c->stream));
            CUDA_TRY(c, launch_mlp_gather(c->stream, (int)b, MLP_IN, c->mlp_idx, Xd, d.act[0]));
            CUDA_TRY(c, launch_mlp_gather(c->stream, (int)b, MLP_OUT, c->mlp_idx, Yd, d.T));
            const bool report = ep == epochs - 1 && s0 + 2 * b > n;
            TRY(mlp_loss(c, (int)b, report ? &last : nullptr));
            CUDA_TRY(c, launch_mlp_adam(c->stream, d, (float)lr));
            c->launches += 3;
        }
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    d.trained = true;
    if (loss_out) *loss_out = last;
    return GSIS_OK;
}

int gsis_mlp_samples(gsis_ctx *c, float *X, float *Y, int64_t n_cells) {
    if (!c || !X || n_cells < c->nc) return fail(c, GSIS_ERR_INVALID_ARG, "sample buffers too short");
    if (c->dim == 3) return fail(c, GSIS_ERR_UNSUPPORTED, "the learned closure's features are built for 1-D and 2-D");
    TRY(mlp_ensure(c, 1));
    TRY(launch(c, K_MCONV, [&] {
        return launch_macro_from_fields(c->stream, c->dim, (int)c->nc, c->model, c->fields, c->W[0]);
    }));
    TRY(launch(c, K_MGRAD, [&] {
        return launch_macro_grad(c->stream, c->mg, 1, 0, c->model, nullptr, c->W[0], c->mq, c->mgrad, c->mphi);
    }));
    TRY(launch(c, K_MLP, [&] {
        return launch_cell_features(c->stream, c->mg, c->model, c->fields, c->mq, c->mgrad, c->mlp_X,
                                    Y ? c->mlp_Y : nullptr);
    }));
    CUDA_TRY(c, cudaMemcpyAsync(X, c->mlp_X, c->nc * MLP_IN * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    if (Y)
        CUDA_TRY(c, cudaMemcpyAsync(Y, c->mlp_Y, c->nc * MLP_OUT * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return GSIS_OK;
}

}  // extern "C"

template <typename Real>
int warm_start(gsis_ctx *c, int n_presolve, bool use_mlp) {
    const MacroGeom &g = c->mg;
    if (use_mlp) TRY(mlp_ensure(c, c->nc));
    for (int k = 0; k < n_presolve; ++k) {
        TRY(launch(c, K_MCONV, [&] {
            return launch_macro_from_fields(c->stream, c->dim, (int)c->nc, c->model, c->fields, c->W[0]);
        }));
        TRY(launch(c, K_MGRAD, [&] {
            return launch_macro_grad(c->stream, g, 1, 0, c->model, nullptr, c->W[0], c->mq, c->mgrad, c->mphi);
        }));
        if (use_mlp) {
            MlpDev &d = c->mlp;
            TRY(launch(c, K_MLP, [&] {
                return launch_cell_features(c->stream, g, c->model, c->fields, c->mq, c->mgrad, d.act[0], nullptr);
            }));
            CUDA_TRY(c, launch_mlp_standardise(c->stream, (int)c->nc, MLP_IN, d.act[0], x_mean(c), x_std(c), 0));
            CUDA_TRY(c, launch_mlp_forward(c->stream, d, (int)c->nc));
            CUDA_TRY(c, launch_mlp_standardise(c->stream, (int)c->nc, MLP_OUT, d.act[MLP_LAYERS], y_mean(c), y_std(c),
                                               1));
            c->launches += 6;
            TRY(launch(c, K_MLP, [&] {
                return launch_hot_from_cells(c->stream, g, c->mq, d.act[MLP_LAYERS], c->hot, c->hot_b);
            }));
        } else {
            CUDA_TRY(c, cudaMemsetAsync(c->hot, 0, (size_t)std::max(g.n_fi, 1) * NHOT * sizeof(double), c->stream));
            CUDA_TRY(c, cudaMemsetAsync(c->hot_b, 0, (size_t)std::max(g.n_bf, 1) * NVM * sizeof(double), c->stream));
        }
        if (c->moff)   // the pre-solve has no kinetic residual: no offset
            CUDA_TRY(c, cudaMemsetAsync(c->moff, 0, (size_t)c->nc * NVM * sizeof(double), c->stream));
        int w = 0;
        TRY(macro_solve(c, &w));
        if (c->closed) {
            TRY(launch(c, K_MCONV, [&] {
                return launch_macro_mass_rescale(c->stream, c->dim, (int)c->nc, c->vol, c->fields, c->W[w]);
            }));
        }
        TRY(launch(c, K_MCONV, [&] {
            return launch_macro_fields_from_W(c->stream, c->dim, (int)c->nc, c->model, c->W[w], c->fields_n);
        }));
        std::swap(c->fields, c->fields_n);
    }
    TRY(launch(c, K_EQUIL, [&] {
        return launch_equilibrium<Real>(c->stream, c->dim, (int)c->nc, vquad<Real>(c), oquad<Real>(c), c->model,
                                        c->fields, (Real *)c->f[c->cur], (Real *)c->I[c->cur]);
    }));
    TRY(refresh(c));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return GSIS_OK;
}

extern "C" {

int gsis_warm_start(gsis_ctx *c, int32_t n_presolve, int32_t use_mlp) {
    if (!c || n_presolve < 0) return GSIS_ERR_INVALID_ARG;
    if (c->sharded) return fail(c, GSIS_ERR_UNSUPPORTED, "the warm start runs on unsharded contexts");
    if (c->dim == 3 && use_mlp)
        return fail(c, GSIS_ERR_UNSUPPORTED, "the learned closure's features are built for 1-D and 2-D");
    if (use_mlp && (!c->mlp.p || !c->mlp.trained))
        return fail(c, GSIS_ERR_INVALID_ARG, "the learned closure has not been trained or set");
    return c->precision == GSIS_FP64 ? warm_start<double>(c, n_presolve, use_mlp != 0)
                                     : warm_start<float>(c, n_presolve, use_mlp != 0);
}

int gsis_macro_stats(gsis_ctx *c, int32_t *inner_iters, double *r0, double *rn) {
    if (!c) return GSIS_ERR_INVALID_ARG;
    CUDA_TRY(c, cudaMemcpyAsync(c->h_mstate, c->mstate, sizeof(MacroState), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (inner_iters) *inner_iters = c->h_mstate->it;
    if (r0) *r0 = c->h_mstate->r0;
    if (rn) *rn = c->h_mstate->rn;
    return GSIS_OK;
}

int gsis_profile_enable(gsis_ctx *c, int32_t on) {
    if (!c) return GSIS_ERR_INVALID_ARG;
    c->prof = on != 0;
    return GSIS_OK;
}

int gsis_profile_reset(gsis_ctx *c) {
    if (!c) return GSIS_ERR_INVALID_ARG;
    TRY(resolve_profile(c));
    for (int k = 0; k < K_COUNT; ++k) {
        c->prof_ms[k] = 0.0;
        c->prof_n[k] = 0;
    }
    return GSIS_OK;
}

int gsis_profile_read(gsis_ctx *c, int32_t n, const char **names, double *ms, int64_t *launches, int32_t *n_out) {
    if (!c) return GSIS_ERR_INVALID_ARG;
    TRY(resolve_profile(c));
    for (int k = 0; k < K_COUNT && k < n; ++k) {
        if (names) names[k] = kKernelNames[k];
        if (ms) ms[k] = c->prof_ms[k];
        if (launches) launches[k] = c->prof_n[k];
    }
    if (n_out) *n_out = K_COUNT;
    return GSIS_OK;
}

int64_t gsis_launch_count(const gsis_ctx *c) { return c ? c->launches : 0; }

int gsis_get_layout(const gsis_ctx *c, int32_t *v_pad, int32_t *o_pad, int32_t *n_chunks, int32_t *block) {
    if (!c) return GSIS_ERR_INVALID_ARG;
    if (v_pad) *v_pad = c->Vp;
    if (o_pad) *o_pad = c->Op;
    if (n_chunks) *n_chunks = c->nch;
    if (block) *block = c->block;
    return GSIS_OK;
}

}  // extern "C"
