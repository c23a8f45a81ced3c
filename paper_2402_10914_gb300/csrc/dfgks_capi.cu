// dfgks_capi.cu -- the extern "C" boundary declared in include/dfgks.h: handle lifecycle,
// state transfer, the step driver (Algorithm 1 of arXiv 2402.10914) and the stage operator.
#include <cuda_runtime.h>
#include <float.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <new>
#include <vector>

#include "../../include/dfgks.h"
#include "dfgks_internal.h"

using namespace dfk;

struct dfgks {
    dfgks_config cfg;
    cudaStream_t stream;
    bool own_stream;
    Mesh mesh;
    SchemeConsts S;
    double* W[2];          // ghosted states (current / next)
    double* A[2];          // ghosted alpha (current / next)
    int cur;
    double* Ws;            // ghosted stage state; also the residual input
    double* As;            // ghosted alpha scratch for the residual input
    double* acc;           // dense [4][ny][nx]: S2O4 accumulator and transfer staging
    SweepBuffers B;
    SweepBuffers By;       // the y-faces' face-line and Gauss-point records of the fused x/y sweeps
    DevState* st;          // device step state
    DevState* st_host;     // pinned mirror
    int* flag;             // device scratch flag
    int* flag_host;        // pinned mirror
    double* dt_scratch;    // device dt for residual calls
    double* dts;           // device dt history of one dfgks_step call
    int dts_cap;
    unsigned long long bytes;
    long long fail_step;
    int fail_i, fail_j;
    KernelTimer* timer;    // per-kernel-class event timing and launch counts
    double* adj_lines;     // reverse sweep: face-line record adjoints
    double* adj_gp;        // reverse sweep: Gauss-point record adjoints
    double* adj_Wg;        // reverse sweep: ghosted cell adjoints
    // checkpointed forward pass kept for dfgks_adjoint_checkpointed
    double* ck_W;          // dense [nseg][4][ny][nx]: W at steps 0, k, 2k, ...
    double* ck_A;          // dense [nseg][ny][nx]: alpha at the same steps
    long long ck_cap;      // checkpoints ck_W / ck_A can hold
    double* ck_dts;        // host [ck_n]: the steps' dt
    int ck_dts_cap;
    int ck_n, ck_k, ck_flux;
    unsigned long long gen;      // bumped by every call that changes the state
    unsigned long long ck_gen;   // gen right after the checkpointed forward pass (0: none)
    // segment arena of the reverse pass: per step of one segment W^s, alpha^s, W* (dense) and,
    // when they fit, the forward sweep records (with tapes); the forward pass fills it for the
    // last segment, so the reverse pass recomputes only the earlier ones
    double* seg_arena;
    long long seg_cap;           // doubles allocated
    int seg_k, seg_records, seg_tape, seg_gks;
    int seg_slots;               // segments the arena holds
    int seg_kept;                // trailing segments of the last forward pass still in the arena (0: none)
};

static dfgks_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return DFGKS_OK;
    if (e == cudaErrorMemoryAllocation) return DFGKS_ENOMEM;
    return DFGKS_ECUDA;
}
#define CK(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) return cuda_status(e_); } while (0)
#define CK_LAUNCH() CK(cudaGetLastError())

extern "C" const char* dfgks_status_string(int s) {
    switch (s) {
        case DFGKS_OK: return "ok";
        case DFGKS_EINVAL: return "invalid argument";
        case DFGKS_ENOMEM: return "out of memory";
        case DFGKS_ECUDA: return "CUDA error";
        case DFGKS_ENONPHYS: return "non-physical state (rho<=0, p<=0 or non-finite)";
        case DFGKS_ENONPOS: return "positivity lost during a step";
        case DFGKS_ENAN: return "non-finite value";
        case DFGKS_ETIMEOUT: return "bounded device wait expired";
        case DFGKS_ENOTSUP: return "not supported";
        default: return "unknown status";
    }
}

extern "C" dfgks_status dfgks_config_default(dfgks_config* c, int nx, int ny) {
    if (!c) return DFGKS_EINVAL;
    memset(c, 0, sizeof(*c));
    c->nx = nx; c->ny = ny;
    c->x0 = 0.0; c->x1 = 1.0; c->y0 = 0.0; c->y1 = 1.0;
    c->gamma = 1.4; c->cfl = 0.5;
    c->bc_xlo = c->bc_xhi = c->bc_ylo = c->bc_yhi = DFGKS_BC_OUTFLOW;
    c->alpha_thres = 0.5; c->dH = 0.85; c->dL = 0.85; c->eps = 1e-6; c->C1 = 0.01; c->C2 = 5.0;
    c->time_limiter = 1; c->tau_reading = 0; c->gp_fallback = 1; c->time_scheme = DFGKS_TIME_S2O4;
    c->dt_rule = 0;
    c->df_states = 0;
    c->alpha_source = 0;
    return DFGKS_OK;
}

static bool config_ok(const dfgks_config* c) {
    if (!c || c->nx < 1 || c->ny < 1 || c->nx > (1 << 20) || c->ny > (1 << 20)) return false;
    if ((long long)c->nx * c->ny > (1LL << 31) / 8) return false;
    if (!(c->x1 > c->x0) || !(c->y1 > c->y0)) return false;
    if (!(c->gamma > 1.0) || !(c->cfl > 0.0) || !(c->eps > 0.0)) return false;
    if (!(c->dH > 0.0 && c->dH <= 1.0) || !(c->dL >= 0.0 && c->dL <= 1.0)) return false;
    if (!(c->C1 >= 0.0) || !(c->C2 >= 0.0)) return false;
    const int bcs[4] = {c->bc_xlo, c->bc_xhi, c->bc_ylo, c->bc_yhi};
    for (int k = 0; k < 4; ++k) if (bcs[k] < 0 || bcs[k] > 2) return false;
    if ((c->bc_xlo == 0) != (c->bc_xhi == 0) || (c->bc_ylo == 0) != (c->bc_yhi == 0)) return false;
    // periodic wrap and wall mirror both copy G interior cells into the ghost layers
    if ((c->bc_xlo != 1 || c->bc_xhi != 1) && c->nx < G) return false;
    if ((c->bc_ylo != 1 || c->bc_yhi != 1) && c->ny < G) return false;
    if (c->time_scheme != 0 && c->time_scheme != 1) return false;
    if (c->tau_reading != 0 && c->tau_reading != 1) return false;
    if (c->dt_rule != 0 && c->dt_rule != 1) return false;
    if (c->df_states != 0 && c->df_states != 1) return false;
    if (c->alpha_source != 0 && c->alpha_source != 1) return false;
    return true;
}

static void free_all(dfgks* h) {
    double* ptrs[] = {h->W[0], h->W[1], h->A[0], h->A[1], h->Ws, h->As, h->acc, h->B.lines, h->B.gp,
                      h->B.flux[0], h->B.flux[1], h->By.lines, h->By.gp, h->dt_scratch, h->dts, h->adj_lines,
                      h->adj_gp, h->adj_Wg};
    for (double* p : ptrs) if (p) cudaFree(p);
    if (h->seg_arena) cudaFree(h->seg_arena);
    if (h->ck_W) cudaFree(h->ck_W);
    if (h->ck_A) cudaFree(h->ck_A);
    free(h->ck_dts);
    if (h->st) cudaFree(h->st);
    if (h->flag) cudaFree(h->flag);
    if (h->st_host) cudaFreeHost(h->st_host);
    if (h->flag_host) cudaFreeHost(h->flag_host);
    if (h->timer) {
        for (cudaEvent_t e : h->timer->ev) cudaEventDestroy(e);
        delete h->timer;
    }
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

static long long round4(long long n) { return (n + 3) & ~3LL; }

static cudaError_t dalloc(dfgks* h, double** p, long long n) {
    cudaError_t e = cudaMalloc((void**)p, (size_t)n * sizeof(double));
    if (e == cudaSuccess) h->bytes += (unsigned long long)n * sizeof(double);
    return e;
}

static dfgks_status reset_devstate(dfgks* h, double t, long long step) {
    DevState s;
    memset(&s, 0, sizeof(s));
    s.t = t;
    s.step = step;
    s.dtmin_bits = 0x7FEFFFFFFFFFFFFFULL;   // DBL_MAX
    s.fail_step = -1;
    s.fail_key = ~0ULL;
    *h->st_host = s;
    CK(cudaMemcpyAsync(h->st, h->st_host, sizeof(DevState), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return DFGKS_OK;
}

extern "C" dfgks_status dfgks_create(const dfgks_config* cfg, void* stream, dfgks** out) {
    if (!out) return DFGKS_EINVAL;
    *out = nullptr;
    if (!config_ok(cfg)) return DFGKS_EINVAL;
    dfgks* h = new (std::nothrow) dfgks;
    if (!h) return DFGKS_ENOMEM;
    memset(h, 0, sizeof(*h));
    h->cfg = *cfg;
    if (stream) { h->stream = (cudaStream_t)stream; h->own_stream = false; }
    else {
        cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete h; return cuda_status(e); }
        h->own_stream = true;
    }
    Mesh& m = h->mesh;
    m.nx = cfg->nx; m.ny = cfg->ny;
    m.P = (int)round4(cfg->nx + 2 * G);
    m.NYg = cfg->ny + 2 * G;
    m.plane = (long long)m.P * m.NYg;
    m.dx = (cfg->x1 - cfg->x0) / cfg->nx;
    m.dy = (cfg->y1 - cfg->y0) / cfg->ny;
    m.rdx = 1.0 / m.dx; m.rdy = 1.0 / m.dy;
    m.bc[0] = cfg->bc_xlo; m.bc[1] = cfg->bc_xhi; m.bc[2] = cfg->bc_ylo; m.bc[3] = cfg->bc_yhi;
    m.dt_rule = cfg->dt_rule;
    SchemeConsts& S = h->S;
    S.gamma = cfg->gamma; S.gm1 = cfg->gamma - 1.0; S.K = (4.0 - 2.0 * cfg->gamma) / (cfg->gamma - 1.0);
    S.inv_K2 = 1.0 / (S.K + 2.0);
    S.r2g = sqrt(2.0 / S.gamma);
    S.d[3] = cfg->dH;
    S.d[0] = (1.0 - cfg->dH) * (1.0 - cfg->dL) / 2.0;
    S.d[1] = (1.0 - cfg->dH) * cfg->dL;
    S.d[2] = S.d[0];
    S.inv_d3 = 1.0 / cfg->dH;
    S.eps = cfg->eps; S.alpha_thres = cfg->alpha_thres; S.C1 = cfg->C1; S.C2 = cfg->C2;
    S.time_limiter = cfg->time_limiter; S.tau_reading = cfg->tau_reading; S.gp_fallback = cfg->gp_fallback;
    S.df_states = cfg->df_states;

    const long long nfx = (long long)(m.nx + 1) * m.ny, nfy = (long long)(m.ny + 1) * m.nx;
    const long long nlx = (long long)(m.nx + 1) * (m.ny + 4), nly = (long long)(m.ny + 1) * (m.nx + 4);
    h->B.line_stride = round4(nlx > nly ? nlx : nly);
    h->B.gp_stride = round4(2 * (nfx > nfy ? nfx : nfy));
    h->B.flux_stride[0] = round4(2 * nfx);
    h->B.flux_stride[1] = round4(2 * nfy);
    const long long dense = (long long)m.nx * m.ny;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dalloc(h, &h->W[0], 4 * m.plane);
    if (e == cudaSuccess) e = dalloc(h, &h->W[1], 4 * m.plane);
    if (e == cudaSuccess) e = dalloc(h, &h->A[0], m.plane);
    if (e == cudaSuccess) e = dalloc(h, &h->A[1], m.plane);
    if (e == cudaSuccess) e = dalloc(h, &h->Ws, 4 * m.plane);
    if (e == cudaSuccess) e = dalloc(h, &h->As, m.plane);
    if (e == cudaSuccess) e = dalloc(h, &h->acc, 4 * dense);
    if (e == cudaSuccess) e = dalloc(h, &h->B.lines, (long long)LR_COUNT * h->B.line_stride);
    if (e == cudaSuccess) e = dalloc(h, &h->B.gp, (long long)GP_COUNT * h->B.gp_stride);
    if (e == cudaSuccess) e = dalloc(h, &h->B.flux[0], (long long)FR_COUNT * h->B.flux_stride[0]);
    if (e == cudaSuccess) e = dalloc(h, &h->B.flux[1], (long long)FR_COUNT * h->B.flux_stride[1]);
    h->By = h->B;
    h->By.lines = nullptr;
    h->By.gp = nullptr;
    if (e == cudaSuccess) e = dalloc(h, &h->By.lines, (long long)LR_COUNT * h->B.line_stride);
    if (e == cudaSuccess) e = dalloc(h, &h->By.gp, (long long)GP_COUNT * h->B.gp_stride);
    if (e == cudaSuccess) e = dalloc(h, &h->dt_scratch, 4);
    if (e == cudaSuccess) { h->dts_cap = 1024; e = dalloc(h, &h->dts, h->dts_cap); }
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->st, sizeof(DevState));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&h->st_host, sizeof(DevState));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&h->flag_host, sizeof(int));
    if (e != cudaSuccess) { free_all(h); delete h; return cuda_status(e); }
    // defined contents everywhere (ghost corners of the alpha scratch, unused pitch columns)
    launch_fill_value(h->W[0], 4 * m.plane, 1.0, h->stream);
    launch_fill_value(h->W[1], 4 * m.plane, 1.0, h->stream);
    launch_fill_value(h->Ws, 4 * m.plane, 1.0, h->stream);
    launch_fill_value(h->A[0], m.plane, 1.0, h->stream);
    launch_fill_value(h->A[1], m.plane, 1.0, h->stream);
    launch_fill_value(h->As, m.plane, 1.0, h->stream);
    h->cur = 0;
    h->fail_step = -1; h->fail_i = -1; h->fail_j = -1;
    h->timer = new (std::nothrow) KernelTimer();
    if (!h->timer) { free_all(h); delete h; return DFGKS_ENOMEM; }
    h->timer->stream = h->stream;
    dfgks_status r = reset_devstate(h, 0.0, 0);
    if (r == DFGKS_OK) r = cuda_status(cudaGetLastError());
    if (r != DFGKS_OK) { free_all(h); delete h; return r; }
    *out = h;
    return DFGKS_OK;
}

extern "C" dfgks_status dfgks_destroy(dfgks* h) {
    if (!h) return DFGKS_OK;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
    return DFGKS_OK;
}

// copy a dense [nc][ny][nx] array (host or device) into h->acc
static dfgks_status stage_in(dfgks* h, const double* src, int nc, int on_device) {
    size_t bytes = (size_t)nc * h->mesh.nx * h->mesh.ny * sizeof(double);
    CK(cudaMemcpyAsync(h->acc, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    return DFGKS_OK;
}

// alpha^0: product of the Gauss-point DF factors of a reconstruction of W with alpha = 1
static dfgks_status compute_alpha0(dfgks* h, double* Wg, double* Ag) {
    launch_fill_value(Ag, h->mesh.plane, 1.0, h->stream);
    launch_fill_ghosts(h->mesh, Wg, nullptr, nullptr, h->stream);
    launch_set_scalar(h->dt_scratch, 1.0, h->stream);
    launch_sweep_xy(h->mesh, h->S, 1, true, Wg, Ag, h->dt_scratch, h->B, h->By, nullptr, nullptr, h->stream);
    UpdateArgs a;
    memset(&a, 0, sizeof(a));
    a.alpha_out = Ag;
    a.alpha_dense = 0;
    launch_update(UM_ALPHA, h->mesh, h->S, a, h->B, h->dt_scratch, nullptr, nullptr, h->stream);
    CK_LAUNCH();
    return DFGKS_OK;
}

static dfgks_status load_state(dfgks* h, const double* W, const double* alpha, double t, long long step, int on_device) {
    dfgks_status r = stage_in(h, W, 4, on_device);
    if (r) return r;
    // validate in the stage buffer first so a rejected state leaves the current one untouched
    launch_dense_to_ghosted(h->mesh, h->acc, 4, h->Ws, h->stream);
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
    launch_check_state(h->mesh, h->Ws, h->S.gm1, h->flag, h->stream);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(h->flag_host, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (*h->flag_host) return DFGKS_ENONPHYS;
    launch_dense_to_ghosted(h->mesh, h->acc, 4, h->W[h->cur], h->stream);
    if (alpha) {
        r = stage_in(h, alpha, 1, on_device);
        if (r) return r;
        launch_fill_value(h->A[h->cur], h->mesh.plane, 1.0, h->stream);
        launch_dense_to_ghosted(h->mesh, h->acc, 1, h->A[h->cur], h->stream);
    } else {
        r = compute_alpha0(h, h->W[h->cur], h->A[h->cur]);
        if (r) return r;
    }
    CK_LAUNCH();
    h->fail_step = -1; h->fail_i = -1; h->fail_j = -1;
    ++h->gen;
    return reset_devstate(h, t, step);
}

extern "C" dfgks_status dfgks_set_ic(dfgks* h, const double* W, int on_device) {
    if (!h || !W) return DFGKS_EINVAL;
    return load_state(h, W, nullptr, 0.0, 0, on_device);
}

extern "C" dfgks_status dfgks_set_state(dfgks* h, const double* W, const double* alpha, double t, long step, int on_device) {
    if (!h || !W || step < 0) return DFGKS_EINVAL;
    return load_state(h, W, alpha, t, step, on_device);
}

extern "C" dfgks_status dfgks_get_state(dfgks* h, double* W, double* alpha, double* t, long* step, int on_device) {
    if (!h) return DFGKS_EINVAL;
    const size_t n = (size_t)h->mesh.nx * h->mesh.ny;
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (W) {
        launch_ghosted_to_dense(h->mesh, h->W[h->cur], 4, h->acc, h->stream);
        CK_LAUNCH();
        CK(cudaMemcpyAsync(W, h->acc, 4 * n * sizeof(double), kind, h->stream));
    }
    if (alpha) {
        launch_ghosted_to_dense(h->mesh, h->A[h->cur], 1, h->acc, h->stream);
        CK_LAUNCH();
        CK(cudaMemcpyAsync(alpha, h->acc, n * sizeof(double), kind, h->stream));
    }
    CK(cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (t) *t = h->st_host->t;
    if (step) *step = (long)h->st_host->step;
    return DFGKS_OK;
}

// one step of Algorithm 1 on buffers (in -> out); every kernel returns at once once st->halt is set
// rec (optional): four sweep-buffer sets, [stage][direction], that keep the stage's face-line,
// Gauss-point and flux records for the reverse sweep instead of the handle's shared buffers
static void enqueue_step(dfgks* h, int s, double dt, int flux, double t_end, int cur0, double* Wstar_store = nullptr,
                         const SweepBuffers* rec = nullptr) {
    const Mesh& m = h->mesh;
    const SchemeConsts& S = h->S;
    cudaStream_t st = h->stream;
    double* in = h->W[(cur0 + s) & 1];
    double* out = h->W[(cur0 + s + 1) & 1];
    double* ain = h->A[(cur0 + s) & 1];
    double* aout = h->A[(cur0 + s + 1) & 1];
    const int* halt = &h->st->halt;
    const double* dtp = &h->st->dt;
    KernelTimer* T = h->timer;
    if (dt <= 0.0) launch_cfl_min(m, in, S.gamma, h->st, st, T);
    launch_begin_step(h->st, h->cfg.cfl, dt, t_end, h->dts, s, st, T);
    launch_fill_ghosts(m, in, ain, halt, st, T);
    UpdateArgs a;
    memset(&a, 0, sizeof(a));
    if (h->cfg.time_scheme == DFGKS_TIME_S2O4) {
        SweepBuffers Bu[2] = {h->B, h->B};
        if (rec)
            for (int q = 0; q < 2; ++q) {
                Bu[q].flux[0] = rec[2 * q].flux[0]; Bu[q].flux_stride[0] = rec[2 * q].flux_stride[0];
                Bu[q].flux[1] = rec[2 * q + 1].flux[1]; Bu[q].flux_stride[1] = rec[2 * q + 1].flux_stride[1];
            }
        if (rec) launch_sweep_xy(m, S, flux, false, in, ain, dtp, rec[0], rec[1], h->st, halt, st, T);
        else launch_sweep_xy(m, S, flux, false, in, ain, dtp, h->B, h->By, h->st, halt, st, T);
        a.Win = in; a.Wout = h->Ws; a.acc = h->acc;
        launch_update(UM_S2O4_1, m, S, a, Bu[0], dtp, h->st, halt, st, T);
        if (Wstar_store) launch_ghosted_to_dense(m, h->Ws, 4, Wstar_store, st);
        launch_fill_ghosts(m, h->Ws, nullptr, halt, st, T);
        if (rec) launch_sweep_xy(m, S, flux, false, h->Ws, ain, dtp, rec[2], rec[3], h->st, halt, st, T);
        else launch_sweep_xy(m, S, flux, false, h->Ws, ain, dtp, h->B, h->By, h->st, halt, st, T);
        a.Win = h->Ws; a.Wout = out; a.alpha_out = aout;
        launch_update(UM_S2O4_2, m, S, a, Bu[1], dtp, h->st, halt, st, T);
    } else {
        launch_sweep_xy(m, S, flux, false, in, ain, dtp, h->B, h->By, h->st, halt, st, T);
        a.Win = in; a.Wout = h->Ws;
        launch_update(UM_RK_1, m, S, a, h->B, dtp, h->st, halt, st, T);
        launch_fill_ghosts(m, h->Ws, nullptr, halt, st, T);
        launch_sweep_xy(m, S, flux, false, h->Ws, ain, dtp, h->B, h->By, h->st, halt, st, T);
        a.Wn = in; a.Win = h->Ws; a.Wout = out;
        launch_update(UM_RK_2, m, S, a, h->B, dtp, h->st, halt, st, T);
        launch_fill_ghosts(m, out, nullptr, halt, st, T);
        launch_sweep_xy(m, S, flux, false, out, ain, dtp, h->B, h->By, h->st, halt, st, T);
        a.Wn = in; a.Win = out; a.Wout = out; a.alpha_out = aout;
        launch_update(UM_RK_3, m, S, a, h->B, dtp, h->st, halt, st, T);
    }
    if (h->cfg.alpha_source == 1) {
        // alpha^{n+1} from one more reconstruction, of W^{n+1} itself with alpha^n deciding its DF
        // branches (Alg. 1 "update DF factor" read as a pass after the stages): the alpha-only sweep
        // of alpha^0 on the new state, overwriting the last stage's product.  No counters (no flux
        // comes from it); a halted step skips it.
        launch_fill_ghosts(m, out, ain, halt, st, T);
        launch_sweep_xy(m, S, DFGKS_FLUX_LF, true, out, ain, dtp, h->B, h->By, nullptr, halt, st, T);
        UpdateArgs aa;
        memset(&aa, 0, sizeof(aa));
        aa.alpha_out = aout;
        launch_update(UM_ALPHA, m, S, aa, h->B, dtp, nullptr, halt, st, T);
    }
    launch_end_step(h->st, t_end, st, T);
}

extern "C" dfgks_status dfgks_step(dfgks* h, int n, double dt, int flux, double t_end, double* dts_out, int* steps_done) {
    if (steps_done) *steps_done = 0;
    if (!h || n < 0 || (flux != DFGKS_FLUX_GKS && flux != DFGKS_FLUX_LF)) return DFGKS_EINVAL;
    if (n == 0) return DFGKS_OK;
    ++h->gen;
    if (n > h->dts_cap) {
        cudaFree(h->dts);
        h->bytes -= (unsigned long long)h->dts_cap * sizeof(double);
        h->dts = nullptr;
        int cap = n;
        CK(dalloc(h, &h->dts, cap));
        h->dts_cap = cap;
    }
    // a new call starts clean: clear the halt and error flags left by an earlier call
    CK(cudaMemsetAsync(&h->st->halt, 0, sizeof(int), h->stream));
    CK(cudaMemsetAsync(&h->st->err, 0, sizeof(int), h->stream));
    CK(cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const long long step0 = h->st_host->step;
    const int cur0 = h->cur;
    for (int s = 0; s < n; ++s) enqueue_step(h, s, dt, flux, t_end, cur0);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->timer->harvest();
    const DevState& hs = *h->st_host;
    const long long done = hs.step - step0;
    h->cur = (int)((cur0 + done) & 1);
    if (steps_done) *steps_done = (int)done;
    if (dts_out && done > 0) CK(cudaMemcpy(dts_out, h->dts, (size_t)done * sizeof(double), cudaMemcpyDeviceToHost));
    if (hs.err) {
        h->fail_step = hs.fail_step;
        h->fail_i = (int)(hs.fail_key % (unsigned long long)h->mesh.nx);
        h->fail_j = (int)(hs.fail_key / (unsigned long long)h->mesh.nx);
        return DFGKS_ENONPOS;
    }
    return DFGKS_OK;
}

static dfgks_status run_stage_operator(dfgks* h, const double* W, const double* alpha, double dt, int flux) {
    if (!W || !alpha || !(dt > 0.0) || (flux != 0 && flux != 1)) return DFGKS_EINVAL;
    launch_dense_to_ghosted(h->mesh, W, 4, h->Ws, h->stream);
    launch_dense_to_ghosted(h->mesh, alpha, 1, h->As, h->stream);
    launch_fill_ghosts(h->mesh, h->Ws, h->As, nullptr, h->stream);
    launch_set_scalar(h->dt_scratch, dt, h->stream);
    for (int d = 0; d < 2; ++d)
        launch_sweep(d, h->mesh, h->S, flux, false, h->Ws, h->As, h->dt_scratch, h->B, nullptr, nullptr, h->stream);
    CK_LAUNCH();
    return DFGKS_OK;
}

extern "C" dfgks_status dfgks_residual(dfgks* h, const double* W, const double* alpha, double dt, int flux,
                                       double* L, double* dtL, double* dtLt, double* alpha_next) {
    if (!h) return DFGKS_EINVAL;
    dfgks_status r = run_stage_operator(h, W, alpha, dt, flux);
    if (r) return r;
    UpdateArgs a;
    memset(&a, 0, sizeof(a));
    a.L = L; a.dtL = dtL; a.dtLt = dtLt; a.alpha_out = alpha_next; a.alpha_dense = 1;
    launch_update(UM_RESIDUAL, h->mesh, h->S, a, h->B, h->dt_scratch, nullptr, nullptr, h->stream);
    CK_LAUNCH();
    return DFGKS_OK;
}

extern "C" dfgks_status dfgks_face_records(dfgks* h, const double* W, const double* alpha, double dt, int flux,
                                           int dir, double* out) {
    if (!h || !out || !W || !alpha || (dir != 0 && dir != 1) || !(dt > 0.0) || (flux != 0 && flux != 1))
        return DFGKS_EINVAL;
    // only the requested direction is swept: the Gauss-point buffer is shared by both directions
    launch_dense_to_ghosted(h->mesh, W, 4, h->Ws, h->stream);
    launch_dense_to_ghosted(h->mesh, alpha, 1, h->As, h->stream);
    launch_fill_ghosts(h->mesh, h->Ws, h->As, nullptr, h->stream);
    launch_set_scalar(h->dt_scratch, dt, h->stream);
    launch_sweep(dir, h->mesh, h->S, flux, false, h->Ws, h->As, h->dt_scratch, h->B, nullptr, nullptr, h->stream);
    launch_pack_faces(dir, h->mesh, h->B, out, h->stream);
    CK_LAUNCH();
    return DFGKS_OK;
}

static dfgks_status ensure_adjoint_buffers(dfgks* h) {
    if (h->adj_lines) return DFGKS_OK;
    CK(dalloc(h, &h->adj_lines, (long long)LR_COUNT * h->B.line_stride));
    CK(dalloc(h, &h->adj_gp, (long long)GP_COUNT * h->B.gp_stride));
    CK(dalloc(h, &h->adj_Wg, 4 * h->mesh.plane));
    return DFGKS_OK;
}

// reverse sweep of the stage operator at (W, alpha, dt); W_bar (dense, device) += J^T (L_bar, ...)
// rec (optional): the stage's forward records per direction, kept by the forward pass; without
// them each direction's forward sweep is recomputed first
static dfgks_status adjoint_stage(dfgks* h, const double* W, const double* alpha, double dt, int flux,
                                  const double* L_bar, const double* dtL_bar, const double* dtLt_bar, double* W_bar,
                                  const SweepBuffers* rec = nullptr) {
    dfgks_status r = ensure_adjoint_buffers(h);
    if (r) return r;
    launch_dense_to_ghosted(h->mesh, W, 4, h->Ws, h->stream);
    launch_dense_to_ghosted(h->mesh, alpha, 1, h->As, h->stream);
    launch_fill_ghosts(h->mesh, h->Ws, h->As, nullptr, h->stream);
    launch_set_scalar(h->dt_scratch, dt, h->stream);
    CK(cudaMemsetAsync(h->adj_Wg, 0, sizeof(double) * 4 * h->mesh.plane, h->stream));
    AdjointArgs a = {L_bar, dtL_bar, dtLt_bar};
    for (int d = 0; d < 2; ++d) {
        // the records of this direction, then its reverse sweep
        if (!rec)
            launch_sweep(d, h->mesh, h->S, flux, false, h->Ws, h->As, h->dt_scratch, h->B, nullptr, nullptr, h->stream);
        launch_adjoint_dir(d, h->mesh, h->S, flux, a, h->Ws, h->As, h->dt_scratch, rec ? rec[d] : h->B, h->adj_lines,
                           h->adj_gp, h->adj_Wg, h->stream, h->timer->on ? h->timer : nullptr);
    }
    launch_adjoint_finish(h->mesh, h->adj_Wg, W_bar, h->stream);
    CK_LAUNCH();
    return DFGKS_OK;
}

extern "C" dfgks_status dfgks_adjoint_residual(dfgks* h, const double* W, const double* alpha, double dt, int flux,
                                               const double* L_bar, const double* dtL_bar, const double* dtLt_bar,
                                               double* W_bar) {
    if (!h || !W || !alpha || !W_bar || !(dt > 0.0) || (flux != 0 && flux != 1)) return DFGKS_EINVAL;
    return adjoint_stage(h, W, alpha, dt, flux, L_bar, dtL_bar, dtLt_bar, W_bar);
}

// doubles of one step's forward records: two stages x two directions of face lines, Gauss points and
// fluxes, and (tape) the reconstructions' intermediates and, for GKS, the flux's intermediates
static long long record_doubles_per_step(const dfgks* h, bool tape, bool gks) {
    const SweepBuffers& B = h->B;
    long long per_dir = (long long)(LR_COUNT + (tape ? 8 * AT_COUNT : 0)) * B.line_stride
                      + (long long)(GP_COUNT + (tape ? 4 * AT_COUNT : 0)) * B.gp_stride;
    long long flux = (long long)(FR_COUNT + (tape && gks ? TG_COUNT : 0)) * (B.flux_stride[0] + B.flux_stride[1]);
    return 2 * (2 * per_dir + flux);
}

static void record_sets(const dfgks* h, double* base, bool tape, bool gks, SweepBuffers rec[4]) {
    const SweepBuffers& B = h->B;
    double* p = base;
    for (int q = 0; q < 4; ++q) {
        const int d = q & 1;
        rec[q] = B;
        rec[q].lines = p; p += (long long)LR_COUNT * B.line_stride;
        rec[q].gp = p; p += (long long)GP_COUNT * B.gp_stride;
        rec[q].flux[0] = rec[q].flux[1] = nullptr;
        rec[q].flux[d] = p; p += (long long)FR_COUNT * B.flux_stride[d];
        rec[q].tape[0] = rec[q].tape[1] = nullptr;
        rec[q].ltape = rec[q].ftape = nullptr;
        if (tape) {
            rec[q].ltape = p; p += (long long)8 * AT_COUNT * B.line_stride;
            rec[q].ftape = p; p += (long long)4 * AT_COUNT * B.gp_stride;
            if (gks) { rec[q].tape[d] = p; p += (long long)TG_COUNT * B.flux_stride[d]; }
        }
    }
}

// Lay out (and allocate if needed) the segment arena for k steps: W^s, alpha^s, W* per step and,
// if they fit in half of the free device memory, the sweep records (with the reconstruction and GKS
// flux tapes when those fit too).
struct SegArena { double* W; double* A; double* Ws; double* recs; bool tape, gks; long long rec_step; };

// doubles of one segment slot: W^s, alpha^s, W* of k steps and, when kept, their records
static long long slot_doubles(const dfgks* h, int k, bool records, bool tape, bool gks) {
    const long long N = (long long)h->mesh.nx * h->mesh.ny;
    return (long long)k * (9 * N) + (records ? (long long)k * record_doubles_per_step(h, tape, gks) : 0);
}

// slot `slot` of the arena in the layout last decided (seg_k, seg_records, seg_tape, seg_gks)
static void arena_view(const dfgks* h, SegArena& a, int slot = 0) {
    const long long N = (long long)h->mesh.nx * h->mesh.ny, N4 = 4 * N;
    const int k = h->seg_k;
    a.W = h->seg_arena + (long long)slot * slot_doubles(h, k, h->seg_records != 0, h->seg_tape != 0, h->seg_gks != 0);
    a.A = a.W + (long long)k * N4;
    a.Ws = a.A + (long long)k * N;
    a.recs = h->seg_records ? a.Ws + (long long)k * N4 : nullptr;
    a.tape = h->seg_tape != 0; a.gks = h->seg_gks != 0;
    a.rec_step = record_doubles_per_step(h, a.tape, a.gks);
}

// Lay out the arena for segments of k steps: the records (with tapes if they fit) of as many as
// `want` segments within 60 % of the free device memory, at least one slot.  The forward pass
// keeps its last segments there, so the reverse pass recomputes only the ones that did not fit.
static dfgks_status ensure_segment_arena(dfgks* h, int k, int flux, int want, SegArena& a) {
    const bool gks = flux == DFGKS_FLUX_GKS;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const double budget = 0.6 * ((double)free_b + (double)h->seg_cap * sizeof(double));
    int records = 1;
    bool tape = true;
    if ((double)slot_doubles(h, k, true, true, gks) * sizeof(double) > budget) tape = false;
    if ((double)slot_doubles(h, k, true, false, gks) * sizeof(double) > budget) records = 0;
    const long long per = slot_doubles(h, k, records, tape, gks);
    int slots = (int)(budget / ((double)per * sizeof(double)));
    if (slots > want) slots = want;
    if (slots < 1) slots = 1;
    const long long need = (long long)slots * per;
    if (need > h->seg_cap) {
        if (h->seg_arena) { cudaFree(h->seg_arena); h->bytes -= (unsigned long long)h->seg_cap * sizeof(double); }
        h->seg_arena = nullptr;
        h->seg_cap = 0;
        if (dalloc(h, &h->seg_arena, need) != cudaSuccess) {
            cudaGetLastError();
            slots = 1;
            const long long one = slot_doubles(h, k, false, false, gks);
            if (dalloc(h, &h->seg_arena, one) != cudaSuccess) { cudaGetLastError(); return DFGKS_ENOMEM; }
            records = 0;
            tape = false;
            h->seg_cap = one;
        } else {
            h->seg_cap = need;
        }
    } else {
        slots = (int)(h->seg_cap / per);
        if (slots > want) slots = want;
    }
    h->seg_k = k; h->seg_records = records; h->seg_tape = tape; h->seg_gks = gks; h->seg_slots = slots;
    arena_view(h, a, 0);
    return DFGKS_OK;
}

// Forward pass from W0 (alpha^0 from W0) over n S2O4 steps, dt from dts_in or, if that is NULL, the
// CFL rule; W and alpha are kept every k steps and the dts on the host, for the reverse pass.
static dfgks_status forward_checkpointed(dfgks* h, const double* W0, int n, const double* dts_in, int k, int flux) {
    const Mesh& m = h->mesh;
    const long long N = (long long)m.nx * m.ny, N4 = 4 * N;
    const int nseg = (n + k - 1) / k;
    h->ck_gen = 0;
    if (nseg > h->ck_cap) {
        if (h->ck_W) { cudaFree(h->ck_W); h->bytes -= (unsigned long long)h->ck_cap * N4 * sizeof(double); h->ck_W = nullptr; }
        if (h->ck_A) { cudaFree(h->ck_A); h->bytes -= (unsigned long long)h->ck_cap * N * sizeof(double); h->ck_A = nullptr; }
        h->ck_cap = 0;
        CK(dalloc(h, &h->ck_W, (long long)nseg * N4));
        CK(dalloc(h, &h->ck_A, (long long)nseg * N));
        h->ck_cap = nseg;
    }
    if (n > h->ck_dts_cap) {
        double* p = (double*)realloc(h->ck_dts, (size_t)n * sizeof(double));
        if (!p) return DFGKS_ENOMEM;
        h->ck_dts = p;
        h->ck_dts_cap = n;
    }
    if (n > h->dts_cap) {
        cudaFree(h->dts);
        h->bytes -= (unsigned long long)h->dts_cap * sizeof(double);
        h->dts = nullptr;
        CK(dalloc(h, &h->dts, n));
        h->dts_cap = n;
    }
    SegArena a;
    h->seg_kept = 0;
    dfgks_status r = ensure_segment_arena(h, k, flux, nseg, a);
    if (r) return r;
    r = load_state(h, W0, nullptr, 0.0, 0, 1);
    if (r) return r;
    const int cur0 = h->cur;
    // the last `kept` segments fill the arena's slots as they run (segment nseg - kept in slot 0)
    const int kept = h->seg_slots < nseg ? h->seg_slots : nseg;
    const int first_kept = nseg - kept;
    for (int s = 0; s < n; ++s) {
        const int c = (cur0 + s) & 1;
        if (s % k == 0) {
            launch_ghosted_to_dense(m, h->W[c], 4, h->ck_W + (long long)(s / k) * N4, h->stream);
            launch_ghosted_to_dense(m, h->A[c], 1, h->ck_A + (long long)(s / k) * N, h->stream);
        }
        if (s / k >= first_kept) {
            arena_view(h, a, s / k - first_kept);
            const int j = s % k;
            launch_ghosted_to_dense(m, h->W[c], 4, a.W + (long long)j * N4, h->stream);
            launch_ghosted_to_dense(m, h->A[c], 1, a.A + (long long)j * N, h->stream);
            SweepBuffers rec[4];
            if (a.recs) record_sets(h, a.recs + (long long)j * a.rec_step, a.tape, a.gks, rec);
            enqueue_step(h, s, dts_in ? dts_in[s] : 0.0, flux, 0.0, cur0, a.Ws + (long long)j * N4,
                         a.recs ? rec : nullptr);
        } else {
            enqueue_step(h, s, dts_in ? dts_in[s] : 0.0, flux, 0.0, cur0);
        }
    }
    CK_LAUNCH();
    CK(cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->timer->harvest();
    const long long done = h->st_host->step;
    h->cur = (int)((cur0 + done) & 1);
    if (h->st_host->err || done != n) return DFGKS_ENONPOS;
    CK(cudaMemcpy(h->ck_dts, h->dts, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost));
    h->ck_n = n; h->ck_k = k; h->ck_flux = flux;
    h->seg_kept = kept;
    h->ck_gen = ++h->gen;
    return DFGKS_OK;
}

// Reverse pass over the checkpointed forward pass: dJ/dW0 = (dW^n/dW0)^T WT_bar.  Each segment of
// k steps is recomputed from its checkpoint (the last one only if the forward pass could not keep
// it), keeping W^s, alpha^s, W* and, if they fit in the memory budget, every stage's forward records;
// then its steps are reversed (Eq. 24 with the time limiter):  W* = W + dt/2 L + dt^2/8 dL,  W' = W + dt L + dt^2/2 dL - dt^2/3 dLt + dt^2/3 dLt(W*).
static dfgks_status backward_checkpointed(dfgks* h, const double* WT_bar, double* W0_bar) {
    const Mesh& m = h->mesh;
    const long long N = (long long)m.nx * m.ny, N4 = 4 * N;
    const int n = h->ck_n, k = h->ck_k, flux = h->ck_flux, nseg = (n + k - 1) / k;
    const double* dts = h->ck_dts;
    // the last segments' states and records are still in the arena if the forward pass kept them
    const int kept = (h->seg_arena && h->seg_k == k && h->seg_gks == (flux == DFGKS_FLUX_GKS)) ? h->seg_kept : 0;
    h->seg_kept = 0;                            // the recompute below overwrites the arena
    const int first_kept = nseg - kept;
    SegArena a;
    dfgks_status r = DFGKS_OK;
    if (kept) arena_view(h, a, 0);              // the layout the forward pass wrote
    else r = ensure_segment_arena(h, k, flux, 1, a);
    if (r) return r;
    std::vector<double*> bufs;
    auto get = [&](long long cnt) -> double* {
        double* p = nullptr;
        if (cudaMalloc((void**)&p, (size_t)cnt * sizeof(double)) != cudaSuccess) return nullptr;
        bufs.push_back(p);
        return p;
    };
    double* Wb = get(N4);
    double* Wsb = get(N4);
    double* bL = get(N4);
    double* bdL = get(N4);
    double* bdLt = get(N4);
    double* WTs = get(N4);
    double* ATs = get(N);
    if (bufs.size() != 7) r = DFGKS_ENOMEM;
    auto cleanup = [&]() { cudaStreamSynchronize(h->stream); for (double* p : bufs) if (p) cudaFree(p); };
    if (r) { cleanup(); return r; }
    r = ensure_adjoint_buffers(h);
    if (r) { cleanup(); return r; }
    // the passes; a CUDA error returns from this lambda, and the scratch is freed either way
    auto passes = [&]() -> dfgks_status {
        CK(cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        const DevState stT = *h->st_host;
        launch_ghosted_to_dense(m, h->W[h->cur], 4, WTs, h->stream);
        launch_ghosted_to_dense(m, h->A[h->cur], 1, ATs, h->stream);
        CK(cudaMemcpyAsync(Wb, WT_bar, (size_t)N4 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        for (int seg = nseg - 1; seg >= 0 && r == DFGKS_OK; --seg) {
            const int s0 = seg * k, s1 = (s0 + k < n) ? s0 + k : n;
            // a kept segment sits in its slot; the others are recomputed into slot 0, which the
            // kept segments (all later than any recomputed one) have already been reversed out of
            arena_view(h, a, seg >= first_kept ? seg - first_kept : 0);
            if (seg < first_kept) {
                // recompute the segment from its checkpoint, keeping W^s, alpha^s, W* and the records
                launch_dense_to_ghosted(m, h->ck_W + (long long)seg * N4, 4, h->W[h->cur], h->stream);
                launch_dense_to_ghosted(m, h->ck_A + (long long)seg * N, 1, h->A[h->cur], h->stream);
                for (int s = s0; s < s1; ++s) {
                    launch_ghosted_to_dense(m, h->W[h->cur], 4, a.W + (s - s0) * N4, h->stream);
                    launch_ghosted_to_dense(m, h->A[h->cur], 1, a.A + (s - s0) * N, h->stream);
                    SweepBuffers rec[4];
                    if (a.recs) record_sets(h, a.recs + (long long)(s - s0) * a.rec_step, a.tape, a.gks, rec);
                    enqueue_step(h, 0, dts[s], flux, 0.0, h->cur, a.Ws + (s - s0) * N4, a.recs ? rec : nullptr);
                    h->cur ^= 1;
                }
            }
            // reverse through the segment: Eq. 24 with the time limiter,
            //   W* = W + dt/2 L + dt^2/8 dL,  W' = W + dt L + dt^2/2 dL - dt^2/3 dLt + dt^2/3 dLt(W*)
            for (int s = s1 - 1; s >= s0 && r == DFGKS_OK; --s) {
                const double dt = dts[s], dt2 = dt * dt;
                const double* Wn = a.W + (s - s0) * N4;
                const double* An = a.A + (s - s0) * N;
                const double* Wst = a.Ws + (s - s0) * N4;
                SweepBuffers rec[4];
                if (a.recs) record_sets(h, a.recs + (long long)(s - s0) * a.rec_step, a.tape, a.gks, rec);
                CK(cudaMemsetAsync(Wsb, 0, (size_t)N4 * sizeof(double), h->stream));
                launch_axpby(N4, dt2 / 3.0, Wb, 0.0, bdLt, h->stream);
                r = adjoint_stage(h, Wst, An, dt, flux, nullptr, nullptr, bdLt, Wsb, a.recs ? rec + 2 : nullptr);
                if (r) break;
                launch_axpby(N4, dt, Wb, 0.0, bL, h->stream);
                launch_axpby(N4, 0.5 * dt, Wsb, 1.0, bL, h->stream);
                launch_axpby(N4, 0.5 * dt2, Wb, 0.0, bdL, h->stream);
                launch_axpby(N4, 0.125 * dt2, Wsb, 1.0, bdL, h->stream);
                launch_axpby(N4, -dt2 / 3.0, Wb, 0.0, bdLt, h->stream);
                launch_axpby(N4, 1.0, Wsb, 1.0, Wb, h->stream);
                r = adjoint_stage(h, Wn, An, dt, flux, bL, bdL, bdLt, Wb, a.recs ? rec : nullptr);
            }
        }
        if (r == DFGKS_OK) CK(cudaMemcpyAsync(W0_bar, Wb, (size_t)N4 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        // leave the handle at the forward solution W^n (state, alpha, time and step count)
        launch_dense_to_ghosted(m, WTs, 4, h->W[h->cur], h->stream);
        launch_dense_to_ghosted(m, ATs, 1, h->A[h->cur], h->stream);
        *h->st_host = stT;
        CK(cudaMemcpyAsync(h->st, h->st_host, sizeof(DevState), cudaMemcpyHostToDevice, h->stream));
        CK_LAUNCH();
        return r;
    };
    r = passes();
    cleanup();
    h->timer->harvest();
    return r;
}

extern "C" dfgks_status dfgks_forward_checkpointed(dfgks* h, const double* W0, int n, const double* dts_in, int flux,
                                                   int ckpt_every, double* dts_out) {
    if (!h || !W0 || n < 1 || ckpt_every < 1 || (flux != 0 && flux != 1)) return DFGKS_EINVAL;
    if (h->cfg.time_scheme != DFGKS_TIME_S2O4) return DFGKS_ENOTSUP;
    if (h->cfg.alpha_source != 0) return DFGKS_ENOTSUP;    // the recompute's extra DF pass is not covered
    if (dts_in) for (int s = 0; s < n; ++s) if (!(dts_in[s] > 0.0)) return DFGKS_EINVAL;
    const int k = ckpt_every < n ? ckpt_every : n;
    dfgks_status r = forward_checkpointed(h, W0, n, dts_in, k, flux);
    if (r == DFGKS_OK && dts_out) memcpy(dts_out, h->ck_dts, (size_t)n * sizeof(double));
    return r;
}

extern "C" dfgks_status dfgks_adjoint_checkpointed(dfgks* h, const double* WT_bar, double* W0_bar) {
    if (!h || !WT_bar || !W0_bar) return DFGKS_EINVAL;
    if (h->ck_gen == 0 || h->ck_gen != h->gen) return DFGKS_EINVAL;     // no forward pass, or the state changed since
    return backward_checkpointed(h, WT_bar, W0_bar);
}

extern "C" dfgks_status dfgks_adjoint_steps(dfgks* h, const double* W0, int n, const double* dts, int flux, int ckpt_every,
                                            const double* WT_bar, double* W0_bar) {
    if (!h || !W0 || !dts || !WT_bar || !W0_bar || n < 1 || ckpt_every < 1 || (flux != 0 && flux != 1))
        return DFGKS_EINVAL;
    dfgks_status r = dfgks_forward_checkpointed(h, W0, n, dts, flux, ckpt_every, nullptr);
    if (r) return r;
    return backward_checkpointed(h, WT_bar, W0_bar);
}

extern "C" dfgks_status dfgks_get_counters(dfgks* h, dfgks_counters* out) {
    if (!h || !out) return DFGKS_EINVAL;
    CK(cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    out->fallbacks = h->st_host->fallbacks;
    out->df_normal = h->st_host->df_normal;
    out->df_tangential = h->st_host->df_tangential;
    return DFGKS_OK;
}

extern "C" dfgks_status dfgks_last_error_detail(dfgks* h, long* step, int* i, int* j) {
    if (!h) return DFGKS_EINVAL;
    if (step) *step = (long)h->fail_step;
    if (i) *i = h->fail_i;
    if (j) *j = h->fail_j;
    return DFGKS_OK;
}

extern "C" dfgks_status dfgks_device_bytes(dfgks* h, unsigned long long* bytes) {
    if (!h || !bytes) return DFGKS_EINVAL;
    *bytes = h->bytes;
    return DFGKS_OK;
}

extern "C" dfgks_status dfgks_set_timing(dfgks* h, int enable) {
    if (!h) return DFGKS_EINVAL;
    KernelTimer* T = h->timer;
    CK(cudaStreamSynchronize(h->stream));
    T->harvest();
    if (enable && T->ev.empty()) {
        const int slots = 4096;
        T->ev.resize(2 * slots);
        T->kind.resize(slots);
        for (auto& e : T->ev) CK(cudaEventCreate(&e));
    }
    T->on = enable != 0;
    return DFGKS_OK;
}

extern "C" dfgks_status dfgks_get_timing(dfgks* h, double* total_ms, long long* timed, long long* launches, int reset) {
    if (!h) return DFGKS_EINVAL;
    KernelTimer* T = h->timer;
    CK(cudaStreamSynchronize(h->stream));
    T->harvest();
    for (int k = 0; k < KK_COUNT; ++k) {
        if (total_ms) total_ms[k] = T->total_ms[k];
        if (timed) timed[k] = T->timed[k];
        if (launches) launches[k] = T->launches[k];
        if (reset) { T->total_ms[k] = 0.0; T->timed[k] = 0; T->launches[k] = 0; }
    }
    return DFGKS_OK;
}
