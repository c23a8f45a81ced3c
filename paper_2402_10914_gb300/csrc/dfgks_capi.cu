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
    if (c->bc_xlo == 0 && c->nx < G) return false;
    if (c->bc_ylo == 0 && c->ny < G) return false;
    if (c->time_scheme != 0 && c->time_scheme != 1) return false;
    if (c->tau_reading != 0 && c->tau_reading != 1) return false;
    return true;
}

static void free_all(dfgks* h) {
    double* ptrs[] = {h->W[0], h->W[1], h->A[0], h->A[1], h->Ws, h->As, h->acc, h->B.lines, h->B.gp,
                      h->B.flux[0], h->B.flux[1], h->dt_scratch, h->dts, h->adj_lines, h->adj_gp, h->adj_Wg};
    for (double* p : ptrs) if (p) cudaFree(p);
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
    m.bc[0] = cfg->bc_xlo; m.bc[1] = cfg->bc_xhi; m.bc[2] = cfg->bc_ylo; m.bc[3] = cfg->bc_yhi;
    SchemeConsts& S = h->S;
    S.gamma = cfg->gamma; S.gm1 = cfg->gamma - 1.0; S.K = (4.0 - 2.0 * cfg->gamma) / (cfg->gamma - 1.0);
    S.inv_K2 = 1.0 / (S.K + 2.0);
    S.d[3] = cfg->dH;
    S.d[0] = (1.0 - cfg->dH) * (1.0 - cfg->dL) / 2.0;
    S.d[1] = (1.0 - cfg->dH) * cfg->dL;
    S.d[2] = S.d[0];
    S.inv_d3 = 1.0 / cfg->dH;
    S.eps = cfg->eps; S.alpha_thres = cfg->alpha_thres; S.C1 = cfg->C1; S.C2 = cfg->C2;
    S.time_limiter = cfg->time_limiter; S.tau_reading = cfg->tau_reading; S.gp_fallback = cfg->gp_fallback;

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
    for (int dir = 0; dir < 2; ++dir)
        launch_sweep(dir, h->mesh, h->S, 1, true, Wg, Ag, h->dt_scratch, h->B, nullptr, nullptr, h->stream);
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
static void enqueue_step(dfgks* h, int s, double dt, int flux, double t_end, int cur0, double* Wstar_store = nullptr) {
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
        for (int d = 0; d < 2; ++d) launch_sweep(d, m, S, flux, false, in, ain, dtp, h->B, h->st, halt, st, T);
        a.Win = in; a.Wout = h->Ws; a.acc = h->acc;
        launch_update(UM_S2O4_1, m, S, a, h->B, dtp, h->st, halt, st, T);
        if (Wstar_store) launch_ghosted_to_dense(m, h->Ws, 4, Wstar_store, st);
        launch_fill_ghosts(m, h->Ws, nullptr, halt, st, T);
        for (int d = 0; d < 2; ++d) launch_sweep(d, m, S, flux, false, h->Ws, ain, dtp, h->B, h->st, halt, st, T);
        a.Win = h->Ws; a.Wout = out; a.alpha_out = aout;
        launch_update(UM_S2O4_2, m, S, a, h->B, dtp, h->st, halt, st, T);
    } else {
        for (int d = 0; d < 2; ++d) launch_sweep(d, m, S, flux, false, in, ain, dtp, h->B, h->st, halt, st, T);
        a.Win = in; a.Wout = h->Ws;
        launch_update(UM_RK_1, m, S, a, h->B, dtp, h->st, halt, st, T);
        launch_fill_ghosts(m, h->Ws, nullptr, halt, st, T);
        for (int d = 0; d < 2; ++d) launch_sweep(d, m, S, flux, false, h->Ws, ain, dtp, h->B, h->st, halt, st, T);
        a.Wn = in; a.Win = h->Ws; a.Wout = out;
        launch_update(UM_RK_2, m, S, a, h->B, dtp, h->st, halt, st, T);
        launch_fill_ghosts(m, out, nullptr, halt, st, T);
        for (int d = 0; d < 2; ++d) launch_sweep(d, m, S, flux, false, out, ain, dtp, h->B, h->st, halt, st, T);
        a.Wn = in; a.Win = out; a.Wout = out; a.alpha_out = aout;
        launch_update(UM_RK_3, m, S, a, h->B, dtp, h->st, halt, st, T);
    }
    launch_end_step(h->st, t_end, st, T);
}

extern "C" dfgks_status dfgks_step(dfgks* h, int n, double dt, int flux, double t_end, double* dts_out, int* steps_done) {
    if (steps_done) *steps_done = 0;
    if (!h || n < 0 || (flux != DFGKS_FLUX_GKS && flux != DFGKS_FLUX_LF)) return DFGKS_EINVAL;
    if (n == 0) return DFGKS_OK;
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
static dfgks_status adjoint_stage(dfgks* h, const double* W, const double* alpha, double dt, int flux,
                                  const double* L_bar, const double* dtL_bar, const double* dtLt_bar, double* W_bar) {
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
        launch_sweep(d, h->mesh, h->S, flux, false, h->Ws, h->As, h->dt_scratch, h->B, nullptr, nullptr, h->stream);
        launch_adjoint_dir(d, h->mesh, h->S, flux, a, h->Ws, h->As, h->dt_scratch, h->B, h->adj_lines, h->adj_gp,
                           h->adj_Wg, h->stream, h->timer->on ? h->timer : nullptr);
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

extern "C" dfgks_status dfgks_adjoint_steps(dfgks* h, const double* W0, int n, const double* dts, int flux, int ckpt_every,
                                            const double* WT_bar, double* W0_bar) {
    if (!h || !W0 || !dts || !WT_bar || !W0_bar || n < 1 || ckpt_every < 1 || (flux != 0 && flux != 1))
        return DFGKS_EINVAL;
    if (h->cfg.time_scheme != DFGKS_TIME_S2O4) return DFGKS_ENOTSUP;
    for (int s = 0; s < n; ++s) if (!(dts[s] > 0.0)) return DFGKS_EINVAL;
    const Mesh& m = h->mesh;
    const long long N = (long long)m.nx * m.ny, N4 = 4 * N;
    const int k = ckpt_every < n ? ckpt_every : n, nseg = (n + k - 1) / k;
    std::vector<double*> bufs;
    auto get = [&](long long cnt) -> double* {
        double* p = nullptr;
        if (cudaMalloc((void**)&p, (size_t)cnt * sizeof(double)) != cudaSuccess) return nullptr;
        bufs.push_back(p);
        return p;
    };
    double* ckW = get(nseg * N4);
    double* ckA = get(nseg * N);
    double* segW = get(k * N4);
    double* segA = get(k * N);
    double* segWs = get(k * N4);
    double* Wb = get(N4);
    double* Wsb = get(N4);
    double* bL = get(N4);
    double* bdL = get(N4);
    double* bdLt = get(N4);
    double* WTs = get(N4);
    double* ATs = get(N);
    dfgks_status r = DFGKS_OK;
    for (double* p : bufs) if (!p) r = DFGKS_ENOMEM;
    if (bufs.size() != 12) r = DFGKS_ENOMEM;
    auto cleanup = [&]() { cudaStreamSynchronize(h->stream); for (double* p : bufs) cudaFree(p); };
    if (r) { cleanup(); return r; }
    // forward pass from W0 with the recorded steps, keeping a checkpoint every k steps
    r = load_state(h, W0, nullptr, 0.0, 0, 1);
    if (r) { cleanup(); return r; }
    CK(cudaMemsetAsync(&h->st->halt, 0, sizeof(int), h->stream));
    auto one_step = [&](double dt, double* Wstar) {
        enqueue_step(h, 0, dt, flux, 0.0, h->cur, Wstar);
        h->cur ^= 1;
    };
    for (int s = 0; s < n; ++s) {
        if (s % k == 0) {
            launch_ghosted_to_dense(m, h->W[h->cur], 4, ckW + (s / k) * N4, h->stream);
            launch_ghosted_to_dense(m, h->A[h->cur], 1, ckA + (s / k) * N, h->stream);
        }
        one_step(dts[s], nullptr);
    }
    CK(cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (h->st_host->err) { cleanup(); return DFGKS_ENONPOS; }
    const DevState stT = *h->st_host;
    launch_ghosted_to_dense(m, h->W[h->cur], 4, WTs, h->stream);
    launch_ghosted_to_dense(m, h->A[h->cur], 1, ATs, h->stream);
    CK(cudaMemcpyAsync(Wb, WT_bar, (size_t)N4 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    for (int seg = nseg - 1; seg >= 0 && r == DFGKS_OK; --seg) {
        const int s0 = seg * k, s1 = (s0 + k < n) ? s0 + k : n;
        // recompute the segment from its checkpoint, keeping W^s, alpha^s and W* of every step
        launch_dense_to_ghosted(m, ckW + seg * N4, 4, h->W[h->cur], h->stream);
        launch_dense_to_ghosted(m, ckA + seg * N, 1, h->A[h->cur], h->stream);
        for (int s = s0; s < s1; ++s) {
            launch_ghosted_to_dense(m, h->W[h->cur], 4, segW + (s - s0) * N4, h->stream);
            launch_ghosted_to_dense(m, h->A[h->cur], 1, segA + (s - s0) * N, h->stream);
            one_step(dts[s], segWs + (s - s0) * N4);
        }
        // reverse through the segment: Eq. 24 with the time limiter,
        //   W* = W + dt/2 L + dt^2/8 dL,  W' = W + dt L + dt^2/2 dL - dt^2/3 dLt + dt^2/3 dLt(W*)
        for (int s = s1 - 1; s >= s0 && r == DFGKS_OK; --s) {
            const double dt = dts[s], dt2 = dt * dt;
            const double* Wn = segW + (s - s0) * N4;
            const double* An = segA + (s - s0) * N;
            const double* Wst = segWs + (s - s0) * N4;
            CK(cudaMemsetAsync(Wsb, 0, (size_t)N4 * sizeof(double), h->stream));
            launch_axpby(N4, dt2 / 3.0, Wb, 0.0, bdLt, h->stream);
            r = adjoint_stage(h, Wst, An, dt, flux, nullptr, nullptr, bdLt, Wsb);
            if (r) break;
            launch_axpby(N4, dt, Wb, 0.0, bL, h->stream);
            launch_axpby(N4, 0.5 * dt, Wsb, 1.0, bL, h->stream);
            launch_axpby(N4, 0.5 * dt2, Wb, 0.0, bdL, h->stream);
            launch_axpby(N4, 0.125 * dt2, Wsb, 1.0, bdL, h->stream);
            launch_axpby(N4, -dt2 / 3.0, Wb, 0.0, bdLt, h->stream);
            launch_axpby(N4, 1.0, Wsb, 1.0, Wb, h->stream);
            r = adjoint_stage(h, Wn, An, dt, flux, bL, bdL, bdLt, Wb);
        }
    }
    if (r == DFGKS_OK) CK(cudaMemcpyAsync(W0_bar, Wb, (size_t)N4 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    // leave the handle at the forward solution W^n (state, alpha, time and step count)
    launch_dense_to_ghosted(m, WTs, 4, h->W[h->cur], h->stream);
    launch_dense_to_ghosted(m, ATs, 1, h->A[h->cur], h->stream);
    *h->st_host = stT;
    CK(cudaMemcpyAsync(h->st, h->st_host, sizeof(DevState), cudaMemcpyHostToDevice, h->stream));
    cleanup();
    CK_LAUNCH();
    return r;
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
