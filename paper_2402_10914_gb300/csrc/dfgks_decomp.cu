// dfgks_decomp.cu -- one problem split into px x py rectangular blocks with halo exchange.
//
// Each block is a ghosted mesh of its own (buffers, sweeps and update as for a whole mesh); the
// ghost layers of a side it shares with another block (or of a periodic side that wraps onto
// another block) are filled by copies of that block's boundary cells instead of by a boundary
// condition.  Before every stage the ghost fill runs as two passes over all blocks, as on the
// whole mesh: (1) the ghost columns of the interior rows (physical sides by their boundary
// condition, shared sides by copying the neighbour's G boundary columns), then (2) the ghost
// rows of all columns, ghost columns included (physical sides by their boundary condition, which
// reads the columns of pass 1; shared sides by copying the neighbour's G boundary rows with its
// ghost columns).  Pass 2 carries the diagonal neighbours' cells into the corners, so no
// diagonal exchange is needed.  Every ghost cell then holds what the whole mesh's fill puts
// there, the per-cell arithmetic is the same, and a decomposed run reproduces the undivided one
// bit for bit.  All blocks share one device step state: the CFL kernels of all blocks take their
// minimum into it (the dt all-reduce of a multi-device run), and one halt flag stops them all.
//
// On one device the copies are device-to-device; the block plan (dfgks_decomp_plan) is the same
// bookkeeping a run with one block per device would use, where the copies become sends and
// receives of the same strips.
#include <cuda_runtime.h>
#include <string.h>
#include <new>
#include <vector>

#include "../../include/dfgks.h"
#include "dfgks_internal.h"

using namespace dfk;

namespace {

struct Block {
    dfgks_block_plan plan;
    Mesh m;
    double* W[2];
    double* A[2];
    double* Ws;
    double* acc;          // dense [4][ny][nx]: S2O4 accumulator and transfer staging
    SweepBuffers B;       // x-faces' records and both flux record sets
    SweepBuffers By;      // y-faces' face-line and Gauss-point records (fused x/y sweeps)
};

long long round4(long long n) { return (n + 3) & ~3LL; }
int split(int n, int parts, int k) { return (int)(((long long)n * k) / parts); }

bool decomp_config_ok(const dfgks_config* c, int px, int py) {
    if (!c || px < 1 || py < 1 || px > 4096 || py > 4096) return false;
    if (c->nx < 1 || c->ny < 1 || c->nx > (1 << 20) || c->ny > (1 << 20)) return false;
    if (!(c->x1 > c->x0) || !(c->y1 > c->y0) || !(c->gamma > 1.0) || !(c->cfl > 0.0) || !(c->eps > 0.0)) return false;
    if (!(c->dH > 0.0 && c->dH <= 1.0) || !(c->dL >= 0.0 && c->dL <= 1.0) || !(c->C1 >= 0.0) || !(c->C2 >= 0.0)) return false;
    const int bcs[4] = {c->bc_xlo, c->bc_xhi, c->bc_ylo, c->bc_yhi};
    for (int k = 0; k < 4; ++k) if (bcs[k] < 0 || bcs[k] > 2) return false;
    if ((c->bc_xlo == 0) != (c->bc_xhi == 0) || (c->bc_ylo == 0) != (c->bc_yhi == 0)) return false;
    // a halo copy takes G boundary cells of the neighbour, and periodic or walled sides copy or
    // mirror G cells of the block itself: every block needs G cells along a split direction,
    // an unsplit direction the whole mesh's rule
    if (px > 1 && c->nx / px < G) return false;
    if (py > 1 && c->ny / py < G) return false;
    if (px == 1 && (c->bc_xlo != 1 || c->bc_xhi != 1) && c->nx < G) return false;
    if (py == 1 && (c->bc_ylo != 1 || c->bc_yhi != 1) && c->ny < G) return false;
    if (c->time_scheme != DFGKS_TIME_S2O4) return false;
    return (c->tau_reading == 0 || c->tau_reading == 1) && (c->dt_rule == 0 || c->dt_rule == 1)
        && (c->df_states == 0 || c->df_states == 1) && c->alpha_source == 0;
}

void make_plan(const dfgks_config* c, int px, int py, int b, dfgks_block_plan* p) {
    const int bx = b % px, by = b / px;
    p->i0 = split(c->nx, px, bx); p->i1 = split(c->nx, px, bx + 1);
    p->j0 = split(c->ny, py, by); p->j1 = split(c->ny, py, by + 1);
    const int bc[4] = {c->bc_xlo, c->bc_xhi, c->bc_ylo, c->bc_yhi};
    // x-low, x-high, y-low, y-high: an inner side, or a periodic side of a split direction, is
    // shared with the neighbouring block; otherwise the side keeps the mesh's boundary condition
    const bool inner[4] = {bx > 0, bx < px - 1, by > 0, by < py - 1};
    const int wrap[4] = {by * px + px - 1, by * px, (py - 1) * px + bx, bx};
    const int next[4] = {b - 1, b + 1, b - px, b + px};
    const bool split_dir[4] = {px > 1, px > 1, py > 1, py > 1};
    for (int s = 0; s < 4; ++s) {
        if (inner[s]) { p->bc[s] = BC_EXTERNAL; p->neighbour[s] = next[s]; }
        else if (bc[s] == DFGKS_BC_PERIODIC && split_dir[s]) { p->bc[s] = BC_EXTERNAL; p->neighbour[s] = wrap[s]; }
        else { p->bc[s] = bc[s]; p->neighbour[s] = -1; }
    }
}

}  // namespace

struct dfgks_decomp {
    dfgks_config cfg;
    int px, py;
    cudaStream_t stream;
    bool own_stream;
    SchemeConsts S;
    std::vector<Block> blk;
    DevState* st;            // shared by all blocks
    DevState* st_host;
    int* flag;
    int* flag_host;
    double* dts;             // device dt history of one step call
    int dts_cap;
    double* one;             // device scalar 1.0 (the alpha^0 pass)
    double* stage;           // dense [4][ny][nx] of the whole mesh: transfers
    int cur;
    std::vector<void*> allocs;
};

static dfgks_status dstat(cudaError_t e) {
    return e == cudaSuccess ? DFGKS_OK : (e == cudaErrorMemoryAllocation ? DFGKS_ENOMEM : DFGKS_ECUDA);
}
#define DCK(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) return dstat(e_); } while (0)

template <class T>
static cudaError_t dalloc(dfgks_decomp* d, T** p, long long n) {
    cudaError_t e = cudaMalloc((void**)p, (size_t)n * sizeof(T));
    if (e == cudaSuccess) d->allocs.push_back((void*)*p);
    return e;
}

static void free_decomp(dfgks_decomp* d) {
    for (void* p : d->allocs) cudaFree(p);
    if (d->st_host) cudaFreeHost(d->st_host);
    if (d->flag_host) cudaFreeHost(d->flag_host);
    if (d->own_stream && d->stream) cudaStreamDestroy(d->stream);
}

// copy a width x height window (doubles x rows) of ncomp planes between two ghosted fields
static cudaError_t copy_window(const Block& dst, double* dfield, int di, int dj, const Block& src,
                               const double* sfield, int si, int sj, int width, int height, int ncomp,
                               cudaStream_t s) {
    for (int k = 0; k < ncomp; ++k) {
        cudaError_t e = cudaMemcpy2DAsync(dfield + k * dst.m.plane + gid(dst.m, di, dj), (size_t)dst.m.P * sizeof(double),
                                          sfield + k * src.m.plane + gid(src.m, si, sj), (size_t)src.m.P * sizeof(double),
                                          (size_t)width * sizeof(double), (size_t)height, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The halo copy of side `side` of block b from its neighbour a: the window of b's ghosted field
// it fills ((di, dj), w x h cells) and where that window starts in a's field ((si, sj)).  Pass 0
// (x sides): the ghost columns of the interior rows from a's G boundary columns; pass 1 (y sides):
// the ghost rows, ghost columns included, from a's G boundary rows (with a's ghost columns, so the
// diagonal neighbour's cells reach the corners).
static void halo_window(const dfgks_block_plan& b, const dfgks_block_plan& a, int side, dfgks_halo_window* w) {
    const int bnx = b.i1 - b.i0, bny = b.j1 - b.j0, anx = a.i1 - a.i0, any = a.j1 - a.j0;
    if (side < 2) {
        w->w = G; w->h = bny; w->dj = 0; w->sj = 0;
        if (side == 0) { w->di = -G; w->si = anx - G; } else { w->di = bnx; w->si = 0; }
    } else {
        w->w = bnx + 2 * G; w->h = G; w->di = -G; w->si = -G;
        if (side == 2) { w->dj = -G; w->sj = any - G; } else { w->dj = bny; w->sj = 0; }
    }
}

// ghost layers of every block: field 0 = W[in] (with alpha[in] when with_alpha), 1 = Ws
static cudaError_t halo(dfgks_decomp* d, int field, int in, bool with_alpha) {
    const int* halt = &d->st->halt;
    auto Wof = [&](Block& b) { return field == 0 ? b.W[in] : b.Ws; };
    for (int pass = 0; pass < 2; ++pass) {
        for (Block& b : d->blk) launch_ghost_pass(pass, b.m, Wof(b), with_alpha ? b.A[in] : nullptr, halt, d->stream);
        for (Block& b : d->blk) {
            for (int side = 2 * pass; side < 2 * pass + 2; ++side) {
                const int nb = b.plan.neighbour[side];
                if (nb < 0) continue;
                Block& a = d->blk[nb];
                dfgks_halo_window hw;
                halo_window(b.plan, a.plan, side, &hw);
                cudaError_t e = copy_window(b, Wof(b), hw.di, hw.dj, a, Wof(a), hw.si, hw.sj, hw.w, hw.h, 4, d->stream);
                if (e == cudaSuccess && with_alpha)
                    e = copy_window(b, b.A[in], hw.di, hw.dj, a, a.A[in], hw.si, hw.sj, hw.w, hw.h, 1, d->stream);
                if (e != cudaSuccess) return e;
            }
        }
    }
    return cudaSuccess;
}

static dfgks_status reset_state(dfgks_decomp* d, double t, long long step) {
    DevState z;
    memset(&z, 0, sizeof(z));
    z.t = t;
    z.step = step;
    z.dtmin_bits = 0x7FEFFFFFFFFFFFFFULL;
    z.fail_step = -1;
    z.fail_key = ~0ULL;
    *d->st_host = z;
    DCK(cudaMemcpyAsync(d->st, d->st_host, sizeof(DevState), cudaMemcpyHostToDevice, d->stream));
    DCK(cudaStreamSynchronize(d->stream));
    return DFGKS_OK;
}

extern "C" DFGKS_API dfgks_status dfgks_decomp_plan(const dfgks_config* cfg, int px, int py, int block,
                                                    dfgks_block_plan* out) {
    if (!out || !decomp_config_ok(cfg, px, py) || block < 0 || block >= px * py) return DFGKS_EINVAL;
    make_plan(cfg, px, py, block, out);
    return DFGKS_OK;
}

extern "C" DFGKS_API dfgks_status dfgks_decomp_halo(const dfgks_config* cfg, int px, int py, int block, int side,
                                                    dfgks_halo_window* out) {
    if (!out || !decomp_config_ok(cfg, px, py) || block < 0 || block >= px * py || side < 0 || side > 3)
        return DFGKS_EINVAL;
    dfgks_block_plan b, a;
    make_plan(cfg, px, py, block, &b);
    out->neighbour = b.neighbour[side];
    if (out->neighbour < 0) { out->di = out->dj = out->si = out->sj = out->w = out->h = 0; return DFGKS_OK; }
    make_plan(cfg, px, py, out->neighbour, &a);
    halo_window(b, a, side, out);
    return DFGKS_OK;
}

extern "C" DFGKS_API dfgks_status dfgks_decomp_create(const dfgks_config* cfg, int px, int py, void* stream,
                                                      dfgks_decomp** out) {
    if (!out) return DFGKS_EINVAL;
    *out = nullptr;
    if (!decomp_config_ok(cfg, px, py)) return DFGKS_EINVAL;
    dfgks_decomp* d = new (std::nothrow) dfgks_decomp();
    if (!d) return DFGKS_ENOMEM;
    d->cfg = *cfg;
    d->px = px; d->py = py;
    d->st_host = nullptr; d->flag_host = nullptr;
    d->cur = 0;
    if (stream) { d->stream = (cudaStream_t)stream; d->own_stream = false; }
    else if (cudaStreamCreateWithFlags(&d->stream, cudaStreamNonBlocking) != cudaSuccess) { delete d; return DFGKS_ECUDA; }
    else d->own_stream = true;
    SchemeConsts& S = d->S;
    memset(&S, 0, sizeof(S));
    S.gamma = cfg->gamma; S.gm1 = cfg->gamma - 1.0; S.K = (4.0 - 2.0 * cfg->gamma) / (cfg->gamma - 1.0);
    S.inv_K2 = 1.0 / (S.K + 2.0);
    S.r2g = sqrt(2.0 / S.gamma);
    S.d[3] = cfg->dH; S.d[0] = (1.0 - cfg->dH) * (1.0 - cfg->dL) / 2.0; S.d[1] = (1.0 - cfg->dH) * cfg->dL; S.d[2] = S.d[0];
    S.inv_d3 = 1.0 / cfg->dH;
    S.eps = cfg->eps; S.alpha_thres = cfg->alpha_thres; S.C1 = cfg->C1; S.C2 = cfg->C2;
    S.time_limiter = cfg->time_limiter; S.tau_reading = cfg->tau_reading; S.gp_fallback = cfg->gp_fallback;
    S.df_states = cfg->df_states;
    const double dx = (cfg->x1 - cfg->x0) / cfg->nx, dy = (cfg->y1 - cfg->y0) / cfg->ny;
    cudaError_t e = cudaSuccess;
    d->blk.resize((size_t)px * py);
    for (int b = 0; b < px * py && e == cudaSuccess; ++b) {
        Block& k = d->blk[b];
        memset(&k, 0, sizeof(k));
        make_plan(cfg, px, py, b, &k.plan);
        Mesh& m = k.m;
        m.nx = k.plan.i1 - k.plan.i0; m.ny = k.plan.j1 - k.plan.j0;
        m.P = (int)round4(m.nx + 2 * G);
        m.NYg = m.ny + 2 * G;
        m.plane = (long long)m.P * m.NYg;
        m.dx = dx; m.dy = dy;
        m.rdx = 1.0 / dx; m.rdy = 1.0 / dy;
        for (int s = 0; s < 4; ++s) m.bc[s] = k.plan.bc[s];
        m.dt_rule = cfg->dt_rule;
        m.gi0 = k.plan.i0; m.gj0 = k.plan.j0; m.gnx = cfg->nx;
        const long long nfx = (long long)(m.nx + 1) * m.ny, nfy = (long long)(m.ny + 1) * m.nx;
        const long long nlx = (long long)(m.nx + 1) * (m.ny + 4), nly = (long long)(m.ny + 1) * (m.nx + 4);
        k.B.line_stride = round4(nlx > nly ? nlx : nly);
        k.B.gp_stride = round4(2 * (nfx > nfy ? nfx : nfy));
        k.B.flux_stride[0] = round4(2 * nfx);
        k.B.flux_stride[1] = round4(2 * nfy);
        if (e == cudaSuccess) e = dalloc(d, &k.W[0], 4 * m.plane);
        if (e == cudaSuccess) e = dalloc(d, &k.W[1], 4 * m.plane);
        if (e == cudaSuccess) e = dalloc(d, &k.A[0], m.plane);
        if (e == cudaSuccess) e = dalloc(d, &k.A[1], m.plane);
        if (e == cudaSuccess) e = dalloc(d, &k.Ws, 4 * m.plane);
        if (e == cudaSuccess) e = dalloc(d, &k.acc, 4LL * m.nx * m.ny);
        if (e == cudaSuccess) e = dalloc(d, &k.B.lines, (long long)LR_COUNT * k.B.line_stride);
        if (e == cudaSuccess) e = dalloc(d, &k.B.gp, (long long)GP_COUNT * k.B.gp_stride);
        if (e == cudaSuccess) e = dalloc(d, &k.B.flux[0], (long long)FR_COUNT * k.B.flux_stride[0]);
        if (e == cudaSuccess) e = dalloc(d, &k.B.flux[1], (long long)FR_COUNT * k.B.flux_stride[1]);
        k.By = k.B;
        if (e == cudaSuccess) e = dalloc(d, &k.By.lines, (long long)LR_COUNT * k.B.line_stride);
        if (e == cudaSuccess) e = dalloc(d, &k.By.gp, (long long)GP_COUNT * k.B.gp_stride);
        if (e == cudaSuccess) {
            launch_fill_value(k.W[0], 4 * m.plane, 1.0, d->stream);
            launch_fill_value(k.W[1], 4 * m.plane, 1.0, d->stream);
            launch_fill_value(k.Ws, 4 * m.plane, 1.0, d->stream);
            launch_fill_value(k.A[0], m.plane, 1.0, d->stream);
            launch_fill_value(k.A[1], m.plane, 1.0, d->stream);
        }
    }
    if (e == cudaSuccess) e = dalloc(d, &d->st, 1);
    if (e == cudaSuccess) e = dalloc(d, &d->flag, 1);
    if (e == cudaSuccess) { d->dts_cap = 1024; e = dalloc(d, &d->dts, d->dts_cap); }
    if (e == cudaSuccess) e = dalloc(d, &d->one, 4);
    if (e == cudaSuccess) e = dalloc(d, &d->stage, 4LL * cfg->nx * cfg->ny);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&d->st_host, sizeof(DevState));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&d->flag_host, sizeof(int));
    if (e == cudaSuccess) launch_set_scalar(d->one, 1.0, d->stream);
    dfgks_status r = dstat(e);
    if (r == DFGKS_OK) r = reset_state(d, 0.0, 0);
    if (r != DFGKS_OK) { free_decomp(d); delete d; return r; }
    *out = d;
    return DFGKS_OK;
}

extern "C" DFGKS_API dfgks_status dfgks_decomp_destroy(dfgks_decomp* d) {
    if (!d) return DFGKS_OK;
    cudaStreamSynchronize(d->stream);
    free_decomp(d);
    delete d;
    return DFGKS_OK;
}

extern "C" DFGKS_API dfgks_status dfgks_decomp_set_ic(dfgks_decomp* d, const double* W, int on_device) {
    if (!d || !W) return DFGKS_EINVAL;
    const int nx = d->cfg.nx, ny = d->cfg.ny;
    const long long N = (long long)nx * ny;
    DCK(cudaMemcpyAsync(d->stage, W, (size_t)(4 * N) * sizeof(double),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, d->stream));
    DCK(cudaMemsetAsync(d->flag, 0, sizeof(int), d->stream));
    d->cur = 0;
    for (Block& b : d->blk) {
        const long long nb = (long long)b.m.nx * b.m.ny;
        for (int k = 0; k < 4; ++k)
            DCK(cudaMemcpy2DAsync(b.acc + k * nb, (size_t)b.m.nx * sizeof(double),
                                  d->stage + k * N + (long long)b.plan.j0 * nx + b.plan.i0, (size_t)nx * sizeof(double),
                                  (size_t)b.m.nx * sizeof(double), (size_t)b.m.ny, cudaMemcpyDeviceToDevice, d->stream));
        launch_dense_to_ghosted(b.m, b.acc, 4, b.W[0], d->stream);
        launch_check_state(b.m, b.W[0], d->S.gm1, d->flag, d->stream);
    }
    DCK(cudaGetLastError());
    DCK(cudaMemcpyAsync(d->flag_host, d->flag, sizeof(int), cudaMemcpyDeviceToHost, d->stream));
    DCK(cudaStreamSynchronize(d->stream));
    if (*d->flag_host) return DFGKS_ENONPHYS;
    // alpha^0: the Gauss-point DF factors of a reconstruction of W^0 with alpha = 1
    dfgks_status r = reset_state(d, 0.0, 0);
    if (r != DFGKS_OK) return r;
    for (Block& b : d->blk) launch_fill_value(b.A[0], b.m.plane, 1.0, d->stream);
    DCK(halo(d, 0, 0, false));
    for (Block& b : d->blk) {
        launch_sweep_xy(b.m, d->S, 1, true, b.W[0], b.A[0], d->one, b.B, b.By, nullptr, nullptr, d->stream);
        UpdateArgs a;
        memset(&a, 0, sizeof(a));
        a.alpha_out = b.A[0];
        launch_update(UM_ALPHA, b.m, d->S, a, b.B, d->one, nullptr, nullptr, d->stream);
    }
    DCK(cudaGetLastError());
    DCK(cudaStreamSynchronize(d->stream));
    return DFGKS_OK;
}

// one S2O4 step (Eq. 24 with the time limiter) of all blocks from buffer `in` to `in ^ 1`; every
// kernel returns at once once the shared halt flag is set, so a queue of steps drains without
// work and the state stays at the last good step (the halo copies then touch ghost cells only)
static cudaError_t enqueue_decomp_step(dfgks_decomp* d, int s, int in, int flux, double t_end) {
    cudaStream_t st = d->stream;
    DevState* ds = d->st;
    const int* halt = &ds->halt;
    const double* dtp = &ds->dt;
    const int out = in ^ 1;
    for (Block& b : d->blk) launch_cfl_min(b.m, b.W[in], d->S.gamma, ds, st);     // minimum over all blocks
    launch_begin_step(ds, d->cfg.cfl, 0.0, t_end, d->dts, s, st);
    cudaError_t e = halo(d, 0, in, true);
    if (e != cudaSuccess) return e;
    for (Block& b : d->blk) {
        launch_sweep_xy(b.m, d->S, flux, false, b.W[in], b.A[in], dtp, b.B, b.By, ds, halt, st);
        UpdateArgs a;
        memset(&a, 0, sizeof(a));
        a.Win = b.W[in]; a.Wout = b.Ws; a.acc = b.acc;
        launch_update(UM_S2O4_1, b.m, d->S, a, b.B, dtp, ds, halt, st);
    }
    e = halo(d, 1, in, false);
    if (e != cudaSuccess) return e;
    for (Block& b : d->blk) {
        launch_sweep_xy(b.m, d->S, flux, false, b.Ws, b.A[in], dtp, b.B, b.By, ds, halt, st);
        UpdateArgs a;
        memset(&a, 0, sizeof(a));
        a.Win = b.Ws; a.Wout = b.W[out]; a.acc = b.acc; a.alpha_out = b.A[out];
        launch_update(UM_S2O4_2, b.m, d->S, a, b.B, dtp, ds, halt, st);
    }
    launch_end_step(ds, t_end, st);
    return cudaGetLastError();
}

// n steps with the CFL dt (the minimum over all blocks), the last clipped to t_end > 0; one
// synchronisation at the end.  ENONPOS on a positivity failure (dfgks_decomp_status gives the cell
// in the whole mesh), with the state left at the last good step.
extern "C" DFGKS_API dfgks_status dfgks_decomp_step(dfgks_decomp* d, int n, int flux, double t_end, int* steps_done) {
    if (steps_done) *steps_done = 0;
    if (!d || n < 0 || (flux != DFGKS_FLUX_GKS && flux != DFGKS_FLUX_LF)) return DFGKS_EINVAL;
    if (n == 0) return DFGKS_OK;
    if (n > d->dts_cap) {
        double* p = nullptr;
        DCK(cudaMalloc((void**)&p, (size_t)n * sizeof(double)));
        d->allocs.push_back(p);
        d->dts = p;
        d->dts_cap = n;
    }
    DCK(cudaMemsetAsync(&d->st->halt, 0, sizeof(int), d->stream));
    DCK(cudaMemsetAsync(&d->st->err, 0, sizeof(int), d->stream));
    DCK(cudaMemcpyAsync(d->st_host, d->st, sizeof(DevState), cudaMemcpyDeviceToHost, d->stream));
    DCK(cudaStreamSynchronize(d->stream));
    const long long step0 = d->st_host->step;
    const int cur0 = d->cur;
    for (int s = 0; s < n; ++s) DCK(enqueue_decomp_step(d, s, (cur0 + s) & 1, flux, t_end));
    DCK(cudaMemcpyAsync(d->st_host, d->st, sizeof(DevState), cudaMemcpyDeviceToHost, d->stream));
    DCK(cudaStreamSynchronize(d->stream));
    const long long done = d->st_host->step - step0;
    d->cur = (int)((cur0 + done) & 1);
    if (steps_done) *steps_done = (int)done;
    return d->st_host->err ? DFGKS_ENONPOS : DFGKS_OK;
}

extern "C" DFGKS_API dfgks_status dfgks_decomp_get_state(dfgks_decomp* d, double* W, double* alpha, double* t, long* step,
                                                         int on_device) {
    if (!d) return DFGKS_EINVAL;
    const int nx = d->cfg.nx;
    const long long N = (long long)nx * d->cfg.ny;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int q = 0; q < 2; ++q) {
        double* dst = q == 0 ? W : alpha;
        if (!dst) continue;
        const int nc = q == 0 ? 4 : 1;
        for (Block& b : d->blk) {
            const long long nb = (long long)b.m.nx * b.m.ny;
            launch_ghosted_to_dense(b.m, q == 0 ? b.W[d->cur] : b.A[d->cur], nc, b.acc, d->stream);
            for (int k = 0; k < nc; ++k)
                DCK(cudaMemcpy2DAsync(d->stage + k * N + (long long)b.plan.j0 * nx + b.plan.i0, (size_t)nx * sizeof(double),
                                      b.acc + k * nb, (size_t)b.m.nx * sizeof(double), (size_t)b.m.nx * sizeof(double),
                                      (size_t)b.m.ny, cudaMemcpyDeviceToDevice, d->stream));
        }
        DCK(cudaGetLastError());
        DCK(cudaMemcpyAsync(dst, d->stage, (size_t)(nc * N) * sizeof(double), kind, d->stream));
    }
    DCK(cudaMemcpyAsync(d->st_host, d->st, sizeof(DevState), cudaMemcpyDeviceToHost, d->stream));
    DCK(cudaStreamSynchronize(d->stream));
    if (t) *t = d->st_host->t;
    if (step) *step = (long)d->st_host->step;
    return DFGKS_OK;
}

extern "C" DFGKS_API dfgks_status dfgks_decomp_status(dfgks_decomp* d, int* err, int* fail_i, int* fail_j,
                                                      dfgks_counters* counters) {
    if (!d) return DFGKS_EINVAL;
    DCK(cudaMemcpyAsync(d->st_host, d->st, sizeof(DevState), cudaMemcpyDeviceToHost, d->stream));
    DCK(cudaStreamSynchronize(d->stream));
    const DevState& h = *d->st_host;
    if (err) *err = h.err;
    const bool failed = h.err != 0;
    if (fail_i) *fail_i = failed ? (int)(h.fail_key % (unsigned long long)d->cfg.nx) : -1;
    if (fail_j) *fail_j = failed ? (int)(h.fail_key / (unsigned long long)d->cfg.nx) : -1;
    if (counters) {
        counters->fallbacks = h.fallbacks;
        counters->df_normal = h.df_normal;
        counters->df_tangential = h.df_tangential;
    }
    return DFGKS_OK;
}
