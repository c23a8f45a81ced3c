// dfgks_noalloc.cu -- the single-stage operator for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the stage operator: code that
// runs while a CUDA graph is being built, host frameworks whose device memory is owned by their own
// pool allocator and which forbid driver allocations once a run has started, or latency-bound loops
// where an allocation (and its implicit synchronisation) is not acceptable.  A dfgks handle
// allocates all of its buffers in dfgks_create, so such callers cannot hold one.  This entry point
// takes a configuration instead of a handle and keeps every intermediate in one file-scope device
// array, so the call itself allocates nothing; the caller still passes inputs and outputs.
#include <cuda_runtime.h>
#include <mutex>
#include <string.h>

#include "../../include/dfgks.h"
#include "dfgks_internal.h"

using namespace dfk;

namespace {

// 16 MiB of scratch, enough for every mesh whose sides are both at most 128 cells (128 x 128
// needs 2,036,956 doubles of the 2,097,152).  Every GPU that loads the library holds this array
// until the process exits.
constexpr long long kScratchDoubles = 2LL * 1024 * 1024;
constexpr int kMaxSide = 128;
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

long long round_up(long long n, long long a) { return (n + a - 1) / a * a; }

// The host-side name of g_noalloc_scratch is only a stand-in; the device address is looked up
// once per device, with that device current.
dfgks_status scratch_for_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DFGKS_ECUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DFGKS_ECUDA;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return DFGKS_OK;
}

bool valid(const dfgks_config* c) {
    if (!c || c->nx < 1 || c->ny < 1) return false;
    if (!(c->x1 > c->x0) || !(c->y1 > c->y0)) return false;
    if (!(c->gamma > 1.0) || !(c->eps > 0.0)) return false;
    if (!(c->dH > 0.0 && c->dH <= 1.0) || !(c->dL >= 0.0 && c->dL <= 1.0)) return false;
    if (!(c->C1 >= 0.0) || !(c->C2 >= 0.0)) return false;
    const int bcs[4] = {c->bc_xlo, c->bc_xhi, c->bc_ylo, c->bc_yhi};
    for (int k = 0; k < 4; ++k) if (bcs[k] < 0 || bcs[k] > 2) return false;
    if ((c->bc_xlo == 0) != (c->bc_xhi == 0) || (c->bc_ylo == 0) != (c->bc_yhi == 0)) return false;
    // periodic wrap and wall mirror both copy G interior cells into the ghost layers (outflow
    // copies one), so a direction with a periodic or reflecting end needs at least G cells
    if ((c->bc_xlo != 1 || c->bc_xhi != 1) && c->nx < G) return false;
    if ((c->bc_ylo != 1 || c->bc_yhi != 1) && c->ny < G) return false;
    if (c->tau_reading != 0 && c->tau_reading != 1) return false;
    if (c->df_states != 0 && c->df_states != 1) return false;
    if (c->alpha_source != 0 && c->alpha_source != 1) return false;    // a step option; no stage effect
    return true;
}

}  // namespace

extern "C" DFGKS_API dfgks_status dfgks_residual_noalloc(const dfgks_config* cfg, void* stream,
                                                         const double* W, const double* alpha, double dt,
                                                         int flux, double* L, double* dtL, double* dtLt,
                                                         double* alpha_next) {
    if (!valid(cfg) || !W || !alpha || !(dt > 0.0) || (flux != 0 && flux != 1)) return DFGKS_EINVAL;
    if (cfg->nx > kMaxSide || cfg->ny > kMaxSide) return DFGKS_EINVAL;

    Mesh m;
    m.nx = cfg->nx; m.ny = cfg->ny;
    m.P = (int)round_up(cfg->nx + 2 * G, 4);
    m.NYg = cfg->ny + 2 * G;
    m.plane = (long long)m.P * m.NYg;
    m.dx = (cfg->x1 - cfg->x0) / cfg->nx;
    m.dy = (cfg->y1 - cfg->y0) / cfg->ny;
    m.rdx = 1.0 / m.dx; m.rdy = 1.0 / m.dy;
    m.bc[0] = cfg->bc_xlo; m.bc[1] = cfg->bc_xhi; m.bc[2] = cfg->bc_ylo; m.bc[3] = cfg->bc_yhi;
    m.dt_rule = cfg->dt_rule;
    m.gi0 = 0; m.gj0 = 0; m.gnx = cfg->nx;
    SchemeConsts S;
    memset(&S, 0, sizeof(S));
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

    // carve the scratch: ghosted W and alpha, line, Gauss-point and flux records, dt
    const long long nfx = (long long)(m.nx + 1) * m.ny, nfy = (long long)(m.ny + 1) * m.nx;
    const long long nlx = (long long)(m.nx + 1) * (m.ny + 4), nly = (long long)(m.ny + 1) * (m.nx + 4);
    SweepBuffers B;
    B.line_stride = round_up(nlx > nly ? nlx : nly, 4);
    B.gp_stride = round_up(2 * (nfx > nfy ? nfx : nfy), 4);
    B.flux_stride[0] = round_up(2 * nfx, 4);
    B.flux_stride[1] = round_up(2 * nfy, 4);
    const long long sizes[7] = {4 * m.plane, m.plane, (long long)LR_COUNT * B.line_stride,
                                (long long)GP_COUNT * B.gp_stride, (long long)FR_COUNT * B.flux_stride[0],
                                (long long)FR_COUNT * B.flux_stride[1], 1};
    long long offs[7], total = 0;
    for (int k = 0; k < 7; ++k) { offs[k] = total; total += round_up(sizes[k], 32); }
    if (total > kScratchDoubles) return DFGKS_EINVAL;

    double* base = nullptr;
    dfgks_status r = scratch_for_current_device(&base);
    if (r != DFGKS_OK) return r;
    double* Wg = base + offs[0];
    double* Ag = base + offs[1];
    B.lines = base + offs[2];
    B.gp = base + offs[3];
    B.flux[0] = base + offs[4];
    B.flux[1] = base + offs[5];
    double* dtp = base + offs[6];

    // Every element read below is written earlier in this call (ghost fill covers all ghost
    // cells, the sweeps write every record they later read), so nothing needs clearing.
    cudaStream_t s = (cudaStream_t)stream;
    launch_dense_to_ghosted(m, W, 4, Wg, s);
    launch_dense_to_ghosted(m, alpha, 1, Ag, s);
    launch_fill_ghosts(m, Wg, Ag, nullptr, s);
    launch_set_scalar(dtp, dt, s);
    for (int d = 0; d < 2; ++d) launch_sweep(d, m, S, flux, false, Wg, Ag, dtp, B, nullptr, nullptr, s);
    UpdateArgs a;
    memset(&a, 0, sizeof(a));
    a.L = L; a.dtL = dtL; a.dtLt = dtLt; a.alpha_out = alpha_next; a.alpha_dense = 1;
    launch_update(UM_RESIDUAL, m, S, a, B, dtp, nullptr, nullptr, s);
    if (cudaGetLastError() != cudaSuccess) return DFGKS_ECUDA;
    return DFGKS_OK;
}
