// dfgks_batch.cu -- many independent problems of uneven mesh sizes advanced together.
//
// Every phase of a step (CFL dt, ghost fill, the three sweep kernels per direction and stage, the
// stage update, bookkeeping) is one launch over all problems: each thread block looks its problem
// up in a prefix table of per-problem block counts and runs the same per-thread body as the
// single-problem kernels (dfgks_bodies.cuh), so small meshes fill the GPU together instead of
// one after another.  The sweep kernels use 1-D blocks over each problem's row-major index space
// (face lines, face sides, Gauss points), so only a problem's last warp is partly idle; their
// block size is chosen by an autotuner.  Each problem keeps its own device-resident dt, time, halt
// flag and state buffer parity, so every step is the same launch sequence: n steps are captured
// once in a CUDA graph and one graph launch advances all problems n steps.
#include <cuda_runtime.h>
#include <float.h>
#include <string.h>
#include <new>
#include <vector>

#include "../../include/dfgks.h"
#include "dfgks_bodies.cuh"

using namespace dfk;

namespace {

struct BatchProblem {
    Mesh m;
    SchemeConsts S;
    int flux;
    double* W[2];
    double* A[2];
    double* Ws;
    double* acc;
    SweepBuffers B;
    DevState* st;
};

// Phases with a per-problem block grid.  The sweep phases run 1-D blocks of a tunable size over a
// problem's index space (lx x ly items, row-major; the face and flux phases twice, once per side /
// Gauss point); the others have fixed shapes.
enum Phase { PH_GX = 0, PH_GY, PH_CFL, PH_LINES0, PH_LINES1, PH_FACES0, PH_FACES1, PH_FLUX0, PH_FLUX1, PH_UPD,
             PH_COUNT };

__host__ __device__ inline void sweep_space(int ph, const Mesh& m, int& lx, int& ly, int& nz) {
    nz = 1;
    switch (ph) {
        case PH_LINES0: lx = lines_lx<0>(m); ly = lines_ly<0>(m); break;
        case PH_LINES1: lx = lines_lx<1>(m); ly = lines_ly<1>(m); break;
        case PH_FACES0: case PH_FLUX0: lx = faces_lx<0>(m); ly = faces_ly<0>(m); nz = 2; break;
        default: lx = faces_lx<1>(m); ly = faces_ly<1>(m); nz = 2; break;   // PH_FACES1, PH_FLUX1
    }
}

__host__ __device__ inline bool is_sweep(int ph) { return ph >= PH_LINES0 && ph <= PH_FLUX1; }

// blocks of one problem in phase ph (bs: threads per block of a sweep phase); for a sweep phase
// also the blocks per side, per_z
__host__ __device__ inline int phase_blocks(int ph, const Mesh& m, int bs, int& per_z) {
    per_z = 0;
    switch (ph) {
        case PH_GX: return (m.ny + 31) / 32;
        case PH_GY: return ((m.nx + 2 * G + 127) / 128) * 2 * G;
        case PH_CFL: return (m.nx * m.ny + 255) / 256;
        case PH_UPD: return ((m.nx + 31) / 32) * ((m.ny + 7) / 8);
        default: {
            int lx, ly, nz;
            sweep_space(ph, m, lx, ly, nz);
            per_z = (int)(((long long)lx * ly + bs - 1) / bs);
            return per_z * nz;
        }
    }
}

struct BlockMap {
    const int* start;     // device: np + 1 prefix of block counts
    int np;
    int bs;               // threads per block of a sweep phase
};

// problem of this block and the block's index inside that problem's part of the grid
__device__ __forceinline__ int locate(const BlockMap& bm, int& local) {
    int lo = 0, hi = bm.np;                 // start[lo] <= blockIdx.x < start[hi]
    const int b = blockIdx.x;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (bm.start[mid] <= b) lo = mid; else hi = mid;
    }
    local = b - bm.start[lo];
    return lo;
}

// item (ax, ay) and side / Gauss point z of this thread in sweep phase ph
__device__ __forceinline__ void sweep_item(int ph, const Mesh& m, int local, int& ax, int& ay, int& z) {
    int lx, ly, nz;
    sweep_space(ph, m, lx, ly, nz);
    const int per_z = (int)(((long long)lx * ly + blockDim.x - 1) / blockDim.x);
    z = local / per_z;
    const long long i = (long long)(local - z * per_z) * blockDim.x + threadIdx.x;
    ax = (int)(i % lx);
    ay = (int)(i / lx);                     // >= ly past the end: rejected by the bodies' bounds checks
}

__global__ void kb_cfl(const BatchProblem* P, BlockMap bm) {
    int local;
    const int p = locate(bm, local);
    const BatchProblem& q = P[p];
    if (q.st->halt) return;
    const int c = local * 256 + threadIdx.x;
    double v = c < q.m.nx * q.m.ny ? cfl_cell(q.m, q.W[q.st->par], q.S.gamma, c) : DBL_MAX;
    v = block_min(v);
    if (threadIdx.x == 0 && v > 0.0) atomicMin(&q.st->dtmin_bits, (unsigned long long)__double_as_longlong(v));
}

__global__ void kb_begin_step(const BatchProblem* P, const double* cfl, int np, double t_end) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    DevState* st = P[p].st;
    const double dtmin = __longlong_as_double((long long)st->dtmin_bits);
    st->dtmin_bits = (unsigned long long)__double_as_longlong(DBL_MAX);
    if (st->halt) return;
    if (t_end > 0.0 && st->t >= t_end) { st->halt = 1; return; }
    double dt = cfl[p] * dtmin;
    st->clipped = 0;
    if (t_end > 0.0 && st->t + dt >= t_end - 1e-12 * fabs(t_end)) { dt = t_end - st->t; st->clipped = 1; }
    st->dt = dt;
}

__global__ void kb_end_step(const BatchProblem* P, int np, double t_end) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    DevState* st = P[p].st;
    if (st->halt) return;
    st->t = st->clipped ? t_end : st->t + st->dt;
    st->step += 1;
    st->par ^= 1;
}

// stage 0 reads W^n (and fills alpha^n ghosts), stage 1 reads W*
__global__ void kb_ghost_x(const BatchProblem* P, BlockMap bm, int stage) {
    int bx;
    const int p = locate(bm, bx);
    const BatchProblem& q = P[p];
    if (q.st->halt) return;
    double* W = stage == 0 ? q.W[q.st->par] : q.Ws;
    double* A = stage == 0 ? q.A[q.st->par] : nullptr;
    ghost_x_body(q.m, W, A, threadIdx.x, bx * blockDim.y + threadIdx.y);
}

__global__ void kb_ghost_y(const BatchProblem* P, BlockMap bm, int stage) {
    int local;
    const int p = locate(bm, local);
    const BatchProblem& q = P[p];
    const int gxb = (q.m.nx + 2 * G + 127) / 128, bx = local % gxb, by = local / gxb;
    if (q.st->halt) return;
    double* W = stage == 0 ? q.W[q.st->par] : q.Ws;
    double* A = stage == 0 ? q.A[q.st->par] : nullptr;
    ghost_y_body(q.m, W, A, bx * blockDim.x + threadIdx.x - G, by);
}

template <int DIR>
__global__ void __launch_bounds__(256) kb_lines(const BatchProblem* P, BlockMap bm, int stage) {
    int local, ax, ay, z;
    const int p = locate(bm, local);
    const BatchProblem& q = P[p];
    if (q.st->halt) return;
    sweep_item(DIR == 0 ? PH_LINES0 : PH_LINES1, q.m, local, ax, ay, z);
    const int par = q.st->par;
    const double* W = stage == 0 ? q.W[par] : q.Ws;
    int ndf = lines_body<DIR>(q.m, q.S, W, q.A[par], q.B.lines, q.B.line_stride, ax, ay);
    warp_count_add(&q.st->df_normal, ndf);
}

template <int DIR>
__global__ void __launch_bounds__(256) kb_faces(const BatchProblem* P, BlockMap bm, int stage) {
    int local, ax, ay, z;
    const int p = locate(bm, local);
    const BatchProblem& q = P[p];
    if (q.st->halt) return;
    sweep_item(DIR == 0 ? PH_FACES0 : PH_FACES1, q.m, local, ax, ay, z);
    const int par = q.st->par;
    const double* W = stage == 0 ? q.W[par] : q.Ws;
    int nfb;
    int ndf = faces_body<DIR>(q.m, q.S, W, q.A[par], q.B.lines, q.B.line_stride, q.B.gp, q.B.gp_stride,
                              ax, ay, z, nfb);
    warp_count_add(&q.st->df_tangential, ndf);
    warp_count_add(&q.st->fallbacks, nfb);
}

template <int DIR>
__global__ void __launch_bounds__(256) kb_flux(const BatchProblem* P, BlockMap bm) {
    int local, ax, ay, z;
    const int p = locate(bm, local);
    const BatchProblem& q = P[p];
    if (q.st->halt) return;
    sweep_item(DIR == 0 ? PH_FLUX0 : PH_FLUX1, q.m, local, ax, ay, z);
    if (q.flux == 0)
        flux_body<DIR, 0, false>(q.m, q.S, q.B.lines, q.B.line_stride, q.B.gp, q.B.gp_stride, q.B.flux[DIR],
                                 q.B.flux_stride[DIR], q.st->dt, ax, ay, z);
    else
        flux_body<DIR, 1, false>(q.m, q.S, q.B.lines, q.B.line_stride, q.B.gp, q.B.gp_stride, q.B.flux[DIR],
                                 q.B.flux_stride[DIR], q.st->dt, ax, ay, z);
}

template <int MODE>
__global__ void __launch_bounds__(256) kb_update(const BatchProblem* P, BlockMap bm) {
    int local;
    const int p = locate(bm, local);
    const BatchProblem& q = P[p];
    const int gxb = (q.m.nx + 31) / 32, bx = local % gxb, by = local / gxb;
    if (q.st->halt) return;
    const int par = q.st->par;
    UpdateArgs a;
    a.Wn = nullptr; a.L = nullptr; a.dtL = nullptr; a.dtLt = nullptr; a.alpha_dense = 0;
    a.acc = q.acc;
    if (MODE == UM_S2O4_1) { a.Win = q.W[par]; a.Wout = q.Ws; a.alpha_out = nullptr; }
    else { a.Win = q.Ws; a.Wout = q.W[par ^ 1]; a.alpha_out = q.A[par ^ 1]; }
    update_body<MODE>(q.m, q.S, a, q.B.flux[0], q.B.flux_stride[0], q.B.flux[1], q.B.flux_stride[1], q.st->dt, q.st,
                      bx * 32 + threadIdx.x, by * 8 + threadIdx.y);
}

}  // namespace

struct dfgks_batch {
    int np;
    cudaStream_t stream;
    bool own_stream;
    std::vector<BatchProblem> host;      // descriptors (device pointers inside)
    BatchProblem* dev;                   // device copy
    DevState* st;                        // np device states
    DevState* st_host;                   // pinned mirror
    double* cfl;                         // per-problem CFL numbers (device)
    int* starts;                         // PH_COUNT x (np + 1) prefix tables (device)
    std::vector<int> hstarts;
    int total[PH_COUNT];
    int block[3];                        // threads per block: face lines, face sides, Gauss points
    std::vector<void*> allocs;
    unsigned long long bytes;
    cudaGraphExec_t graph;               // n_graph steps of every problem
    bool graph_ok;
    int n_graph;
    double t_end;
};

static dfgks_status cst(cudaError_t e) {
    return e == cudaSuccess ? DFGKS_OK : (e == cudaErrorMemoryAllocation ? DFGKS_ENOMEM : DFGKS_ECUDA);
}
#define BCK(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) return cst(e_); } while (0)

static long long rup(long long n, long long a) { return (n + a - 1) / a * a; }

static int block_of(const dfgks_batch* b, int ph) {
    if (ph == PH_LINES0 || ph == PH_LINES1) return b->block[0];
    if (ph == PH_FACES0 || ph == PH_FACES1) return b->block[1];
    if (ph == PH_FLUX0 || ph == PH_FLUX1) return b->block[2];
    return 0;
}

static dfgks_status build_maps(dfgks_batch* b) {
    b->hstarts.assign((size_t)PH_COUNT * (b->np + 1), 0);
    for (int ph = 0; ph < PH_COUNT; ++ph) {
        long long acc = 0;
        for (int p = 0; p < b->np; ++p) {
            int per_z;
            b->hstarts[(size_t)ph * (b->np + 1) + p] = (int)acc;
            acc += phase_blocks(ph, b->host[p].m, block_of(b, ph), per_z);
        }
        if (acc > 0x7fffffffLL) return DFGKS_EINVAL;            // grid.x limit
        b->hstarts[(size_t)ph * (b->np + 1) + b->np] = (int)acc;
        b->total[ph] = (int)acc;
    }
    BCK(cudaMemcpyAsync(b->starts, b->hstarts.data(), b->hstarts.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    return DFGKS_OK;
}

static BlockMap bmap(const dfgks_batch* b, int ph) {
    BlockMap m;
    m.start = b->starts + (size_t)ph * (b->np + 1);
    m.np = b->np;
    m.bs = block_of(b, ph);
    return m;
}

static void enqueue_batch_step(dfgks_batch* b) {
    cudaStream_t s = b->stream;
    const BatchProblem* P = b->dev;
    const int np = b->np, tb = 128, nb = (np + tb - 1) / tb;
    kb_cfl<<<b->total[PH_CFL], 256, 0, s>>>(P, bmap(b, PH_CFL));
    kb_begin_step<<<nb, tb, 0, s>>>(P, b->cfl, np, b->t_end);
    for (int stage = 0; stage < 2; ++stage) {
        kb_ghost_x<<<b->total[PH_GX], dim3(2 * G, 32), 0, s>>>(P, bmap(b, PH_GX), stage);
        kb_ghost_y<<<b->total[PH_GY], 128, 0, s>>>(P, bmap(b, PH_GY), stage);
        kb_lines<0><<<b->total[PH_LINES0], b->block[0], 0, s>>>(P, bmap(b, PH_LINES0), stage);
        kb_faces<0><<<b->total[PH_FACES0], b->block[1], 0, s>>>(P, bmap(b, PH_FACES0), stage);
        kb_flux<0><<<b->total[PH_FLUX0], b->block[2], 0, s>>>(P, bmap(b, PH_FLUX0));
        kb_lines<1><<<b->total[PH_LINES1], b->block[0], 0, s>>>(P, bmap(b, PH_LINES1), stage);
        kb_faces<1><<<b->total[PH_FACES1], b->block[1], 0, s>>>(P, bmap(b, PH_FACES1), stage);
        kb_flux<1><<<b->total[PH_FLUX1], b->block[2], 0, s>>>(P, bmap(b, PH_FLUX1));
        if (stage == 0) kb_update<UM_S2O4_1><<<b->total[PH_UPD], dim3(32, 8), 0, s>>>(P, bmap(b, PH_UPD));
        else kb_update<UM_S2O4_2><<<b->total[PH_UPD], dim3(32, 8), 0, s>>>(P, bmap(b, PH_UPD));
    }
    kb_end_step<<<nb, tb, 0, s>>>(P, np, b->t_end);
}

static void drop_graph(dfgks_batch* b) {
    if (b->graph_ok) cudaGraphExecDestroy(b->graph);
    b->graph_ok = false;
    b->n_graph = 0;
}

// capture n steps of every problem into one CUDA graph (n x 21 kernel nodes)
static dfgks_status capture_steps(dfgks_batch* b, int n) {
    drop_graph(b);
    cudaGraph_t g;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < n; ++k) enqueue_batch_step(b);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess) return cst(e);
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cst(e);
    b->graph_ok = true;
    b->n_graph = n;
    return DFGKS_OK;
}

static void free_batch(dfgks_batch* b) {
    drop_graph(b);
    for (void* p : b->allocs) cudaFree(p);
    if (b->st_host) cudaFreeHost(b->st_host);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

template <class T>
static cudaError_t balloc(dfgks_batch* b, T** p, size_t n) {
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e == cudaSuccess) { b->allocs.push_back((void*)*p); b->bytes += n * sizeof(T); }
    return e;
}

static bool batch_config_ok(const dfgks_config* c) {
    if (!c || c->nx < 1 || c->ny < 1 || c->nx > 8192 || c->ny > 8192) return false;
    if (!(c->x1 > c->x0) || !(c->y1 > c->y0) || !(c->gamma > 1.0) || !(c->cfl > 0.0) || !(c->eps > 0.0)) return false;
    if (!(c->dH > 0.0 && c->dH <= 1.0) || !(c->dL >= 0.0 && c->dL <= 1.0) || !(c->C1 >= 0.0) || !(c->C2 >= 0.0)) return false;
    const int bcs[4] = {c->bc_xlo, c->bc_xhi, c->bc_ylo, c->bc_yhi};
    for (int k = 0; k < 4; ++k) if (bcs[k] < 0 || bcs[k] > 2) return false;
    if ((c->bc_xlo == 0) != (c->bc_xhi == 0) || (c->bc_ylo == 0) != (c->bc_yhi == 0)) return false;
    // periodic wrap and wall mirror both copy G interior cells into the ghost layers
    if ((c->bc_xlo != 1 || c->bc_xhi != 1) && c->nx < G) return false;
    if ((c->bc_ylo != 1 || c->bc_yhi != 1) && c->ny < G) return false;
    return c->time_scheme == 0 && (c->tau_reading == 0 || c->tau_reading == 1) && (c->dt_rule == 0 || c->dt_rule == 1)
        && (c->df_states == 0 || c->df_states == 1) && c->alpha_source == 0;
}

extern "C" DFGKS_API dfgks_status dfgks_batch_create(const dfgks_config* cfgs, const int* flux, int np, void* stream,
                                                     dfgks_batch** out) {
    if (!out || !cfgs || !flux || np < 1 || np > 65536) return DFGKS_EINVAL;
    *out = nullptr;
    for (int p = 0; p < np; ++p)
        if (!batch_config_ok(&cfgs[p]) || (flux[p] != 0 && flux[p] != 1)) return DFGKS_EINVAL;
    dfgks_batch* b = new (std::nothrow) dfgks_batch();
    if (!b) return DFGKS_ENOMEM;
    b->np = np;
    b->bytes = 0;
    b->graph_ok = false;
    b->n_graph = 0;
    b->t_end = 0.0;
    b->st_host = nullptr;
    b->dev = nullptr;
    b->block[0] = b->block[1] = b->block[2] = 128;
    if (stream) { b->stream = (cudaStream_t)stream; b->own_stream = false; }
    else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) { delete b; return DFGKS_ECUDA; }
    else b->own_stream = true;
    cudaError_t e = balloc(b, &b->st, (size_t)np);
    if (e == cudaSuccess) e = balloc(b, &b->dev, (size_t)np);
    if (e == cudaSuccess) e = balloc(b, &b->cfl, (size_t)np);
    if (e == cudaSuccess) e = balloc(b, &b->starts, (size_t)PH_COUNT * (np + 1));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->st_host, (size_t)np * sizeof(DevState));
    std::vector<double> cfl(np);
    b->host.resize(np);
    for (int p = 0; p < np && e == cudaSuccess; ++p) {
        const dfgks_config* c = &cfgs[p];
        BatchProblem& q = b->host[p];
        memset(&q, 0, sizeof(q));
        Mesh& m = q.m;
        m.nx = c->nx; m.ny = c->ny;
        m.P = (int)rup(c->nx + 2 * G, 4);
        m.NYg = c->ny + 2 * G;
        m.plane = (long long)m.P * m.NYg;
        m.dx = (c->x1 - c->x0) / c->nx;
        m.dy = (c->y1 - c->y0) / c->ny;
        m.rdx = 1.0 / m.dx; m.rdy = 1.0 / m.dy;
        m.bc[0] = c->bc_xlo; m.bc[1] = c->bc_xhi; m.bc[2] = c->bc_ylo; m.bc[3] = c->bc_yhi;
        m.dt_rule = c->dt_rule;
        SchemeConsts& S = q.S;
        S.gamma = c->gamma; S.gm1 = c->gamma - 1.0; S.K = (4.0 - 2.0 * c->gamma) / (c->gamma - 1.0);
        S.inv_K2 = 1.0 / (S.K + 2.0);
        S.r2g = sqrt(2.0 / S.gamma);
        S.d[3] = c->dH; S.d[0] = (1.0 - c->dH) * (1.0 - c->dL) / 2.0; S.d[1] = (1.0 - c->dH) * c->dL; S.d[2] = S.d[0];
        S.inv_d3 = 1.0 / c->dH;
        S.eps = c->eps; S.alpha_thres = c->alpha_thres; S.C1 = c->C1; S.C2 = c->C2;
        S.time_limiter = c->time_limiter; S.tau_reading = c->tau_reading; S.gp_fallback = c->gp_fallback;
        S.df_states = c->df_states;
        q.flux = flux[p];
        cfl[p] = c->cfl;
        const long long nfx = (long long)(m.nx + 1) * m.ny, nfy = (long long)(m.ny + 1) * m.nx;
        const long long nlx = (long long)(m.nx + 1) * (m.ny + 4), nly = (long long)(m.ny + 1) * (m.nx + 4);
        q.B.line_stride = rup(nlx > nly ? nlx : nly, 4);
        q.B.gp_stride = rup(2 * (nfx > nfy ? nfx : nfy), 4);
        q.B.flux_stride[0] = rup(2 * nfx, 4);
        q.B.flux_stride[1] = rup(2 * nfy, 4);
        const long long dense = (long long)m.nx * m.ny;
        if (e == cudaSuccess) e = balloc(b, &q.W[0], (size_t)(4 * m.plane));
        if (e == cudaSuccess) e = balloc(b, &q.W[1], (size_t)(4 * m.plane));
        if (e == cudaSuccess) e = balloc(b, &q.A[0], (size_t)m.plane);
        if (e == cudaSuccess) e = balloc(b, &q.A[1], (size_t)m.plane);
        if (e == cudaSuccess) e = balloc(b, &q.Ws, (size_t)(4 * m.plane));
        if (e == cudaSuccess) e = balloc(b, &q.acc, (size_t)(4 * dense));
        if (e == cudaSuccess) e = balloc(b, &q.B.lines, (size_t)(LR_COUNT * q.B.line_stride));
        if (e == cudaSuccess) e = balloc(b, &q.B.gp, (size_t)(GP_COUNT * q.B.gp_stride));
        if (e == cudaSuccess) e = balloc(b, &q.B.flux[0], (size_t)(FR_COUNT * q.B.flux_stride[0]));
        if (e == cudaSuccess) e = balloc(b, &q.B.flux[1], (size_t)(FR_COUNT * q.B.flux_stride[1]));
        q.st = b->st + p;
        if (e == cudaSuccess) {
            launch_fill_value(q.W[0], 4 * m.plane, 1.0, b->stream);
            launch_fill_value(q.W[1], 4 * m.plane, 1.0, b->stream);
            launch_fill_value(q.Ws, 4 * m.plane, 1.0, b->stream);
            launch_fill_value(q.A[0], m.plane, 1.0, b->stream);
            launch_fill_value(q.A[1], m.plane, 1.0, b->stream);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->dev, b->host.data(), (size_t)np * sizeof(BatchProblem), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->cfl, cfl.data(), (size_t)np * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) {
        for (int p = 0; p < np; ++p) {
            DevState z;
            memset(&z, 0, sizeof(z));
            z.dtmin_bits = 0x7FEFFFFFFFFFFFFFULL;
            z.fail_step = -1;
            z.fail_key = ~0ULL;
            b->st_host[p] = z;
        }
        e = cudaMemcpyAsync(b->st, b->st_host, (size_t)np * sizeof(DevState), cudaMemcpyHostToDevice, b->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    dfgks_status r = cst(e);
    if (r == DFGKS_OK) r = build_maps(b);
    if (r != DFGKS_OK) { free_batch(b); delete b; return r; }
    *out = b;
    return DFGKS_OK;
}

extern "C" DFGKS_API dfgks_status dfgks_batch_destroy(dfgks_batch* b) {
    if (!b) return DFGKS_OK;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    delete b;
    return DFGKS_OK;
}

// W host or device [4][ny][nx] for problem p; alpha^0 as in dfgks_set_ic (reconstruction with alpha = 1)
extern "C" DFGKS_API dfgks_status dfgks_batch_set_ic(dfgks_batch* b, int p, const double* W, int on_device) {
    if (!b || p < 0 || p >= b->np || !W) return DFGKS_EINVAL;
    BatchProblem& q = b->host[p];
    const Mesh& m = q.m;
    const size_t bytes = (size_t)4 * m.nx * m.ny * sizeof(double);
    BCK(cudaMemcpyAsync(q.acc, W, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->stream));
    int* bad = reinterpret_cast<int*>(q.B.flux[1]);          // scratch: a flux record plane is free here
    BCK(cudaMemsetAsync(bad, 0, sizeof(int), b->stream));
    launch_dense_to_ghosted(m, q.acc, 4, q.Ws, b->stream);
    launch_check_state(m, q.Ws, q.S.gm1, bad, b->stream);
    int hbad = 0;
    BCK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    if (hbad) return DFGKS_ENONPHYS;
    // the state starts in buffer 0
    launch_dense_to_ghosted(m, q.acc, 4, q.W[0], b->stream);
    launch_fill_value(q.A[0], m.plane, 1.0, b->stream);
    launch_fill_ghosts(m, q.W[0], nullptr, nullptr, b->stream);
    double* dts = q.acc;                                       // scratch scalar
    launch_set_scalar(dts, 1.0, b->stream);
    for (int d = 0; d < 2; ++d) launch_sweep(d, m, q.S, 1, true, q.W[0], q.A[0], dts, q.B, nullptr, nullptr, b->stream);
    UpdateArgs a;
    memset(&a, 0, sizeof(a));
    a.alpha_out = q.A[0];
    launch_update(UM_ALPHA, m, q.S, a, q.B, dts, nullptr, nullptr, b->stream);
    DevState z;
    memset(&z, 0, sizeof(z));
    z.dtmin_bits = 0x7FEFFFFFFFFFFFFFULL;
    z.fail_step = -1;
    z.fail_key = ~0ULL;
    b->st_host[p] = z;
    BCK(cudaMemcpyAsync(b->st + p, &b->st_host[p], sizeof(DevState), cudaMemcpyHostToDevice, b->stream));
    BCK(cudaGetLastError());
    BCK(cudaStreamSynchronize(b->stream));
    return DFGKS_OK;
}

extern "C" DFGKS_API dfgks_status dfgks_batch_get_state(dfgks_batch* b, int p, double* W, double* alpha, double* t,
                                                        long* step, int on_device) {
    if (!b || p < 0 || p >= b->np) return DFGKS_EINVAL;
    BCK(cudaMemcpyAsync(&b->st_host[p], b->st + p, sizeof(DevState), cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    const DevState hs = b->st_host[p];
    BatchProblem& q = b->host[p];
    const size_t n = (size_t)q.m.nx * q.m.ny;
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (W) {
        launch_ghosted_to_dense(q.m, q.W[hs.par], 4, q.acc, b->stream);
        BCK(cudaMemcpyAsync(W, q.acc, 4 * n * sizeof(double), kind, b->stream));
    }
    if (alpha) {
        launch_ghosted_to_dense(q.m, q.A[hs.par], 1, q.acc, b->stream);
        BCK(cudaMemcpyAsync(alpha, q.acc, n * sizeof(double), kind, b->stream));
    }
    BCK(cudaGetLastError());
    BCK(cudaStreamSynchronize(b->stream));
    if (t) *t = hs.t;
    if (step) *step = (long)hs.step;
    return DFGKS_OK;
}

// Capture the graph that advances every problem n steps (done by dfgks_batch_step on first use
// of that n; calling it ahead keeps the capture out of a timed region).
extern "C" DFGKS_API dfgks_status dfgks_batch_prepare(dfgks_batch* b, int n) {
    if (!b || n < 1 || n > 100000) return DFGKS_EINVAL;
    if (b->graph_ok && b->n_graph == n) return DFGKS_OK;
    return capture_steps(b, n);
}

// Advance every problem n steps (each with its own CFL dt).  use_graph != 0: one launch of a CUDA
// graph holding all n steps (captured on first use of this n).  Returns DFGKS_ENONPOS if any
// problem lost positivity (that problem stops at its last good step; the others continue).
extern "C" DFGKS_API dfgks_status dfgks_batch_step(dfgks_batch* b, int n, int use_graph) {
    if (!b || n < 0 || n > 100000) return DFGKS_EINVAL;
    if (n > 0 && use_graph) {
        if (!b->graph_ok || b->n_graph != n) {
            dfgks_status r = capture_steps(b, n);
            if (r != DFGKS_OK) return r;
        }
        BCK(cudaGraphLaunch(b->graph, b->stream));
    } else {
        for (int s = 0; s < n; ++s) enqueue_batch_step(b);
    }
    BCK(cudaGetLastError());
    BCK(cudaMemcpyAsync(b->st_host, b->st, (size_t)b->np * sizeof(DevState), cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    for (int p = 0; p < b->np; ++p) if (b->st_host[p].err) return DFGKS_ENONPOS;
    return DFGKS_OK;
}

static bool block_ok(int bs) { return bs == 64 || bs == 128 || bs == 256; }

// Threads per block (64, 128 or 256) of the face-line, tangential and flux kernels.
extern "C" DFGKS_API dfgks_status dfgks_batch_set_blocks(dfgks_batch* b, const int* blocks3) {
    if (!b || !blocks3) return DFGKS_EINVAL;
    for (int k = 0; k < 3; ++k) if (!block_ok(blocks3[k])) return DFGKS_EINVAL;
    for (int k = 0; k < 3; ++k) b->block[k] = blocks3[k];
    drop_graph(b);
    return build_maps(b);
}

// Autotuner: for each of the three sweep kernels in turn, time one batched step per candidate
// block size (64, 128, 256 threads) with the others fixed, keep the fastest.  The problems' states
// are saved before and restored after, so tuning does not advance them.  blocks3 receives the choice.
extern "C" DFGKS_API dfgks_status dfgks_batch_autotune(dfgks_batch* b, int* blocks3, double* best_ms) {
    if (!b) return DFGKS_EINVAL;
    // snapshot: both state buffers, both alpha buffers, DevStates
    std::vector<double*> saved;
    auto restore_or_save = [&](bool save) -> cudaError_t {
        size_t k = 0;
        for (int p = 0; p < b->np; ++p) {
            BatchProblem& q = b->host[p];
            double* bufs[4] = {q.W[0], q.W[1], q.A[0], q.A[1]};
            size_t sz[4] = {(size_t)(4 * q.m.plane), (size_t)(4 * q.m.plane), (size_t)q.m.plane, (size_t)q.m.plane};
            for (int i = 0; i < 4; ++i, ++k) {
                cudaError_t e;
                if (save) {
                    double* c = nullptr;
                    e = cudaMalloc((void**)&c, sz[i] * sizeof(double));
                    if (e != cudaSuccess) return e;
                    saved.push_back(c);
                    e = cudaMemcpyAsync(c, bufs[i], sz[i] * sizeof(double), cudaMemcpyDeviceToDevice, b->stream);
                } else {
                    e = cudaMemcpyAsync(bufs[i], saved[k], sz[i] * sizeof(double), cudaMemcpyDeviceToDevice, b->stream);
                }
                if (e != cudaSuccess) return e;
            }
        }
        return cudaSuccess;
    };
    BCK(cudaMemcpyAsync(b->st_host, b->st, (size_t)b->np * sizeof(DevState), cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    std::vector<DevState> st0(b->st_host, b->st_host + b->np);
    cudaError_t e = restore_or_save(true);
    if (e != cudaSuccess) { for (double* c : saved) cudaFree(c); return cst(e); }
    const int cand[3] = {64, 128, 256};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_total = 0.f;
    dfgks_status r = DFGKS_OK;
    for (int k = 0; k < 3 && r == DFGKS_OK; ++k) {
        float best = 1e30f;
        int keep = b->block[k];
        for (int c = 0; c < 3 && r == DFGKS_OK; ++c) {
            b->block[k] = cand[c];
            r = build_maps(b);
            if (r != DFGKS_OK) break;
            enqueue_batch_step(b);                           // warm-up
            cudaEventRecord(e0, b->stream);
            enqueue_batch_step(b);
            cudaEventRecord(e1, b->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) { r = DFGKS_ECUDA; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) { best = ms; keep = cand[c]; }
            // undo the two trial steps
            if (restore_or_save(false) != cudaSuccess) { r = DFGKS_ECUDA; break; }
            memcpy(b->st_host, st0.data(), (size_t)b->np * sizeof(DevState));
            if (cudaMemcpyAsync(b->st, b->st_host, (size_t)b->np * sizeof(DevState), cudaMemcpyHostToDevice, b->stream) != cudaSuccess) { r = DFGKS_ECUDA; break; }
            cudaStreamSynchronize(b->stream);
        }
        b->block[k] = keep;
        best_total = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(b->stream);
    for (double* c : saved) cudaFree(c);
    if (r != DFGKS_OK) return r;
    r = build_maps(b);
    drop_graph(b);
    if (blocks3) for (int k = 0; k < 3; ++k) blocks3[k] = b->block[k];
    if (best_ms) *best_ms = best_total;
    return r;
}

extern "C" DFGKS_API dfgks_status dfgks_batch_status(dfgks_batch* b, int p, long* step, int* err, unsigned long long* df_normal) {
    if (!b || p < 0 || p >= b->np) return DFGKS_EINVAL;
    BCK(cudaMemcpyAsync(&b->st_host[p], b->st + p, sizeof(DevState), cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    if (step) *step = (long)b->st_host[p].step;
    if (err) *err = b->st_host[p].err;
    if (df_normal) *df_normal = b->st_host[p].df_normal;
    return DFGKS_OK;
}
