// dfgks_kernels.cu -- sm_103a kernels of one step of Algorithm 1 (arXiv 2402.10914):
//   ghost fill -> CFL dt -> per stage and per direction:
//     k_lines  : one thread per face line, normal WENO-AO / DF reconstruction of both sides
//                (characteristic variables of the line's mean state)           [Sect. 3.1, 3.3]
//     k_faces  : one thread per face side, tangential reconstruction at the two Gauss points,
//                Gauss-point fallback                                         [Sect. 3, Alg. 1]
//     k_flux   : one thread per Gauss point, GKS or L-F flux and its time derivative, DF factor
//                                                                             [Sect. 2.2, 2.3, 3.2]
//   -> k_update: one thread per cell, Eq. 2 residual, time limiter, S2O4 / SSP-RK3 combination,
//                alpha^{n+1} product, positivity check.                       [Sect. 2.1-2.3]
// The path is bound by the FP64 pipe: line results are computed once and shared through the
// (L2-resident) line buffer by the five tangential stencils that read them.
#include "dfgks_bodies.cuh"

namespace dfk {

__device__ __forceinline__ bool halted(const int* halt) { return halt != nullptr && *(volatile const int*)halt != 0; }

// ---------------------------------------------------------------------------------------------
// Ghost fill: x pass over interior rows, then y pass over all columns (corners included)
// ---------------------------------------------------------------------------------------------
__global__ void k_ghost_x(Mesh m, double* W, double* alpha, const int* halt) {
    if (halted(halt)) return;
    ghost_x_body(m, W, alpha, threadIdx.x, blockIdx.x * blockDim.y + threadIdx.y);
}

__global__ void k_ghost_y(Mesh m, double* W, double* alpha, const int* halt) {
    if (halted(halt)) return;
    ghost_y_body(m, W, alpha, blockIdx.x * blockDim.x + threadIdx.x - G, blockIdx.y);
}

void launch_ghost_pass(int dir, const Mesh& m, double* W, double* alpha, const int* halt, cudaStream_t s) {
    if (dir == 0) {
        dim3 bx(2 * G, 32), gx((m.ny + 31) / 32);
        k_ghost_x<<<gx, bx, 0, s>>>(m, W, alpha, halt);
    } else {
        dim3 by(128), gy((m.nx + 2 * G + 127) / 128, 2 * G);
        k_ghost_y<<<gy, by, 0, s>>>(m, W, alpha, halt);
    }
}

void launch_fill_ghosts(const Mesh& m, double* W, double* alpha, const int* halt, cudaStream_t s, KernelTimer* T) {
    if (T) T->begin(KK_OTHER);
    launch_ghost_pass(0, m, W, alpha, halt, s);
    launch_ghost_pass(1, m, W, alpha, halt, s);
    if (T) T->end(KK_OTHER, 2);
}

// ---------------------------------------------------------------------------------------------
// CFL time step (Algorithm 1, first line): min over cells of min(dx/(|U|+c), dy/(|V|+c))
// ---------------------------------------------------------------------------------------------
__global__ void k_cfl_min(Mesh m, const double* W, double gamma, DevState* st) {
    if (st->halt) return;
    double best = DBL_MAX;
    const int n = m.nx * m.ny;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        best = fmin(best, cfl_cell(m, W, gamma, c));
    best = block_min(best);
    // positive doubles order like their bit patterns; a non-positive or NaN bound (a
    // non-physical cell) is left out here and caught by the positivity checks
    if (threadIdx.x == 0 && best > 0.0) atomicMin(&st->dtmin_bits, (unsigned long long)__double_as_longlong(best));
}

void launch_cfl_min(const Mesh& m, const double* W, double gamma, DevState* st, cudaStream_t s, KernelTimer* T) {
    int n = m.nx * m.ny;
    int blocks = (n + 255) / 256;
    if (blocks > 4 * 152) blocks = 4 * 152;
    if (T) T->begin(KK_OTHER);
    k_cfl_min<<<blocks, 256, 0, s>>>(m, W, gamma, st);
    if (T) T->end(KK_OTHER, 1);
}

__global__ void k_begin_step(DevState* st, double cfl, double dt_fixed, double t_end, double* dts, int idx) {
    // consume and reset the CFL accumulator first, so a halted step leaves it clean
    const double dtmin = __longlong_as_double((long long)st->dtmin_bits);
    st->dtmin_bits = (unsigned long long)__double_as_longlong(DBL_MAX);
    if (st->halt) return;
    if (t_end > 0.0 && st->t >= t_end) { st->halt = 1; return; }
    double dt = dt_fixed > 0.0 ? dt_fixed : cfl * dtmin;
    st->clipped = 0;
    // last step: clip to t_end; a remainder below 1e-12 relative is absorbed into this step
    if (t_end > 0.0 && st->t + dt >= t_end - 1e-12 * fabs(t_end)) { dt = t_end - st->t; st->clipped = 1; }
    st->dt = dt;
    if (dts) dts[idx] = dt;
}

__global__ void k_end_step(DevState* st, double t_end) {
    if (st->halt) return;
    st->t = st->clipped ? t_end : st->t + st->dt;
    st->step += 1;
}

void launch_begin_step(DevState* st, double cfl, double dt_fixed, double t_end, double* dts, int idx, cudaStream_t s,
                       KernelTimer* T) {
    k_begin_step<<<1, 1, 0, s>>>(st, cfl, dt_fixed, t_end, dts, idx);
    if (T) T->end(KK_OTHER, 1);
}
void launch_end_step(DevState* st, double t_end, cudaStream_t s, KernelTimer* T) {
    k_end_step<<<1, 1, 0, s>>>(st, t_end);
    if (T) T->end(KK_OTHER, 1);
}

// ---------------------------------------------------------------------------------------------
// Sweep geometry of one direction.  DIR 0: x-faces, normal index = i, tangential index = j.
// DIR 1: y-faces in the frame rotated by pi/2: normal = +y, tangential = -x, so the local
// tangential offset b maps to global column t - b.  Face f lies between normal cells f-1, f.
// ---------------------------------------------------------------------------------------------
template <int DIR, bool TAPE = false>
__global__ void __launch_bounds__(128, 3) k_lines(Mesh m, SchemeConsts S, const double* __restrict__ W,
                                               const double* __restrict__ alpha, double* __restrict__ lines,
                                               long long ls, DevState* st, const int* halt,
                                               double* __restrict__ ltape = nullptr) {
    if (halted(halt)) return;
    int ax, ay;
    sweep_xy(lines_lx<DIR>(m), ax, ay);
    int ndf = lines_body<DIR, TAPE>(m, S, W, alpha, lines, ls, ax, ay, ltape);
    if (st) warp_count_add(&st->df_normal, ndf);
}

template <int DIR, bool TAPE = false>
__global__ void __launch_bounds__(128) k_faces(Mesh m, SchemeConsts S, const double* __restrict__ W,
                                               const double* __restrict__ alpha, const double* __restrict__ lines,
                                               long long ls, double* __restrict__ gp, long long gs,
                                               DevState* st, const int* halt, double* __restrict__ ftape = nullptr) {
    if (halted(halt)) return;
    int nfb, ax, ay;
    sweep_xy(faces_lx<DIR>(m), ax, ay);
    int ndf = faces_body<DIR, TAPE>(m, S, W, alpha, lines, ls, gp, gs, ax, ay, blockIdx.y, nfb, ftape);
    if (st) { warp_count_add(&st->df_tangential, ndf); warp_count_add(&st->fallbacks, nfb); }
}

template <int DIR, int FLUX, bool ALPHA_ONLY, bool TAPE = false>
__global__ void __launch_bounds__(128) k_flux(Mesh m, SchemeConsts S, const double* __restrict__ lines,
                                              long long ls, const double* __restrict__ gp, long long gs,
                                              double* __restrict__ fr, long long fs, const double* dtp,
                                              const int* halt, double* __restrict__ tape = nullptr) {
    if (halted(halt)) return;
    int ax, ay;
    sweep_xy(faces_lx<DIR>(m), ax, ay);
    flux_body<DIR, FLUX, ALPHA_ONLY, TAPE>(m, S, lines, ls, gp, gs, fr, fs, ALPHA_ONLY ? 0.0 : *dtp, ax, ay,
                                           blockIdx.y, tape);
}

// ---------------------------------------------------------------------------------------------
// Both directions of a sweep in one launch: blocks [0, nb0) take the x-faces' index space, the
// rest the y-faces', each on its own face-line and Gauss-point buffers.  The two halves are
// independent; one launch of twice the blocks evens out the last round of blocks over the SMs and
// saves three launches per stage.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void sweep_at(int b, int lx, int& ax, int& ay) {
    const int i = b * (int)blockDim.x + (int)threadIdx.x;
    ax = i % lx;
    ay = i / lx;
}

template <bool TAPE>
__global__ void __launch_bounds__(128, 3) k_lines_xy(Mesh m, SchemeConsts S, const double* __restrict__ W,
                                                  const double* __restrict__ alpha, double* __restrict__ lines0,
                                                  double* __restrict__ lines1, long long ls, double* __restrict__ ltape0,
                                                  double* __restrict__ ltape1, int nb0, DevState* st, const int* halt) {
    if (halted(halt)) return;
    int ax, ay, ndf;
    if ((int)blockIdx.x < nb0) {
        sweep_at(blockIdx.x, lines_lx<0>(m), ax, ay);
        ndf = lines_body<0, TAPE>(m, S, W, alpha, lines0, ls, ax, ay, ltape0);
    } else {
        sweep_at(blockIdx.x - nb0, lines_lx<1>(m), ax, ay);
        ndf = lines_body<1, TAPE>(m, S, W, alpha, lines1, ls, ax, ay, ltape1);
    }
    if (st) warp_count_add(&st->df_normal, ndf);
}

template <bool TAPE>
__global__ void __launch_bounds__(128) k_faces_xy(Mesh m, SchemeConsts S, const double* __restrict__ W,
                                               const double* __restrict__ alpha, const double* __restrict__ lines0,
                                               const double* __restrict__ lines1, long long ls, double* __restrict__ gp0,
                                               double* __restrict__ gp1, long long gs, double* __restrict__ ftape0,
                                               double* __restrict__ ftape1, int nb0, DevState* st, const int* halt) {
    if (halted(halt)) return;
    int nfb, ax, ay, ndf;
    if ((int)blockIdx.x < nb0) {
        sweep_at(blockIdx.x, faces_lx<0>(m), ax, ay);
        ndf = faces_body<0, TAPE>(m, S, W, alpha, lines0, ls, gp0, gs, ax, ay, blockIdx.y, nfb, ftape0);
    } else {
        sweep_at(blockIdx.x - nb0, faces_lx<1>(m), ax, ay);
        ndf = faces_body<1, TAPE>(m, S, W, alpha, lines1, ls, gp1, gs, ax, ay, blockIdx.y, nfb, ftape1);
    }
    if (st) { warp_count_add(&st->df_tangential, ndf); warp_count_add(&st->fallbacks, nfb); }
}

template <int FLUX, bool ALPHA_ONLY, bool TAPE = false>
__global__ void __launch_bounds__(128) k_flux_xy(Mesh m, SchemeConsts S, const double* __restrict__ lines0,
                                              const double* __restrict__ lines1, long long ls,
                                              const double* __restrict__ gp0, const double* __restrict__ gp1,
                                              long long gs, double* __restrict__ fr0, long long fs0,
                                              double* __restrict__ fr1, long long fs1, double* __restrict__ tape0,
                                              double* __restrict__ tape1, const double* dtp, int nb0, const int* halt) {
    if (halted(halt)) return;
    const double dt = ALPHA_ONLY ? 0.0 : *dtp;
    // the direction selects the records and the index map; the flux arithmetic is inlined once
    int ax, ay, dir;
    FluxSite site;
    if ((int)blockIdx.x < nb0) {
        sweep_at(blockIdx.x, faces_lx<0>(m), ax, ay);
        site = flux_site<0>(m, ax, ay, blockIdx.y);
        dir = 0;
    } else {
        sweep_at(blockIdx.x - nb0, faces_lx<1>(m), ax, ay);
        site = flux_site<1>(m, ax, ay, blockIdx.y);
        dir = 1;
    }
    if (!site.ok) return;
    flux_point<FLUX, ALPHA_ONLY, TAPE>(dir, S, site, dir == 0 ? lines0 : lines1, ls, dir == 0 ? gp0 : gp1, gs,
                                       dir == 0 ? fr0 : fr1, dir == 0 ? fs0 : fs1, dt, blockIdx.y,
                                       dir == 0 ? tape0 : tape1);
}

void launch_sweep_xy(const Mesh& m, const SchemeConsts& S, int flux, bool alpha_only, const double* W,
                     const double* alpha, const double* dtp, const SweepBuffers& Bx, const SweepBuffers& By,
                     DevState* st, const int* halt, cudaStream_t s, KernelTimer* T) {
    const dim3 blk(128);
    const int nl0 = (int)sweep_blocks(lines_lx<0>(m), lines_ly<0>(m)), nl1 = (int)sweep_blocks(lines_lx<1>(m), lines_ly<1>(m));
    const int nf0 = (int)sweep_blocks(faces_lx<0>(m), faces_ly<0>(m)), nf1 = (int)sweep_blocks(faces_lx<1>(m), faces_ly<1>(m));
    const bool tape = Bx.ltape != nullptr;      // both directions' record sets carry tapes or neither
    const long long ls = Bx.line_stride, gs = Bx.gp_stride;
    if (T) T->begin(KK_LINES);
    if (tape)
        k_lines_xy<true><<<dim3(nl0 + nl1), blk, 0, s>>>(m, S, W, alpha, Bx.lines, By.lines, ls, Bx.ltape, By.ltape, nl0,
                                                         st, halt);
    else
        k_lines_xy<false><<<dim3(nl0 + nl1), blk, 0, s>>>(m, S, W, alpha, Bx.lines, By.lines, ls, nullptr, nullptr, nl0,
                                                          st, halt);
    if (T) T->end(KK_LINES, 1);
    const dim3 gf(nf0 + nf1, 2);
    if (T) T->begin(KK_FACES);
    if (tape)
        k_faces_xy<true><<<gf, blk, 0, s>>>(m, S, W, alpha, Bx.lines, By.lines, ls, Bx.gp, By.gp, gs, Bx.ftape,
                                            By.ftape, nf0, st, halt);
    else
        k_faces_xy<false><<<gf, blk, 0, s>>>(m, S, W, alpha, Bx.lines, By.lines, ls, Bx.gp, By.gp, gs, nullptr,
                                             nullptr, nf0, st, halt);
    if (T) T->end(KK_FACES, 1);
    double* f0 = Bx.flux[0];
    double* f1 = By.flux[1];
    const long long fs0 = Bx.flux_stride[0], fs1 = By.flux_stride[1];
    if (T) T->begin(KK_FLUX);
    if (alpha_only)
        k_flux_xy<1, true><<<gf, blk, 0, s>>>(m, S, Bx.lines, By.lines, ls, Bx.gp, By.gp, gs, f0, fs0, f1, fs1,
                                               nullptr, nullptr, dtp, nf0, halt);
    else if (flux == 0 && Bx.tape[0])        // GKS forward that also tapes its intermediates for a reverse sweep
        k_flux_xy<0, false, true><<<gf, blk, 0, s>>>(m, S, Bx.lines, By.lines, ls, Bx.gp, By.gp, gs, f0, fs0, f1, fs1,
                                                     Bx.tape[0], By.tape[1], dtp, nf0, halt);
    else if (flux == 0)
        k_flux_xy<0, false><<<gf, blk, 0, s>>>(m, S, Bx.lines, By.lines, ls, Bx.gp, By.gp, gs, f0, fs0, f1, fs1,
                                                nullptr, nullptr, dtp, nf0, halt);
    else
        k_flux_xy<1, false><<<gf, blk, 0, s>>>(m, S, Bx.lines, By.lines, ls, Bx.gp, By.gp, gs, f0, fs0, f1, fs1,
                                                nullptr, nullptr, dtp, nf0, halt);
    if (T) T->end(KK_FLUX, 1);
}

template <int DIR>
static void sweep_dir(const Mesh& m, const SchemeConsts& S, int flux, bool alpha_only, const double* W,
                      const double* alpha, const double* dtp, const SweepBuffers& B, DevState* st,
                      const int* halt, cudaStream_t s, KernelTimer* T) {
    // 1-D grids over the row-major index spaces of face lines ((nn+1) x (nt+4)) and of face sides /
    // Gauss points ((nn+1) x nt, two of each per face: grid y); rows run along the contiguous index
    const dim3 blk(128);
    const dim3 gl(sweep_blocks(lines_lx<DIR>(m), lines_ly<DIR>(m)));
    if (T) T->begin(KK_LINES);
    if (B.ltape) k_lines<DIR, true><<<gl, blk, 0, s>>>(m, S, W, alpha, B.lines, B.line_stride, st, halt, B.ltape);
    else k_lines<DIR><<<gl, blk, 0, s>>>(m, S, W, alpha, B.lines, B.line_stride, st, halt);
    if (T) T->end(KK_LINES, 1);
    const dim3 gf(sweep_blocks(faces_lx<DIR>(m), faces_ly<DIR>(m)), 2);
    if (T) T->begin(KK_FACES);
    if (B.ftape)
        k_faces<DIR, true><<<gf, blk, 0, s>>>(m, S, W, alpha, B.lines, B.line_stride, B.gp, B.gp_stride, st, halt, B.ftape);
    else
        k_faces<DIR><<<gf, blk, 0, s>>>(m, S, W, alpha, B.lines, B.line_stride, B.gp, B.gp_stride, st, halt);
    if (T) T->end(KK_FACES, 1);
    double* fr = B.flux[DIR];
    long long fs = B.flux_stride[DIR];
    if (T) T->begin(KK_FLUX);
    if (alpha_only) k_flux<DIR, 1, true><<<gf, blk, 0, s>>>(m, S, B.lines, B.line_stride, B.gp, B.gp_stride, fr, fs, dtp, halt);
    else if (flux == 0 && B.tape[DIR])      // GKS forward that also tapes its intermediates for a reverse sweep
        k_flux<DIR, 0, false, true><<<gf, blk, 0, s>>>(m, S, B.lines, B.line_stride, B.gp, B.gp_stride, fr, fs, dtp, halt,
                                                       B.tape[DIR]);
    else if (flux == 0) k_flux<DIR, 0, false><<<gf, blk, 0, s>>>(m, S, B.lines, B.line_stride, B.gp, B.gp_stride, fr, fs, dtp, halt);
    else k_flux<DIR, 1, false><<<gf, blk, 0, s>>>(m, S, B.lines, B.line_stride, B.gp, B.gp_stride, fr, fs, dtp, halt);
    if (T) T->end(KK_FLUX, 1);
}

void launch_sweep(int dir, const Mesh& m, const SchemeConsts& S, int flux, bool alpha_only,
                  const double* W, const double* alpha, const double* dtp, const SweepBuffers& B,
                  DevState* st, const int* halt, cudaStream_t s, KernelTimer* T) {
    if (dir == 0) sweep_dir<0>(m, S, flux, alpha_only, W, alpha, dtp, B, st, halt, s, T);
    else sweep_dir<1>(m, S, flux, alpha_only, W, alpha, dtp, B, st, halt, s, T);
}

// ---------------------------------------------------------------------------------------------
// Stage update: Eq. 2 with two Gauss points per face, the limited time derivative, the S2O4 or
// SSP-RK3 combination, alpha^{n+1} = product of the cell's 8 Gauss-point DF factors.
// ---------------------------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256) k_update(Mesh m, SchemeConsts S, UpdateArgs a,
                                                const double* __restrict__ frx, long long fsx,
                                                const double* __restrict__ fry, long long fsy,
                                                const double* dtp, DevState* st, const int* halt) {
    if (halted(halt)) return;
    const double dt = (MODE == UM_RESIDUAL || MODE == UM_ALPHA) ? 0.0 : *dtp;
    update_body<MODE>(m, S, a, frx, fsx, fry, fsy, dt, st, blockIdx.x * blockDim.x + threadIdx.x,
                      blockIdx.y * blockDim.y + threadIdx.y);
}

void launch_update(int mode, const Mesh& m, const SchemeConsts& S, const UpdateArgs& a, const SweepBuffers& B,
                   const double* dtp, DevState* st, const int* halt, cudaStream_t s, KernelTimer* T) {
    dim3 blk(32, 8), grd((m.nx + 31) / 32, (m.ny + 7) / 8);
    if (T) T->begin(KK_UPDATE);
    const double* fx = B.flux[0];
    const double* fy = B.flux[1];
    long long sx = B.flux_stride[0], sy = B.flux_stride[1];
    switch (mode) {
        case UM_RESIDUAL: k_update<UM_RESIDUAL><<<grd, blk, 0, s>>>(m, S, a, fx, sx, fy, sy, dtp, st, halt); break;
        case UM_S2O4_1: k_update<UM_S2O4_1><<<grd, blk, 0, s>>>(m, S, a, fx, sx, fy, sy, dtp, st, halt); break;
        case UM_S2O4_2: k_update<UM_S2O4_2><<<grd, blk, 0, s>>>(m, S, a, fx, sx, fy, sy, dtp, st, halt); break;
        case UM_RK_1: k_update<UM_RK_1><<<grd, blk, 0, s>>>(m, S, a, fx, sx, fy, sy, dtp, st, halt); break;
        case UM_RK_2: k_update<UM_RK_2><<<grd, blk, 0, s>>>(m, S, a, fx, sx, fy, sy, dtp, st, halt); break;
        case UM_RK_3: k_update<UM_RK_3><<<grd, blk, 0, s>>>(m, S, a, fx, sx, fy, sy, dtp, st, halt); break;
        default: k_update<UM_ALPHA><<<grd, blk, 0, s>>>(m, S, a, fx, sx, fy, sy, dtp, st, halt); break;
    }
    if (T) T->end(KK_UPDATE, 1);
}

// ---------------------------------------------------------------------------------------------
// Layout helpers
// ---------------------------------------------------------------------------------------------
__global__ void k_dense_to_ghosted(Mesh m, const double* __restrict__ d, int nc, double* __restrict__ g) {
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= m.nx || j >= m.ny) return;
    const long long dp = (long long)m.nx * m.ny;
    for (int k = 0; k < nc; ++k) g[k * m.plane + gid(m, i, j)] = d[k * dp + (long long)j * m.nx + i];
}
__global__ void k_ghosted_to_dense(Mesh m, const double* __restrict__ g, int nc, double* __restrict__ d) {
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= m.nx || j >= m.ny) return;
    const long long dp = (long long)m.nx * m.ny;
    for (int k = 0; k < nc; ++k) d[k * dp + (long long)j * m.nx + i] = g[k * m.plane + gid(m, i, j)];
}
void launch_dense_to_ghosted(const Mesh& m, const double* dense, int nc, double* ghosted, cudaStream_t s) {
    dim3 blk(32, 8), grd((m.nx + 31) / 32, (m.ny + 7) / 8);
    k_dense_to_ghosted<<<grd, blk, 0, s>>>(m, dense, nc, ghosted);
}
void launch_ghosted_to_dense(const Mesh& m, const double* ghosted, int nc, double* dense, cudaStream_t s) {
    dim3 blk(32, 8), grd((m.nx + 31) / 32, (m.ny + 7) / 8);
    k_ghosted_to_dense<<<grd, blk, 0, s>>>(m, ghosted, nc, dense);
}

__global__ void k_fill_value(double* p, long long n, double v) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) p[q] = v;
}
void launch_fill_value(double* p, long long n, double v, cudaStream_t s) {
    long long b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    k_fill_value<<<(unsigned)b, 256, 0, s>>>(p, n, v);
}

__global__ void k_check_state(Mesh m, const double* __restrict__ W, double gm1, int* bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= m.nx || j >= m.ny) return;
    long long g = gid(m, i, j);
    double w[4] = {W[g], W[m.plane + g], W[2 * m.plane + g], W[3 * m.plane + g]};
    if (!state_ok(w, gm1)) atomicExch(bad, 1);
}
void launch_check_state(const Mesh& m, const double* W, double gm1, int* bad, cudaStream_t s) {
    dim3 blk(32, 8), grd((m.nx + 31) / 32, (m.ny + 7) / 8);
    k_check_state<<<grd, blk, 0, s>>>(m, W, gm1, bad);
}

__global__ void k_set_scalar(double* p, double v) { *p = v; }
void launch_set_scalar(double* p, double v, cudaStream_t s) { k_set_scalar<<<1, 1, 0, s>>>(p, v); }

// 59 doubles per face: F, dF (Gauss-averaged, global frame), omega, alpha_1, alpha_2, then
// side x Gauss point x {W, Wn, Wt} in the local frame
template <int DIR>
__global__ void k_pack_faces(Mesh m, const double* __restrict__ gp, long long gs, const double* __restrict__ fr,
                             long long fs, double* __restrict__ out) {
    Geo<DIR> g(m);
    long long nf = g.nfaces();
    long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= nf) return;
    // output order: DIR 0 [ny][nx+1], DIR 1 [nx][ny+1] -- the oracle's (t, f) order
    int t = (int)(q / (g.nn + 1)), f = (int)(q % (g.nn + 1));
    long long fid = g.face(f, t);
    double* o = out + q * 59;
    for (int k = 0; k < 4; ++k) {
        o[k] = 0.5 * fr[(FR_F + k) * fs + fid] + 0.5 * fr[(FR_F + k) * fs + nf + fid];
        o[4 + k] = 0.5 * fr[(FR_DF + k) * fs + fid] + 0.5 * fr[(FR_DF + k) * fs + nf + fid];
    }
    o[8] = fr[FR_OMEGA * fs + fid];
    o[9] = fr[FR_ALPHA * fs + fid];
    o[10] = fr[FR_ALPHA * fs + nf + fid];
    int c = 11;
    for (int side = 0; side < 2; ++side)
        for (int mm = 0; mm < 2; ++mm)
            for (int fld = 0; fld < 12; ++fld) o[c++] = gp[(mm * 12 + fld) * gs + side * nf + fid];
}
void launch_pack_faces(int dir, const Mesh& m, const SweepBuffers& B, double* out, cudaStream_t s) {
    long long nf = dir == 0 ? (long long)(m.nx + 1) * m.ny : (long long)(m.ny + 1) * m.nx;
    unsigned blocks = (unsigned)((nf + 127) / 128);
    if (dir == 0) k_pack_faces<0><<<blocks, 128, 0, s>>>(m, B.gp, B.gp_stride, B.flux[0], B.flux_stride[0], out);
    else k_pack_faces<1><<<blocks, 128, 0, s>>>(m, B.gp, B.gp_stride, B.flux[1], B.flux_stride[1], out);
}

}  // namespace dfk
