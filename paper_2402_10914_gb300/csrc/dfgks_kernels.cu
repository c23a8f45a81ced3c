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
#include "dfgks_internal.h"
#include <float.h>

namespace dfk {

__device__ __forceinline__ bool halted(const int* halt) { return halt != nullptr && *(volatile const int*)halt != 0; }

// ---------------------------------------------------------------------------------------------
// Ghost fill: x pass over interior rows, then y pass over all columns (corners included)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int ghost_src(int k, int n, int lo, int hi, bool& mir) {
    mir = false;
    if (k < 0) {
        if (lo == 0) return k + n;
        if (lo == 1) return 0;
        mir = true; return -1 - k;
    }
    if (k >= n) {
        if (hi == 0) return k - n;
        if (hi == 1) return n - 1;
        mir = true; return 2 * n - 1 - k;
    }
    return k;
}

__global__ void k_ghost_x(Mesh m, double* W, double* alpha, const int* halt) {
    if (halted(halt)) return;
    int gc = threadIdx.x;                                  // 0 .. 2G-1
    int j = blockIdx.x * blockDim.y + threadIdx.y;
    if (gc >= 2 * G || j >= m.ny) return;
    int i = gc < G ? gc - G : m.nx + gc - G;
    bool mir;
    int s = ghost_src(i, m.nx, m.bc[0], m.bc[1], mir);
    long long d = gid(m, i, j), o = gid(m, s, j);
    if (W) {
#pragma unroll
        for (int k = 0; k < 4; ++k) W[k * m.plane + d] = W[k * m.plane + o];
        if (mir) W[1 * m.plane + d] = -W[1 * m.plane + d];
    }
    if (alpha) alpha[d] = alpha[o];
}

__global__ void k_ghost_y(Mesh m, double* W, double* alpha, const int* halt) {
    if (halted(halt)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x - G;    // -G .. nx+G-1
    int gr = blockIdx.y;                                   // 0 .. 2G-1
    if (i >= m.nx + G) return;
    int j = gr < G ? gr - G : m.ny + gr - G;
    bool mir;
    int s = ghost_src(j, m.ny, m.bc[2], m.bc[3], mir);
    long long d = gid(m, i, j), o = gid(m, i, s);
    if (W) {
#pragma unroll
        for (int k = 0; k < 4; ++k) W[k * m.plane + d] = W[k * m.plane + o];
        if (mir) W[2 * m.plane + d] = -W[2 * m.plane + d];
    }
    if (alpha) alpha[d] = alpha[o];
}

void launch_fill_ghosts(const Mesh& m, double* W, double* alpha, const int* halt, cudaStream_t s, KernelTimer* T) {
    if (T) T->begin(KK_OTHER);
    dim3 bx(2 * G, 32), gx((m.ny + 31) / 32);
    k_ghost_x<<<gx, bx, 0, s>>>(m, W, alpha, halt);
    dim3 by(128), gy((m.nx + 2 * G + 127) / 128, 2 * G);
    k_ghost_y<<<gy, by, 0, s>>>(m, W, alpha, halt);
    if (T) T->end(KK_OTHER, 2);
}

// ---------------------------------------------------------------------------------------------
// CFL time step (Algorithm 1, first line): min over cells of min(dx/(|U|+c), dy/(|V|+c))
// ---------------------------------------------------------------------------------------------
__global__ void k_cfl_min(Mesh m, const double* W, double gamma, DevState* st) {
    if (st->halt) return;
    double best = DBL_MAX;
    const int n = m.nx * m.ny;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        int i = c % m.nx, j = c / m.nx;
        long long g = gid(m, i, j);
        double r = W[g], U = W[m.plane + g] / r, V = W[2 * m.plane + g] / r;
        double p = (gamma - 1.0) * (W[3 * m.plane + g] - 0.5 * r * (U * U + V * V));
        double cs = sqrt(gamma * p / r);
        best = fmin(best, fmin(m.dx / (fabs(U) + cs), m.dy / (fabs(V) + cs)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
    __shared__ double red[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = best;
    __syncthreads();
    if (w == 0) {
        best = (lane < (int)(blockDim.x >> 5)) ? red[lane] : DBL_MAX;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
        // positive doubles order like their bit patterns; a non-positive or NaN bound (a
        // non-physical cell) is left out here and caught by the positivity checks
        if (lane == 0 && best > 0.0) atomicMin(&st->dtmin_bits, (unsigned long long)__double_as_longlong(best));
    }
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
template <int DIR>
struct Geo {
    int nn, nt;                  // cells along normal / tangential
    double dn, dtan;             // cell sizes along normal / tangential
    __device__ __forceinline__ Geo(const Mesh& m) {
        nn = DIR == 0 ? m.nx : m.ny;
        nt = DIR == 0 ? m.ny : m.nx;
        dn = DIR == 0 ? m.dx : m.dy;
        dtan = DIR == 0 ? m.dy : m.dx;
    }
    static constexpr int sigma = DIR == 0 ? 1 : -1;
    __device__ __forceinline__ long long cell(const Mesh& m, int n, int t) const {
        return DIR == 0 ? gid(m, n, t) : gid(m, t, n);
    }
    // line (f, t), t in [-2, nt+2): contiguous along the thread-x direction
    __device__ __forceinline__ long long line(int f, int t) const {
        return DIR == 0 ? (long long)(t + 2) * (nn + 1) + f : (long long)f * (nt + 4) + (t + 2);
    }
    // face (f, t), t in [0, nt)
    __device__ __forceinline__ long long face(int f, int t) const {
        return DIR == 0 ? (long long)t * (nn + 1) + f : (long long)f * nt + t;
    }
    __device__ __forceinline__ long long nfaces() const { return (long long)(nn + 1) * nt; }
};

__device__ __forceinline__ void warp_count_add(unsigned long long* dst, int v) {
    int s = __reduce_add_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(dst, (unsigned long long)s);
}

template <int DIR>
__global__ void __launch_bounds__(128) k_lines(Mesh m, SchemeConsts S, const double* __restrict__ W,
                                               const double* __restrict__ alpha, double* __restrict__ lines,
                                               long long ls, DevState* st, const int* halt) {
    if (halted(halt)) return;
    Geo<DIR> g(m);
    int ax = blockIdx.x * blockDim.x + threadIdx.x, ay = blockIdx.y * blockDim.y + threadIdx.y;
    int f = DIR == 0 ? ax : ay;
    int tt = DIR == 0 ? ay : ax;                           // t + 2
    bool active = f <= g.nn && tt < g.nt + 4;
    int ndf = 0;
    if (active) {
        const int t = tt - 2;
        double Wc[6][4];
        double al[6];
#pragma unroll
        for (int s = 0; s < 6; ++s) {
            long long c = g.cell(m, f - 3 + s, t);
#pragma unroll
            for (int k = 0; k < 4; ++k) Wc[s][k] = W[k * m.plane + c];
            to_local<DIR>(Wc[s]);
            al[s] = alpha[c];
        }
        CharBasis B = make_basis(Wc[2], Wc[3], S);
        double Q[6][4];
#pragma unroll
        for (int s = 0; s < 6; ++s) project(B, Wc[s], Q[s]);
        const bool dfL = fmax(fmax(al[1], al[2]), al[3]) < S.alpha_thres;     // Eq. 34, cell f-1
        const bool dfR = fmax(fmax(al[2], al[3]), al[4]) < S.alpha_thres;     // Eq. 34, cell f
        ndf = (int)dfL + (int)dfR;
        const double idn = 1.0 / g.dn;
        double qL[4], qLn[4], qR[4], qRn[4];
        double tl = 1.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double sL[5] = {Q[0][k], Q[1][k], Q[2][k], Q[3][k], Q[4][k]};
            double sR[5] = {Q[5][k], Q[4][k], Q[3][k], Q[2][k], Q[1][k]};   // mirrored about cell f
            double v, sl;
            if (!dfL || S.time_limiter) {
                AO o = weno_ao(sL, S, S.time_limiter);
                if (S.time_limiter) tl = fmin(tl, limiter_alpha(o, S.eps));
                if (!dfL) ao_at_right_edge(o, sL[2], v, sl);
            }
            if (dfL) df_at_right_edge(sL, al[2], v, sl);
            qL[k] = v; qLn[k] = sl * idn;
            if (!dfR || S.time_limiter) {
                AO o = weno_ao(sR, S, S.time_limiter);
                if (S.time_limiter) tl = fmin(tl, limiter_alpha(o, S.eps));
                if (!dfR) ao_at_right_edge(o, sR[2], v, sl);
            }
            if (dfR) df_at_right_edge(sR, al[3], v, sl);
            qR[k] = v; qRn[k] = -sl * idn;
        }
        double out[16];
        back_project(B, qL, out + LR_WL);
        back_project(B, qLn, out + LR_WLN);
        back_project(B, qR, out + LR_WR);
        back_project(B, qRn, out + LR_WRN);
        long long li = g.line(f, t);
#pragma unroll
        for (int q = 0; q < 16; ++q) lines[q * ls + li] = out[q];
        lines[LR_TL * ls + li] = tl;
        lines[LR_U * ls + li] = B.u;
        lines[LR_V * ls + li] = B.v;
        lines[LR_C * ls + li] = B.c;
        lines[LR_IC * ls + li] = B.ic;
        lines[LR_H * ls + li] = B.H;
        lines[LR_B1 * ls + li] = B.b1;
        lines[LR_B2 * ls + li] = B.b2;
        lines[LR_Q2 * ls + li] = B.q2;
    }
    if (st) warp_count_add(&st->df_normal, ndf);
}

template <int DIR>
__global__ void __launch_bounds__(128) k_faces(Mesh m, SchemeConsts S, const double* __restrict__ W,
                                               const double* __restrict__ alpha, const double* __restrict__ lines,
                                               long long ls, double* __restrict__ gp, long long gs,
                                               DevState* st, const int* halt) {
    if (halted(halt)) return;
    Geo<DIR> g(m);
    int ax = blockIdx.x * blockDim.x + threadIdx.x, ay = blockIdx.y * blockDim.y + threadIdx.y;
    const int side = blockIdx.z;
    int f = DIR == 0 ? ax : ay;
    int t = DIR == 0 ? ay : ax;
    bool active = f <= g.nn && t < g.nt;
    int ndf = 0, nfb = 0;
    if (active) {
        const long long l0 = g.line(f, t);
        CharBasis B;
        B.u = lines[LR_U * ls + l0]; B.v = lines[LR_V * ls + l0]; B.c = lines[LR_C * ls + l0];
        B.ic = lines[LR_IC * ls + l0]; B.H = lines[LR_H * ls + l0]; B.b1 = lines[LR_B1 * ls + l0];
        B.b2 = lines[LR_B2 * ls + l0]; B.q2 = lines[LR_Q2 * ls + l0];
        const int wbase = side == 0 ? LR_WL : LR_WR;
        double Q[5][4];
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            long long lb = g.line(f, t + Geo<DIR>::sigma * (b - 2));
            double Wl[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) Wl[k] = lines[(wbase + k) * ls + lb];
            project(B, Wl, Q[b]);
        }
        const int ncell = f - 1 + side;
        double al[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) al[b] = alpha[g.cell(m, ncell, t + Geo<DIR>::sigma * (b - 1))];
        const bool df = fmax(fmax(al[0], al[1]), al[2]) < S.alpha_thres;    // Eq. 34, tangential
        ndf = (int)df;
        double qv[2][4], qt[2][4];
        const double idt = 1.0 / g.dtan;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double sq[5] = {Q[0][k], Q[1][k], Q[2][k], Q[3][k], Q[4][k]};
            double v[2], s[2];
            if (df) df_at_gauss(sq, al[1], v, s);
            else { AO o = weno_ao(sq, S, false); ao_at_gauss(o, sq[2], v, s); }
            qv[0][k] = v[0]; qv[1][k] = v[1];
            qt[0][k] = s[0] * idt; qt[1][k] = s[1] * idt;
        }
        const long long e = (long long)side * g.nfaces() + g.face(f, t);
        const int nbase = side == 0 ? LR_WLN : LR_WRN;
#pragma unroll
        for (int mm = 0; mm < 2; ++mm) {
            double Wg[4], Wt[4], Wn[4];
            back_project(B, qv[mm], Wg);
            back_project(B, qt[mm], Wt);
#pragma unroll
            for (int k = 0; k < 4; ++k) Wn[k] = lines[(nbase + k) * ls + l0];
            if (S.gp_fallback && !physical_state(Wg, S.gm1)) {
                long long c = g.cell(m, ncell, t);
#pragma unroll
                for (int k = 0; k < 4; ++k) { Wg[k] = W[k * m.plane + c]; Wn[k] = 0.0; Wt[k] = 0.0; }
                to_local<DIR>(Wg);
                ++nfb;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                gp[(mm * 12 + k) * gs + e] = Wg[k];
                gp[(mm * 12 + 4 + k) * gs + e] = Wn[k];
                gp[(mm * 12 + 8 + k) * gs + e] = Wt[k];
            }
        }
    }
    if (st) { warp_count_add(&st->df_tangential, ndf); warp_count_add(&st->fallbacks, nfb); }
}

template <int DIR, int FLUX, bool ALPHA_ONLY>
__global__ void __launch_bounds__(128) k_flux(Mesh m, SchemeConsts S, const double* __restrict__ lines,
                                              long long ls, const double* __restrict__ gp, long long gs,
                                              double* __restrict__ fr, long long fs, const double* dtp,
                                              const int* halt) {
    if (halted(halt)) return;
    Geo<DIR> g(m);
    int ax = blockIdx.x * blockDim.x + threadIdx.x, ay = blockIdx.y * blockDim.y + threadIdx.y;
    const int mm = blockIdx.z;
    int f = DIR == 0 ? ax : ay;
    int t = DIR == 0 ? ay : ax;
    if (f > g.nn || t >= g.nt) return;
    const long long fid = g.face(f, t);
    const long long eL = fid, eR = g.nfaces() + fid;
    GPState L, R;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        L.W[k] = gp[(mm * 12 + k) * gs + eL];
        L.Wn[k] = gp[(mm * 12 + 4 + k) * gs + eL];
        L.Wt[k] = gp[(mm * 12 + 8 + k) * gs + eL];
        R.W[k] = gp[(mm * 12 + k) * gs + eR];
        R.Wn[k] = gp[(mm * 12 + 4 + k) * gs + eR];
        R.Wt[k] = gp[(mm * 12 + 8 + k) * gs + eR];
    }
    const long long e = (long long)mm * g.nfaces() + fid;
    fr[FR_ALPHA * fs + e] = df_alpha(L.W, R.W, S);
    if (ALPHA_ONLY) return;
    double F[4], dF[4];
    if (FLUX == 0) gks_flux(L, R, *dtp, S, F, dF);
    else lf_flux(L, R, S, F, dF);
    to_global<DIR>(F);
    to_global<DIR>(dF);
#pragma unroll
    for (int k = 0; k < 4; ++k) { fr[(FR_F + k) * fs + e] = F[k]; fr[(FR_DF + k) * fs + e] = dF[k]; }
    fr[FR_OMEGA * fs + e] = S.time_limiter ? lines[LR_TL * ls + g.line(f, t)] : 1.0;
}

template <int DIR>
static void sweep_dir(const Mesh& m, const SchemeConsts& S, int flux, bool alpha_only, const double* W,
                      const double* alpha, const double* dtp, const SweepBuffers& B, DevState* st,
                      const int* halt, cudaStream_t s, KernelTimer* T) {
    const int nn = DIR == 0 ? m.nx : m.ny, nt = DIR == 0 ? m.ny : m.nx;
    dim3 blk(32, 4);
    // lines: (nn+1) x (nt+4); faces/flux: (nn+1) x nt; thread-x runs along the contiguous index
    int lx = DIR == 0 ? nn + 1 : nt + 4, ly = DIR == 0 ? nt + 4 : nn + 1;
    dim3 gl((lx + 31) / 32, (ly + 3) / 4);
    if (T) T->begin(KK_LINES);
    k_lines<DIR><<<gl, blk, 0, s>>>(m, S, W, alpha, B.lines, B.line_stride, st, halt);
    if (T) T->end(KK_LINES, 1);
    int fx = DIR == 0 ? nn + 1 : nt, fy = DIR == 0 ? nt : nn + 1;
    dim3 gf((fx + 31) / 32, (fy + 3) / 4, 2);
    if (T) T->begin(KK_FACES);
    k_faces<DIR><<<gf, blk, 0, s>>>(m, S, W, alpha, B.lines, B.line_stride, B.gp, B.gp_stride, st, halt);
    if (T) T->end(KK_FACES, 1);
    double* fr = B.flux[DIR];
    long long fs = B.flux_stride[DIR];
    if (T) T->begin(KK_FLUX);
    if (alpha_only) k_flux<DIR, 1, true><<<gf, blk, 0, s>>>(m, S, B.lines, B.line_stride, B.gp, B.gp_stride, fr, fs, dtp, halt);
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
__device__ __forceinline__ void report_fail(DevState* st, int key) {
    atomicMin(&st->fail_key, (unsigned long long)key);
    if (atomicCAS(&st->err, 0, 5) == 0) st->fail_step = st->step;
    atomicExch(&st->halt, 1);
}

__device__ __forceinline__ bool state_ok(const double W[4], double gm1) {
    bool fin = isfinite(W[0]) && isfinite(W[1]) && isfinite(W[2]) && isfinite(W[3]);
    return fin && physical_state(W, gm1);
}

template <int MODE>
__global__ void __launch_bounds__(256) k_update(Mesh m, SchemeConsts S, UpdateArgs a,
                                                const double* __restrict__ frx, long long fsx,
                                                const double* __restrict__ fry, long long fsy,
                                                const double* dtp, DevState* st, const int* halt) {
    if (halted(halt)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= m.nx || j >= m.ny) return;
    const long long nfx = (long long)(m.nx + 1) * m.ny, nfy = (long long)(m.ny + 1) * m.nx;
    const long long fw = (long long)j * (m.nx + 1) + i, fe = fw + 1;
    const long long fsf = (long long)j * m.nx + i, fn = fsf + m.nx;
    // alpha product in the fixed order W(m1,m2), E, S, N
    double an = frx[FR_ALPHA * fsx + fw] * frx[FR_ALPHA * fsx + nfx + fw];
    an *= frx[FR_ALPHA * fsx + fe];
    an *= frx[FR_ALPHA * fsx + nfx + fe];
    an *= fry[FR_ALPHA * fsy + fsf];
    an *= fry[FR_ALPHA * fsy + nfy + fsf];
    an *= fry[FR_ALPHA * fsy + fn];
    an *= fry[FR_ALPHA * fsy + nfy + fn];
    const long long g = gid(m, i, j);
    const long long dn = (long long)j * m.nx + i, dplane = (long long)m.nx * m.ny;
    if (MODE == UM_ALPHA) {
        if (a.alpha_out) a.alpha_out[a.alpha_dense ? dn : g] = an;
        return;
    }
    double L[4], dL[4], dLt[4];
    const double ow = frx[FR_OMEGA * fsx + fw], oe = frx[FR_OMEGA * fsx + fe];
    const double os = fry[FR_OMEGA * fsy + fsf], on = fry[FR_OMEGA * fsy + fn];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double FW = 0.5 * frx[(FR_F + k) * fsx + fw] + 0.5 * frx[(FR_F + k) * fsx + nfx + fw];
        double FE = 0.5 * frx[(FR_F + k) * fsx + fe] + 0.5 * frx[(FR_F + k) * fsx + nfx + fe];
        double FS = 0.5 * fry[(FR_F + k) * fsy + fsf] + 0.5 * fry[(FR_F + k) * fsy + nfy + fsf];
        double FN = 0.5 * fry[(FR_F + k) * fsy + fn] + 0.5 * fry[(FR_F + k) * fsy + nfy + fn];
        double DW = 0.5 * frx[(FR_DF + k) * fsx + fw] + 0.5 * frx[(FR_DF + k) * fsx + nfx + fw];
        double DE = 0.5 * frx[(FR_DF + k) * fsx + fe] + 0.5 * frx[(FR_DF + k) * fsx + nfx + fe];
        double DS = 0.5 * fry[(FR_DF + k) * fsy + fsf] + 0.5 * fry[(FR_DF + k) * fsy + nfy + fsf];
        double DN = 0.5 * fry[(FR_DF + k) * fsy + fn] + 0.5 * fry[(FR_DF + k) * fsy + nfy + fn];
        L[k] = -(FE - FW) / m.dx - (FN - FS) / m.dy;
        dL[k] = -(DE - DW) / m.dx - (DN - DS) / m.dy;
        dLt[k] = -(oe * DE - ow * DW) / m.dx - (on * DN - os * DS) / m.dy;
    }
    if (MODE == UM_RESIDUAL) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (a.L) a.L[k * dplane + dn] = L[k];
            if (a.dtL) a.dtL[k * dplane + dn] = dL[k];
            if (a.dtLt) a.dtLt[k * dplane + dn] = dLt[k];
        }
        if (a.alpha_out) a.alpha_out[a.alpha_dense ? dn : g] = an;
        return;
    }
    const double dt = *dtp;
    double Wo[4];
    if (MODE == UM_S2O4_1) {
        double Ws[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double w = a.Win[k * m.plane + g];
            Ws[k] = w + 0.5 * dt * L[k] + 0.125 * dt * dt * dL[k];
            a.acc[k * dplane + dn] = w + dt * L[k] + 0.5 * dt * dt * dL[k] - (1.0 / 3.0) * dt * dt * dLt[k];
            a.Wout[k * m.plane + g] = Ws[k];
        }
        if (!state_ok(Ws, S.gm1)) report_fail(st, (int)dn);
        return;
    }
    if (MODE == UM_S2O4_2) {
#pragma unroll
        for (int k = 0; k < 4; ++k) Wo[k] = a.acc[k * dplane + dn] + (1.0 / 3.0) * dt * dt * dLt[k];
    } else if (MODE == UM_RK_1) {
#pragma unroll
        for (int k = 0; k < 4; ++k) Wo[k] = a.Win[k * m.plane + g] + dt * L[k];
    } else if (MODE == UM_RK_2) {
#pragma unroll
        for (int k = 0; k < 4; ++k) Wo[k] = 0.75 * a.Wn[k * m.plane + g] + 0.25 * a.Win[k * m.plane + g] + 0.25 * dt * L[k];
    } else {  // UM_RK_3
#pragma unroll
        for (int k = 0; k < 4; ++k)
            Wo[k] = (1.0 / 3.0) * a.Wn[k * m.plane + g] + (2.0 / 3.0) * a.Win[k * m.plane + g] + (2.0 / 3.0) * dt * L[k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) a.Wout[k * m.plane + g] = Wo[k];
    if ((MODE == UM_S2O4_2 || MODE == UM_RK_3) && a.alpha_out) a.alpha_out[a.alpha_dense ? dn : g] = an;
    if (!state_ok(Wo, S.gm1)) report_fail(st, (int)dn);
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
