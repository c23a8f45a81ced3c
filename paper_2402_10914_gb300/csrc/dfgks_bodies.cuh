// dfgks_bodies.cuh -- per-thread bodies of the step kernels (one face line, face side, Gauss point,
// cell or ghost cell), shared by the single-problem kernels (dfgks_kernels.cu) and the batched
// kernels (dfgks_batch.cu), so both run exactly the same arithmetic.  The bodies are also
// host-callable, so a test can run the GPU path's per-thread arithmetic on the CPU.
#pragma once
#include <float.h>
#include "dfgks_internal.h"

namespace dfk {

DFK_HD int ghost_src(int k, int n, int lo, int hi, bool& mir) {
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

template <int DIR>
struct Geo {
    int nn, nt;                  // cells along normal / tangential
    double dn, dtan;             // cell sizes along normal / tangential
    double idn, idtan;           // their reciprocals
    DFK_HD Geo(const Mesh& m) {
        nn = DIR == 0 ? m.nx : m.ny;
        nt = DIR == 0 ? m.ny : m.nx;
        dn = DIR == 0 ? m.dx : m.dy;
        dtan = DIR == 0 ? m.dy : m.dx;
        idn = DIR == 0 ? m.rdx : m.rdy;
        idtan = DIR == 0 ? m.rdy : m.rdx;
    }
    static constexpr int sigma = DIR == 0 ? 1 : -1;
    DFK_HD long long cell(const Mesh& m, int n, int t) const {
        return DIR == 0 ? gid(m, n, t) : gid(m, t, n);
    }
    // line (f, t), t in [-2, nt+2): contiguous along the thread-x direction
    DFK_HD long long line(int f, int t) const {
        return DIR == 0 ? (long long)(t + 2) * (nn + 1) + f : (long long)f * (nt + 4) + (t + 2);
    }
    // face (f, t), t in [0, nt)
    DFK_HD long long face(int f, int t) const {
        return DIR == 0 ? (long long)t * (nn + 1) + f : (long long)f * nt + t;
    }
    DFK_HD long long nfaces() const { return (long long)(nn + 1) * nt; }
};

// Index spaces of the sweep kernels, row-major, rows lx wide (the thread-x direction of the bodies):
// face lines (f, t+2) and face sides / Gauss points (f, t), with f the normal and t the tangential
// index, f along the rows for x-faces and t along the rows for y-faces.
template <int DIR> DFK_HD int lines_lx(const Mesh& m) { return DIR == 0 ? m.nx + 1 : m.nx + 4; }
template <int DIR> DFK_HD int lines_ly(const Mesh& m) { return DIR == 0 ? m.ny + 4 : m.ny + 1; }
template <int DIR> DFK_HD int faces_lx(const Mesh& m) { return DIR == 0 ? m.nx + 1 : m.nx; }
template <int DIR> DFK_HD int faces_ly(const Mesh& m) { return DIR == 0 ? m.ny : m.ny + 1; }

// The sweep kernels run on 1-D grids of 128-thread blocks over such a space: thread i takes
// (i mod lx, i / lx), so only the grid's last warp is partly idle, where a 2-D grid of 32-wide rows
// would idle part of every row's last warp (15 of 416 lanes on a 401-face row).  Threads past the
// end get ay >= ly, which the bodies' bounds checks reject.
inline unsigned sweep_blocks(int lx, int ly) { return (unsigned)(((long long)lx * ly + 127) / 128); }
__device__ __forceinline__ void sweep_xy(int lx, int& ax, int& ay) {
    const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    ax = i % lx;
    ay = i / lx;
}

__device__ __forceinline__ void warp_count_add(unsigned long long* dst, int v) {
    int s = __reduce_add_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(dst, (unsigned long long)s);
}

DFK_HD void report_fail(DevState* st, long long key) {
#ifdef __CUDA_ARCH__
    atomicMin(&st->fail_key, (unsigned long long)key);
    if (atomicCAS(&st->err, 0, 5) == 0) st->fail_step = st->step;
    atomicExch(&st->halt, 1);
#else   // host build of the bodies (sequential)
    if ((unsigned long long)key < st->fail_key) st->fail_key = (unsigned long long)key;
    if (st->err == 0) { st->err = 5; st->fail_step = st->step; }
    st->halt = 1;
#endif
}

// linear index j*nx + i of cell (i, j) in the enclosing mesh (the mesh itself unless a block)
DFK_HD long long fail_key(const Mesh& m, int i, int j) {
    const long long gnx = m.gnx > 0 ? m.gnx : m.nx;
    return (long long)(j + m.gj0) * gnx + (i + m.gi0);
}

DFK_HD bool state_ok(const double W[4], double gm1) {
    bool fin = isfinite(W[0]) && isfinite(W[1]) && isfinite(W[2]) && isfinite(W[3]);
    return fin && physical_state(W, gm1);
}

// CFL bound of one interior cell: min(dx/(|U|+c), dy/(|V|+c)), or 1/((|U|+c)/dx + (|V|+c)/dy)
__device__ __forceinline__ double cfl_cell(const Mesh& m, const double* W, double gamma, int c) {
    int i = c % m.nx, j = c / m.nx;
    long long g = gid(m, i, j);
    double r = W[g], U = W[m.plane + g] / r, V = W[2 * m.plane + g] / r;
    double p = (gamma - 1.0) * (W[3 * m.plane + g] - 0.5 * r * (U * U + V * V));
    double cs = sqrt(gamma * p / r);
    if (m.dt_rule) return 1.0 / ((fabs(U) + cs) / m.dx + (fabs(V) + cs) / m.dy);
    return fmin(m.dx / (fabs(U) + cs), m.dy / (fabs(V) + cs));
}

// block-wide minimum of v (all threads call); thread 0 of the block receives the result
__device__ __forceinline__ double block_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    __shared__ double red[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : DBL_MAX;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;
}

// one ghost cell of the x pass: ghost column gc in [0, 2G), interior row j (a side marked
// BC_EXTERNAL is left to the halo copy)
DFK_HD void ghost_x_body(const Mesh& m, double* W, double* alpha, int gc, int j) {
    if (gc >= 2 * G || j >= m.ny) return;
    if (m.bc[gc < G ? 0 : 1] == BC_EXTERNAL) return;
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

// one ghost cell of the y pass: column i in [-G, nx+G), ghost row gr in [0, 2G)
DFK_HD void ghost_y_body(const Mesh& m, double* W, double* alpha, int i, int gr) {
    if (i >= m.nx + G) return;
    if (m.bc[gr < G ? 2 : 3] == BC_EXTERNAL) return;
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

// one face line (normal reconstruction of both sides); returns the number of DF branches taken
// TAPE: also write the reconstructions' intermediates for a reverse sweep (ltape, see SweepBuffers)
template <int DIR, bool TAPE = false>
DFK_HD int lines_body(const Mesh& m, const SchemeConsts& S, const double* __restrict__ W,
                                          const double* __restrict__ alpha, double* __restrict__ lines,
                                          long long ls, int ax, int ay, double* __restrict__ ltape = nullptr) {
    Geo<DIR> g(m);
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
        const bool dfL = nn_less(nn_max(nn_max(al[1], al[2]), al[3]), S.alpha_thres);   // Eq. 34, cell f-1
        const bool dfR = nn_less(nn_max(nn_max(al[2], al[3]), al[4]), S.alpha_thres);   // Eq. 34, cell f
        ndf = (int)dfL + (int)dfR;
        const double idn = g.idn;
        const long long li = g.line(f, t);
        // the cell-average reading of the DF states, stored before the reconstructions so that
        // the two cell states need not stay live through them
        if (S.df_states) lines[LR_DFC * ls + li] = df_alpha(Wc[2], Wc[3], S);
        double qL[4], qLn[4], qR[4], qRn[4];
        // the limiter weight so far as tn / td (1 until a reconstruction gives less); fractions are
        // compared by cross-multiplication (denominators >= 2), one division at the end
        double tn = 1.0, td = 1.0;
        int tlk = -1;                                     // the reconstruction that set it
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double sL[5] = {Q[0][k], Q[1][k], Q[2][k], Q[3][k], Q[4][k]};
            double sR[5] = {Q[5][k], Q[4][k], Q[3][k], Q[2][k], Q[1][k]};   // mirrored about cell f
            double v, sl;
            if (!TAPE) {
                // both reconstructions at once: the mirrored stencils share two of their three
                // quadratic second differences, and the weights' normalisers one division
                if (!dfL || !dfR || S.time_limiter) {
                    const double h = 0.5 * kS13;
                    const double d01 = h * (Q[0][k] - 2.0 * Q[1][k] + Q[2][k]);
                    const double d12 = h * (Q[1][k] - 2.0 * Q[2][k] + Q[3][k]);
                    const double d23 = h * (Q[2][k] - 2.0 * Q[3][k] + Q[4][k]);
                    const double d34 = h * (Q[3][k] - 2.0 * Q[4][k] + Q[5][k]);
                    const double aL[3] = {d01, d12, d23}, aR[3] = {d34, d23, d12};
                    AO oL, oR;
                    ao_finish_pair(ao_core(sL, aL, S), ao_core(sR, aR, S), S, oL, oR);
                    if (S.time_limiter) {
                        double n, d;
                        limiter_fraction(oL, n, d);
                        if (nn_less(n * td, tn * d)) { tn = n; td = d; tlk = 2 * k; }
                        limiter_fraction(oR, n, d);
                        if (nn_less(n * td, tn * d)) { tn = n; td = d; tlk = 2 * k + 1; }
                    }
                    if (!dfL) { ao_at_right_edge(oL, sL[2], v, sl); qL[k] = v; qLn[k] = sl * idn; }
                    if (!dfR) { ao_at_right_edge(oR, sR[2], v, sl); qR[k] = v; qRn[k] = -sl * idn; }
                }
                if (dfL) { df_at_right_edge(sL, al[2], v, sl); qL[k] = v; qLn[k] = sl * idn; }
                if (dfR) { df_at_right_edge(sR, al[3], v, sl); qR[k] = v; qRn[k] = -sl * idn; }
                continue;
            }
            if (!dfL || S.time_limiter) {
                AO o = TAPE ? weno_ao_t(sL, S, PlaneTape{ltape + li, ls}, 2 * k * AT_COUNT) : weno_ao(sL, S);
                if (S.time_limiter) {
                    double n, d;
                    limiter_fraction(o, n, d);
                    if (nn_less(n * td, tn * d)) { tn = n; td = d; tlk = 2 * k; }
                }
                if (!dfL) ao_at_right_edge(o, sL[2], v, sl);
            }
            if (dfL) df_at_right_edge(sL, al[2], v, sl);
            qL[k] = v; qLn[k] = sl * idn;
            if (!dfR || S.time_limiter) {
                AO o = TAPE ? weno_ao_t(sR, S, PlaneTape{ltape + li, ls}, (2 * k + 1) * AT_COUNT) : weno_ao(sR, S);
                if (S.time_limiter) {
                    double n, d;
                    limiter_fraction(o, n, d);
                    if (nn_less(n * td, tn * d)) { tn = n; td = d; tlk = 2 * k + 1; }
                }
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
#pragma unroll
        for (int q = 0; q < 16; ++q) lines[q * ls + li] = out[q];
        lines[LR_TL * ls + li] = tn / td;
        lines[LR_TLK * ls + li] = (double)tlk;
        lines[LR_U * ls + li] = B.u;
        lines[LR_V * ls + li] = B.v;
        lines[LR_C * ls + li] = B.c;
        lines[LR_IC * ls + li] = B.ic;
        lines[LR_H * ls + li] = B.H;
        lines[LR_B1 * ls + li] = B.b1;
        lines[LR_B2 * ls + li] = B.b2;
        lines[LR_Q2 * ls + li] = B.q2;
    }
    return ndf;
}

// one face side (tangential reconstruction at both Gauss points, fallback); returns the number of
// DF branches taken and sets nfb to the number of fallbacks
// TAPE: also write the reconstructions' intermediates for a reverse sweep (ftape, see SweepBuffers)
template <int DIR, bool TAPE = false>
DFK_HD int faces_body(const Mesh& m, const SchemeConsts& S, const double* __restrict__ W,
                                          const double* __restrict__ alpha, const double* __restrict__ lines,
                                          long long ls, double* __restrict__ gp, long long gs,
                                          int ax, int ay, int side, int& nfb,
                                          double* __restrict__ ftape = nullptr) {
    Geo<DIR> g(m);
    int f = DIR == 0 ? ax : ay;
    int t = DIR == 0 ? ay : ax;
    bool active = f <= g.nn && t < g.nt;
    int ndf = 0;
    nfb = 0;
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
        const bool df = nn_less(nn_max(nn_max(al[0], al[1]), al[2]), S.alpha_thres);    // Eq. 34, tangential
        ndf = (int)df;
        double qv[2][4], qt[2][4];
        const double idt = g.idtan;
        const long long e = (long long)side * g.nfaces() + g.face(f, t);
        if (!TAPE && !df) {
            // the four components' reconstructions in two pairs, one division per pair
#pragma unroll
            for (int k = 0; k < 4; k += 2) {
                const double sa[5] = {Q[0][k], Q[1][k], Q[2][k], Q[3][k], Q[4][k]};
                const double sb[5] = {Q[0][k + 1], Q[1][k + 1], Q[2][k + 1], Q[3][k + 1], Q[4][k + 1]};
                double da[3], db[3];
                ao_second_differences(sa, da);
                ao_second_differences(sb, db);
                AO oa, ob;
                ao_finish_pair(ao_core(sa, da, S), ao_core(sb, db, S), S, oa, ob);
                double v[2], s[2];
                ao_at_gauss(oa, sa[2], v, s);
                qv[0][k] = v[0]; qv[1][k] = v[1];
                qt[0][k] = s[0] * idt; qt[1][k] = s[1] * idt;
                ao_at_gauss(ob, sb[2], v, s);
                qv[0][k + 1] = v[0]; qv[1][k + 1] = v[1];
                qt[0][k + 1] = s[0] * idt; qt[1][k + 1] = s[1] * idt;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                double sq[5] = {Q[0][k], Q[1][k], Q[2][k], Q[3][k], Q[4][k]};
                double v[2], s[2];
                if (df) df_at_gauss(sq, al[1], v, s);
                else {
                    AO o = TAPE ? weno_ao_t(sq, S, PlaneTape{ftape + e, gs}, k * AT_COUNT) : weno_ao(sq, S);
                    ao_at_gauss(o, sq[2], v, s);
                }
                qv[0][k] = v[0]; qv[1][k] = v[1];
                qt[0][k] = s[0] * idt; qt[1][k] = s[1] * idt;
            }
        }
        const int nbase = side == 0 ? LR_WLN : LR_WRN;
        int fbits = 0;
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
                fbits |= 1 << mm;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                gp[(mm * 12 + k) * gs + e] = Wg[k];
                gp[(mm * 12 + 4 + k) * gs + e] = Wn[k];
                gp[(mm * 12 + 8 + k) * gs + e] = Wt[k];
            }
        }
        gp[GP_FB * gs + e] = (double)fbits;
    }
    return ndf;
}

// where one Gauss point's records live: side records eL / eR, its flux record e, its face line li
struct FluxSite { long long eL, eR, e, li; bool ok; };

template <int DIR>
DFK_HD FluxSite flux_site(const Mesh& m, int ax, int ay, int mm) {
    Geo<DIR> g(m);
    const int f = DIR == 0 ? ax : ay;
    const int t = DIR == 0 ? ay : ax;
    FluxSite s;
    s.ok = f <= g.nn && t < g.nt;
    if (!s.ok) { s.eL = s.eR = s.e = s.li = 0; return s; }
    const long long fid = g.face(f, t);
    s.eL = fid;
    s.eR = g.nfaces() + fid;
    s.e = (long long)mm * g.nfaces() + fid;
    s.li = g.line(f, t);
    return s;
}

// one Gauss point (flux, time derivative, DF factor, omega^t) of direction dir at a site
template <int FLUX, bool ALPHA_ONLY, bool TAPE = false>
DFK_HD void flux_point(int dir, const SchemeConsts& S, const FluxSite& site, const double* __restrict__ lines,
                       long long ls, const double* __restrict__ gp, long long gs, double* __restrict__ fr,
                       long long fs, double dt, int mm, double* __restrict__ tape = nullptr) {
    GPState L, R;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        L.W[k] = gp[(mm * 12 + k) * gs + site.eL];
        L.Wn[k] = gp[(mm * 12 + 4 + k) * gs + site.eL];
        L.Wt[k] = gp[(mm * 12 + 8 + k) * gs + site.eL];
        R.W[k] = gp[(mm * 12 + k) * gs + site.eR];
        R.Wn[k] = gp[(mm * 12 + 4 + k) * gs + site.eR];
        R.Wt[k] = gp[(mm * 12 + 8 + k) * gs + site.eR];
    }
    const long long e = site.e;
    // the two sides' Maxwellians serve the DF factor and the GKS flux.  The Gauss-point reading of
    // Eq. 33 is always evaluated (the default path stays branch-free); the cell-average reading,
    // when selected, overwrites it with its face line's value
    Maxw sl, sr;
    maxw_pair(L.W, R.W, S, sl, sr);
    fr[FR_ALPHA * fs + e] = df_alpha_maxw(sl, sr, S);
    if (S.df_states) fr[FR_ALPHA * fs + e] = lines[LR_DFC * ls + site.li];
    if (ALPHA_ONLY) return;
    double F[4], dF[4];
    if (FLUX == 0) {
        if (TAPE) gks_flux_t(L, R, sl, sr, dt, S, F, dF, PlaneTape{tape + e, fs});
        else gks_flux_t(L, R, sl, sr, dt, S, F, dF, NoTape{});
    }
    else lf_flux(L, R, S, F, dF);
    if (dir == 1) { to_global<1>(F); to_global<1>(dF); }
#pragma unroll
    for (int k = 0; k < 4; ++k) { fr[(FR_F + k) * fs + e] = F[k]; fr[(FR_DF + k) * fs + e] = dF[k]; }
    fr[FR_OMEGA * fs + e] = S.time_limiter ? lines[LR_TL * ls + site.li] : 1.0;
}

// one Gauss point (flux, time derivative, DF factor, omega^t)
template <int DIR, int FLUX, bool ALPHA_ONLY, bool TAPE = false>
DFK_HD void flux_body(const Mesh& m, const SchemeConsts& S, const double* __restrict__ lines,
                                          long long ls, const double* __restrict__ gp, long long gs,
                                          double* __restrict__ fr, long long fs, double dt, int ax, int ay, int mm,
                         double* __restrict__ tape = nullptr) {
    const FluxSite site = flux_site<DIR>(m, ax, ay, mm);
    if (!site.ok) return;
    flux_point<FLUX, ALPHA_ONLY, TAPE>(DIR, S, site, lines, ls, gp, gs, fr, fs, dt, mm, tape);
}

// one cell: residual, limited time derivative, stage combination, alpha product, positivity
template <int MODE>
DFK_HD void update_body(const Mesh& m, const SchemeConsts& S, const UpdateArgs& a,
                                            const double* __restrict__ frx, long long fsx,
                                            const double* __restrict__ fry, long long fsy,
                                            double dt, DevState* st, int i, int j) {
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
    const double idx = m.rdx, idy = m.rdy;
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
        L[k] = -(FE - FW) * idx - (FN - FS) * idy;
        dL[k] = -(DE - DW) * idx - (DN - DS) * idy;
        dLt[k] = -(oe * DE - ow * DW) * idx - (on * DN - os * DS) * idy;
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
        if (!state_ok(Ws, S.gm1)) report_fail(st, fail_key(m, i, j));
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
    if (!state_ok(Wo, S.gm1)) report_fail(st, fail_key(m, i, j));
}

}  // namespace dfk
