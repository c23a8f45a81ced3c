// dfgks_adjoint.cu -- reverse (vector-Jacobian product) of the single-stage operator.
//
// With the forward records of one direction in place (face lines, Gauss-point states, fluxes),
// three kernels walk that direction's sweep backwards:
//   ka_flux  : one thread per Gauss point.  Face adjoints from the cells' L, dL/dt and limited
//              dL/dt adjoints (Eq. 2 with A_m = 1/2), then the GKS / L-F flux adjoint into the
//              Gauss-point record adjoints, and the time-limiter weight's adjoint.  When the
//              forward sweep taped the GKS flux's intermediates, its reverse reads them instead
//              of recomputing the flux.
//   ka_faces : one thread per face side.  Evaluates each tangential reconstruction once, with its
//              intermediates kept for its reverse (or reads them from the forward sweep's tape),
//              and scatters (atomically) into the adjoints of
//              the five face lines and of the face basis; a Gauss point that fell back to the cell
//              average (flagged in the forward record) sends its adjoint to that cell.
//   ka_lines : one thread per face line.  The same for the eight normal reconstructions and the
//              limiter weight (the forward record names the reconstruction that set it), then
//              scatters into the ghosted cell adjoints.
// A final pass folds ghost-cell adjoints back into the interior cells they were copied from.
// alpha, dt and every branch decision are those of the forward pass.
#include "dfgks_adjoint.cuh"
#include "dfgks_bodies.cuh"

namespace dfk {

DFK_HD void aadd(double* p, double v) {
#ifdef __CUDA_ARCH__
    if (v != 0.0) atomicAdd(p, v);
#else
    *p += v;
#endif
}

// TAPED: the GKS forward intermediates are read from the tape the forward sweep wrote
template <int DIR, int FLUX, bool TAPED = false>
DFK_HD void ka_flux_body(const Mesh& m, const SchemeConsts& S, const AdjointArgs& a, const double* __restrict__ gp,
                         long long gs, const double* __restrict__ fr, long long fs, double dt, double* __restrict__ lb,
                         long long ls, double* __restrict__ gb, int ax, int ay, int mm,
                         double* __restrict__ tape = nullptr) {
    Geo<DIR> g(m);
    int f = DIR == 0 ? ax : ay;
    int t = DIR == 0 ? ay : ax;
    if (f > g.nn || t >= g.nt) return;
    const long long fid = g.face(f, t), nf = g.nfaces();
    const long long dplane = (long long)m.nx * m.ny;
    // adjoints of the two cells' residuals (cells outside the mesh have none)
    double dL[4] = {0, 0, 0, 0}, ddL[4] = {0, 0, 0, 0}, ddLt[4] = {0, 0, 0, 0};
    for (int side = 0; side < 2; ++side) {
        const int n = f - 1 + side;
        if (n < 0 || n >= g.nn) continue;
        const long long c = DIR == 0 ? (long long)t * m.nx + n : (long long)n * m.nx + t;
        const double sg = side == 0 ? -1.0 : 1.0;    // F enters L of the left cell with -1/dn
        for (int k = 0; k < 4; ++k) {
            if (a.Lb) dL[k] += sg * a.Lb[k * dplane + c];
            if (a.dtLb) ddL[k] += sg * a.dtLb[k * dplane + c];
            if (a.dtLtb) ddLt[k] += sg * a.dtLtb[k * dplane + c];
        }
    }
    const double idn = g.idn;
    const double om = fr[FR_OMEGA * fs + fid];
    double Fb[4], dFb[4];
    for (int k = 0; k < 4; ++k) {
        Fb[k] = 0.5 * dL[k] * idn;                              // Gauss weight 1/2
        dFb[k] = 0.5 * (ddL[k] + om * ddLt[k]) * idn;
    }
    if (mm == 0 && S.time_limiter) {
        double wb = 0.0;
        for (int k = 0; k < 4; ++k) {
            double dFface = 0.5 * fr[(FR_DF + k) * fs + fid] + 0.5 * fr[(FR_DF + k) * fs + nf + fid];
            wb += dFface * ddLt[k] * idn;
        }
        lb[LR_TL * ls + g.line(f, t)] = wb;
    }
    to_local<DIR>(Fb);                                          // F = T^{-1} F~, T orthogonal
    to_local<DIR>(dFb);
    const long long eL = fid, eR = nf + fid;
    GPState L, R;
    for (int k = 0; k < 4; ++k) {
        L.W[k] = gp[(mm * 12 + k) * gs + eL];
        L.Wn[k] = gp[(mm * 12 + 4 + k) * gs + eL];
        L.Wt[k] = gp[(mm * 12 + 8 + k) * gs + eL];
        R.W[k] = gp[(mm * 12 + k) * gs + eR];
        R.Wn[k] = gp[(mm * 12 + 4 + k) * gs + eR];
        R.Wt[k] = gp[(mm * 12 + 8 + k) * gs + eR];
    }
    GPStateBar Lbar, Rbar;
    for (int k = 0; k < 4; ++k) { Lbar.W[k] = Lbar.Wn[k] = Lbar.Wt[k] = Rbar.W[k] = Rbar.Wn[k] = Rbar.Wt[k] = 0.0; }
    if (FLUX == 0 && TAPED) gks_flux_reverse(PlaneTape{tape + (long long)mm * nf + fid, fs}, L, R, dt, S, Fb, dFb, Lbar, Rbar);
    else if (FLUX == 0) gks_flux_vjp(L, R, dt, S, Fb, dFb, Lbar, Rbar);
    else lf_flux_vjp(L, R, S, Fb, dFb, Lbar, Rbar);
    for (int k = 0; k < 4; ++k) {
        gb[(mm * 12 + k) * gs + eL] = Lbar.W[k];
        gb[(mm * 12 + 4 + k) * gs + eL] = Lbar.Wn[k];
        gb[(mm * 12 + 8 + k) * gs + eL] = Lbar.Wt[k];
        gb[(mm * 12 + k) * gs + eR] = Rbar.W[k];
        gb[(mm * 12 + 4 + k) * gs + eR] = Rbar.Wn[k];
        gb[(mm * 12 + 8 + k) * gs + eR] = Rbar.Wt[k];
    }
}

// TAPED: the tangential reconstructions' intermediates are read from the tape the forward sweep wrote
template <int DIR, bool TAPED = false>
DFK_HD void ka_faces_body(const Mesh& m, const SchemeConsts& S, const double* __restrict__ alpha,
                          const double* __restrict__ lines, long long ls, const double* __restrict__ gp,
                          const double* __restrict__ gb, long long gs, double* __restrict__ lb,
                          double* __restrict__ Wb, int ax, int ay, int side, double* __restrict__ ftape = nullptr) {
    Geo<DIR> g(m);
    int f = DIR == 0 ? ax : ay;
    int t = DIR == 0 ? ay : ax;
    if (f > g.nn || t >= g.nt) return;
    const long long l0 = g.line(f, t);
    CharBasis B;
    B.u = lines[LR_U * ls + l0]; B.v = lines[LR_V * ls + l0]; B.c = lines[LR_C * ls + l0];
    B.ic = lines[LR_IC * ls + l0]; B.H = lines[LR_H * ls + l0]; B.b1 = lines[LR_B1 * ls + l0];
    B.b2 = lines[LR_B2 * ls + l0]; B.q2 = lines[LR_Q2 * ls + l0];
    const int wbase = side == 0 ? LR_WL : LR_WR;
    const int nbase = side == 0 ? LR_WLN : LR_WRN;
    double Wl[5][4], Q[5][4];
    for (int b = 0; b < 5; ++b) {
        long long lbb = g.line(f, t + Geo<DIR>::sigma * (b - 2));
        for (int k = 0; k < 4; ++k) Wl[b][k] = lines[(wbase + k) * ls + lbb];
        project(B, Wl[b], Q[b]);
    }
    const int ncell = f - 1 + side;
    double al[3];
    for (int b = 0; b < 3; ++b) al[b] = alpha[g.cell(m, ncell, t + Geo<DIR>::sigma * (b - 1))];
    const bool df = nn_less(nn_max(nn_max(al[0], al[1]), al[2]), S.alpha_thres);
    const double idt = g.idtan;
    const long long e = (long long)side * g.nfaces() + g.face(f, t);
    const int fbits = (int)gp[GP_FB * gs + e];
    // Gauss-point adjoints -> characteristic value and tangential-slope adjoints (R^T, independent
    // of the reconstruction); a Gauss point that used the cell average sends its adjoint there
    double wb[2][4], wtb[2][4], qvb[2][4], slb[2][4];
    for (int mm = 0; mm < 2; ++mm) {
        for (int k = 0; k < 4; ++k) {
            wb[mm][k] = gb[(mm * 12 + k) * gs + e];
            wtb[mm][k] = gb[(mm * 12 + 8 + k) * gs + e];
            qvb[mm][k] = 0.0;
            slb[mm][k] = 0.0;
        }
        if ((fbits >> mm) & 1) {
            double wg[4] = {wb[mm][0], wb[mm][1], wb[mm][2], wb[mm][3]};
            to_global<DIR>(wg);
            const long long c = g.cell(m, ncell, t);
            for (int k = 0; k < 4; ++k) { aadd(&Wb[k * m.plane + c], wg[k]); wb[mm][k] = 0.0; wtb[mm][k] = 0.0; }
            continue;
        }
        double qtb[4] = {0, 0, 0, 0};
        back_project_T(B, wb[mm], qvb[mm]);
        back_project_T(B, wtb[mm], qtb);
        for (int k = 0; k < 4; ++k) {
            slb[mm][k] = qtb[k] * idt;
            aadd(&lb[(nbase + k) * ls + l0], gb[(mm * 12 + 4 + k) * gs + e]);   // normal slope copied from the line
        }
    }
    // per characteristic component: the reconstruction once, then its reverse
    double qv[2][4], qt[2][4], Qb[5][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double sq[5] = {Q[0][k], Q[1][k], Q[2][k], Q[3][k], Q[4][k]};
        double vb[2] = {qvb[0][k], qvb[1][k]}, sb[2] = {slb[0][k], slb[1][k]};
        double v[2], sl[2], qb[5] = {0, 0, 0, 0, 0};
        if (df) {
            df_at_gauss(sq, al[1], v, sl);
            df_at_gauss_vjp(al[1], vb, sb, qb);
        } else if (TAPED) {
            const PlaneTape T{ftape + e, gs};
            AO o = ao_from_tape(T, k * AT_COUNT, S);
            ao_at_gauss(o, sq[2], v, sl);
            AOBar ob;
            ao_bar_zero(ob);
            ao_at_gauss_vjp(vb, sb, qb[2], ob);
            weno_ao_rev(T, k * AT_COUNT, S, ob, qb);
        } else {
            double tb[AT_COUNT];
            const ArrayTape T{tb};
            AO o = weno_ao_t(sq, S, T, 0);
            ao_at_gauss(o, sq[2], v, sl);
            AOBar ob;
            ao_bar_zero(ob);
            ao_at_gauss_vjp(vb, sb, qb[2], ob);
            weno_ao_rev(T, 0, S, ob, qb);
        }
        qv[0][k] = v[0]; qv[1][k] = v[1];
        qt[0][k] = sl[0] * idt; qt[1][k] = sl[1] * idt;
        for (int b = 0; b < 5; ++b) Qb[b][k] = qb[b];
    }
    BasisBar Bb;
    basis_bar_zero(Bb);
    for (int mm = 0; mm < 2; ++mm) {          // zero adjoints (fallback) add nothing
        back_project_basis_vjp(B, qv[mm], wb[mm], Bb);
        back_project_basis_vjp(B, qt[mm], wtb[mm], Bb);
    }
    for (int b = 0; b < 5; ++b) {
        double wl[4] = {0, 0, 0, 0};
        project_vjp(B, Wl[b], Qb[b], wl, Bb);
        long long lbb = g.line(f, t + Geo<DIR>::sigma * (b - 2));
        for (int k = 0; k < 4; ++k) aadd(&lb[(wbase + k) * ls + lbb], wl[k]);
    }
    aadd(&lb[LR_U * ls + l0], Bb.u); aadd(&lb[LR_V * ls + l0], Bb.v); aadd(&lb[LR_C * ls + l0], Bb.c);
    aadd(&lb[LR_IC * ls + l0], Bb.ic); aadd(&lb[LR_H * ls + l0], Bb.H); aadd(&lb[LR_B1 * ls + l0], Bb.b1);
    aadd(&lb[LR_B2 * ls + l0], Bb.b2); aadd(&lb[LR_Q2 * ls + l0], Bb.q2);
}

// TAPED: the normal reconstructions' intermediates are read from the tape the forward sweep wrote
template <int DIR, bool TAPED = false>
DFK_HD void ka_lines_body(const Mesh& m, const SchemeConsts& S, const double* __restrict__ W,
                          const double* __restrict__ alpha, const double* __restrict__ lines,
                          const double* __restrict__ lb, long long ls, double* __restrict__ Wb, int ax, int ay,
                          double* __restrict__ ltape = nullptr) {
    Geo<DIR> g(m);
    int f = DIR == 0 ? ax : ay;
    int tt = DIR == 0 ? ay : ax;
    if (f > g.nn || tt >= g.nt + 4) return;
    const int t = tt - 2;
    const long long li = g.line(f, t);
    double Wc[6][4], al[6];
    for (int s = 0; s < 6; ++s) {
        long long c = g.cell(m, f - 3 + s, t);
        for (int k = 0; k < 4; ++k) Wc[s][k] = W[k * m.plane + c];
        to_local<DIR>(Wc[s]);
        al[s] = alpha[c];
    }
    CharBasis B = make_basis(Wc[2], Wc[3], S);
    double Q[6][4];
    for (int s = 0; s < 6; ++s) project(B, Wc[s], Q[s]);
    const bool dfL = nn_less(nn_max(nn_max(al[1], al[2]), al[3]), S.alpha_thres);
    const bool dfR = nn_less(nn_max(nn_max(al[2], al[3]), al[4]), S.alpha_thres);
    const double idn = g.idn;
    // the reconstruction that set the limiter weight in the forward pass (2k + side) and the
    // weight's adjoint
    const int tlk = S.time_limiter ? (int)lines[LR_TLK * ls + li] : -1;
    const double tlb = S.time_limiter ? lb[LR_TL * ls + li] : 0.0;
    BasisBar Bb;
    Bb.u = lb[LR_U * ls + li]; Bb.v = lb[LR_V * ls + li]; Bb.c = lb[LR_C * ls + li]; Bb.ic = lb[LR_IC * ls + li];
    Bb.H = lb[LR_H * ls + li]; Bb.b1 = lb[LR_B1 * ls + li]; Bb.b2 = lb[LR_B2 * ls + li]; Bb.q2 = lb[LR_Q2 * ls + li];
    double WLb[4], WLnb[4], WRb[4], WRnb[4];
    for (int k = 0; k < 4; ++k) {
        WLb[k] = lb[(LR_WL + k) * ls + li]; WLnb[k] = lb[(LR_WLN + k) * ls + li];
        WRb[k] = lb[(LR_WR + k) * ls + li]; WRnb[k] = lb[(LR_WRN + k) * ls + li];
    }
    double qLb[4] = {0, 0, 0, 0}, qLnb[4] = {0, 0, 0, 0}, qRb[4] = {0, 0, 0, 0}, qRnb[4] = {0, 0, 0, 0};
    back_project_T(B, WLb, qLb);
    back_project_T(B, WLnb, qLnb);
    back_project_T(B, WRb, qRb);
    back_project_T(B, WRnb, qRnb);
    double qL[4], qLn[4], qR[4], qRn[4], Qb[6][4];
    for (int s = 0; s < 6; ++s) for (int k = 0; k < 4; ++k) Qb[s][k] = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
            // side 0: cell f-1, value at xi = +1/2; side 1: cell f, mirrored stencil, slope sign reversed
            double sq[5];
            for (int i = 0; i < 5; ++i) sq[i] = sd == 0 ? Q[i][k] : Q[5 - i][k];
            const bool dfs = sd == 0 ? dfL : dfR;
            const double as = sd == 0 ? al[2] : al[3];
            const double sgn = sd == 0 ? 1.0 : -1.0;
            const double vb = sd == 0 ? qLb[k] : qRb[k];
            const double sb = sgn * (sd == 0 ? qLnb[k] : qRnb[k]) * idn;
            const bool lim = tlk == 2 * k + sd && tlb != 0.0;
            double v = 0.0, sl = 0.0, qb[5] = {0, 0, 0, 0, 0};
            if (!dfs || lim) {
                double tb[AT_COUNT];
                const int base = TAPED ? (2 * k + sd) * AT_COUNT : 0;
                const PlaneTape PT{ltape + (TAPED ? li : 0), ls};
                const ArrayTape AT{tb};
                AO o = TAPED ? ao_from_tape(PT, base, S) : weno_ao_t(sq, S, AT, 0);
                AOBar ob;
                ao_bar_zero(ob);
                if (!dfs) {
                    ao_at_right_edge(o, sq[2], v, sl);
                    ao_at_right_edge_vjp(vb, sb, qb[2], ob);
                }
                if (lim) limiter_alpha_vjp(o, tlb, ob);
                if (TAPED) weno_ao_rev(PT, base, S, ob, qb);
                else weno_ao_rev(AT, 0, S, ob, qb);
            }
            if (dfs) {
                df_at_right_edge(sq, as, v, sl);
                df_at_right_edge_vjp(as, vb, sb, qb);
            }
            if (sd == 0) { qL[k] = v; qLn[k] = sl * idn; }
            else { qR[k] = v; qRn[k] = -sl * idn; }
            for (int i = 0; i < 5; ++i) Qb[sd == 0 ? i : 5 - i][k] += qb[i];
        }
    }
    back_project_basis_vjp(B, qL, WLb, Bb);
    back_project_basis_vjp(B, qLn, WLnb, Bb);
    back_project_basis_vjp(B, qR, WRb, Bb);
    back_project_basis_vjp(B, qRn, WRnb, Bb);
    double Wcb[6][4];
    for (int s = 0; s < 6; ++s) {
        for (int k = 0; k < 4; ++k) Wcb[s][k] = 0.0;
        project_vjp(B, Wc[s], Qb[s], Wcb[s], Bb);
    }
    make_basis_vjp(Wc[2], Wc[3], S, Bb, Wcb[2], Wcb[3]);
    for (int s = 0; s < 6; ++s) {
        to_global<DIR>(Wcb[s]);                                // the rotation is orthogonal
        long long c = g.cell(m, f - 3 + s, t);
        for (int k = 0; k < 4; ++k) aadd(&Wb[k * m.plane + c], Wcb[s][k]);
    }
}

// Reverse of the ghost fill: the y pass (all columns) first, then the x pass (interior rows).
DFK_HD void ka_fold_y_body(const Mesh& m, double* Wb, int i) {
    if (i >= m.nx + G) return;
    for (int gr = 2 * G - 1; gr >= 0; --gr) {
        int j = gr < G ? gr - G : m.ny + gr - G;
        bool mir;
        int s = ghost_src(j, m.ny, m.bc[2], m.bc[3], mir);
        long long d = gid(m, i, j), o = gid(m, i, s);
        for (int k = 0; k < 4; ++k) {
            double v = Wb[k * m.plane + d];
            Wb[k * m.plane + d] = 0.0;
            Wb[k * m.plane + o] += (mir && k == 2) ? -v : v;
        }
    }
}

DFK_HD void ka_fold_x_body(const Mesh& m, double* Wb, int j) {
    if (j >= m.ny) return;
    for (int gc = 2 * G - 1; gc >= 0; --gc) {
        int i = gc < G ? gc - G : m.nx + gc - G;
        bool mir;
        int s = ghost_src(i, m.nx, m.bc[0], m.bc[1], mir);
        long long d = gid(m, i, j), o = gid(m, s, j);
        for (int k = 0; k < 4; ++k) {
            double v = Wb[k * m.plane + d];
            Wb[k * m.plane + d] = 0.0;
            Wb[k * m.plane + o] += (mir && k == 1) ? -v : v;
        }
    }
}

DFK_HD void ka_accumulate_body(const Mesh& m, const double* __restrict__ Wbg, double* __restrict__ out, int i, int j) {
    if (i >= m.nx || j >= m.ny) return;
    const long long dp = (long long)m.nx * m.ny;
    for (int k = 0; k < 4; ++k) out[k * dp + (long long)j * m.nx + i] += Wbg[k * m.plane + gid(m, i, j)];
}

// ---- kernels: one thread per body invocation ----
template <int DIR, int FLUX, bool TAPED = false>
__global__ void __launch_bounds__(128) ka_flux(Mesh m, SchemeConsts S, AdjointArgs a, const double* __restrict__ gp,
                                               long long gs, const double* __restrict__ fr, long long fs,
                                               const double* dtp, double* __restrict__ lb, long long ls,
                                               double* __restrict__ gb, double* __restrict__ tape = nullptr) {
    int ax, ay;
    sweep_xy(faces_lx<DIR>(m), ax, ay);
    ka_flux_body<DIR, FLUX, TAPED>(m, S, a, gp, gs, fr, fs, *dtp, lb, ls, gb, ax, ay, blockIdx.y, tape);
}

template <int DIR, bool TAPED>
__global__ void __launch_bounds__(128) ka_faces(Mesh m, SchemeConsts S, const double* __restrict__ alpha,
                                                const double* __restrict__ lines, long long ls,
                                                const double* __restrict__ gp, const double* __restrict__ gb,
                                                long long gs, double* __restrict__ lb, double* __restrict__ Wb,
                                                double* __restrict__ ftape) {
    int ax, ay;
    sweep_xy(faces_lx<DIR>(m), ax, ay);
    ka_faces_body<DIR, TAPED>(m, S, alpha, lines, ls, gp, gb, gs, lb, Wb, ax, ay, blockIdx.y, ftape);
}

template <int DIR, bool TAPED>
__global__ void __launch_bounds__(128) ka_lines(Mesh m, SchemeConsts S, const double* __restrict__ W,
                                                const double* __restrict__ alpha, const double* __restrict__ lines,
                                                const double* __restrict__ lb, long long ls, double* __restrict__ Wb,
                                                double* __restrict__ ltape) {
    int ax, ay;
    sweep_xy(lines_lx<DIR>(m), ax, ay);
    ka_lines_body<DIR, TAPED>(m, S, W, alpha, lines, lb, ls, Wb, ax, ay, ltape);
}

__global__ void ka_fold_y(Mesh m, double* Wb) { ka_fold_y_body(m, Wb, blockIdx.x * blockDim.x + threadIdx.x - G); }
__global__ void ka_fold_x(Mesh m, double* Wb) { ka_fold_x_body(m, Wb, blockIdx.x * blockDim.x + threadIdx.x); }
__global__ void ka_accumulate_dense(Mesh m, const double* __restrict__ Wbg, double* __restrict__ out) {
    ka_accumulate_body(m, Wbg, out, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
}

template <int DIR>
static void adjoint_dir(const Mesh& m, const SchemeConsts& S, int flux, const AdjointArgs& a, const double* W,
                        const double* alpha, const double* dtp, const SweepBuffers& B, double* lb, double* gbuf,
                        double* Wb, cudaStream_t s, KernelTimer* T) {
    // the forward sweep's 1-D grids (sweep_xy)
    const dim3 blk(128);
    const dim3 gf(sweep_blocks(faces_lx<DIR>(m), faces_ly<DIR>(m)), 2);
    const dim3 gl(sweep_blocks(lines_lx<DIR>(m), lines_ly<DIR>(m)));
    cudaMemsetAsync(lb, 0, sizeof(double) * LR_COUNT * B.line_stride, s);
    if (T) T->begin(KK_FLUX);
    if (flux == 0 && B.tape[DIR])
        ka_flux<DIR, 0, true><<<gf, blk, 0, s>>>(m, S, a, B.gp, B.gp_stride, B.flux[DIR], B.flux_stride[DIR], dtp, lb,
                                                 B.line_stride, gbuf, B.tape[DIR]);
    else if (flux == 0)
        ka_flux<DIR, 0><<<gf, blk, 0, s>>>(m, S, a, B.gp, B.gp_stride, B.flux[DIR], B.flux_stride[DIR], dtp, lb,
                                           B.line_stride, gbuf);
    else
        ka_flux<DIR, 1><<<gf, blk, 0, s>>>(m, S, a, B.gp, B.gp_stride, B.flux[DIR], B.flux_stride[DIR], dtp, lb,
                                           B.line_stride, gbuf);
    if (T) { T->end(KK_FLUX, 1); T->begin(KK_FACES); }
    if (B.ftape)
        ka_faces<DIR, true><<<gf, blk, 0, s>>>(m, S, alpha, B.lines, B.line_stride, B.gp, gbuf, B.gp_stride, lb, Wb, B.ftape);
    else
        ka_faces<DIR, false><<<gf, blk, 0, s>>>(m, S, alpha, B.lines, B.line_stride, B.gp, gbuf, B.gp_stride, lb, Wb, nullptr);
    if (T) { T->end(KK_FACES, 1); T->begin(KK_LINES); }
    if (B.ltape)
        ka_lines<DIR, true><<<gl, blk, 0, s>>>(m, S, W, alpha, B.lines, lb, B.line_stride, Wb, B.ltape);
    else
        ka_lines<DIR, false><<<gl, blk, 0, s>>>(m, S, W, alpha, B.lines, lb, B.line_stride, Wb, nullptr);
    if (T) T->end(KK_LINES, 1);
}

void launch_adjoint_dir(int dir, const Mesh& m, const SchemeConsts& S, int flux, const AdjointArgs& a,
                        const double* W, const double* alpha, const double* dtp, const SweepBuffers& B,
                        double* lb, double* gbuf, double* Wb, cudaStream_t s, KernelTimer* T) {
    if (dir == 0) adjoint_dir<0>(m, S, flux, a, W, alpha, dtp, B, lb, gbuf, Wb, s, T);
    else adjoint_dir<1>(m, S, flux, a, W, alpha, dtp, B, lb, gbuf, Wb, s, T);
}

void launch_adjoint_finish(const Mesh& m, double* Wbg, double* Wb_dense, cudaStream_t s) {
    ka_fold_y<<<(m.nx + 2 * G + 127) / 128, 128, 0, s>>>(m, Wbg);
    ka_fold_x<<<(m.ny + 127) / 128, 128, 0, s>>>(m, Wbg);
    dim3 blk(32, 8), grd((m.nx + 31) / 32, (m.ny + 7) / 8);
    ka_accumulate_dense<<<grd, blk, 0, s>>>(m, Wbg, Wb_dense);
}

// y <- a x + b y on dense arrays (step-adjoint combinations)
__global__ void ka_axpby(long long n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        y[q] = a * x[q] + b * y[q];
}
void launch_axpby(long long n, double a, const double* x, double b, double* y, cudaStream_t s) {
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    ka_axpby<<<(unsigned)blocks, 256, 0, s>>>(n, a, x, b, y);
}

}  // namespace dfk
