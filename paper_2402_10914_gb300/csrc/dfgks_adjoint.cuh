// dfgks_adjoint.cuh -- hand-written reverse (vector-Jacobian) products of the building blocks in
// dfgks_device.cuh.  Each *_vjp routine recomputes what it needs of its forward counterpart and
// accumulates (+=) adjoints into its inputs.  Branch decisions (DF switch, fallback, the sign of
// |.|, the arguments selected by min/max) are those of the forward values; at an exact tie the
// derivative of the first argument is taken, and |x| has slope +1 at x = 0.
#pragma once
#include "dfgks_device.cuh"

namespace dfk {

// ------------------------------------------------------------------------------------------
// Characteristic basis
// ------------------------------------------------------------------------------------------
struct BasisBar { double u, v, c, ic, H, b1, b2, q2; };

DFK_HD void basis_bar_zero(BasisBar& b) { b.u = b.v = b.c = b.ic = b.H = b.b1 = b.b2 = b.q2 = 0.0; }

// adjoint of make_basis: accumulates into Wlb, Wrb (the two cell states)
DFK_HD void make_basis_vjp(const double Wl[4], const double Wr[4], const SchemeConsts& S, const BasisBar& Bb,
                           double Wlb[4], double Wrb[4]) {
    double r = 0.5 * (Wl[0] + Wr[0]), m = 0.5 * (Wl[1] + Wr[1]);
    double n = 0.5 * (Wl[2] + Wr[2]), E = 0.5 * (Wl[3] + Wr[3]);
    double ir = 1.0 / r, u = m * ir, v = n * ir, q2 = 0.5 * (u * u + v * v);
    double p = S.gm1 * (E - r * q2);
    double c = sqrt(S.gamma * p * ir), ic = 1.0 / c, H = (E + p) * ir, b1 = S.gm1 * ic * ic;
    double b1b = Bb.b1 + Bb.b2 * q2;
    double q2b = Bb.q2 + Bb.b2 * b1;
    double icb = Bb.ic + b1b * S.gm1 * 2.0 * ic;
    double cb = Bb.c - icb * ic * ic;
    double Eb = Bb.H * ir, pb = Bb.H * ir, irb = Bb.H * (E + p);
    double sb = cb * 0.5 / c;
    pb += sb * S.gamma * ir;
    irb += sb * S.gamma * p;
    Eb += pb * S.gm1;
    double rb = -pb * S.gm1 * q2;
    q2b += -pb * S.gm1 * r;
    double ub = Bb.u + q2b * u, vb = Bb.v + q2b * v;
    double mb = ub * ir, nb = vb * ir;
    irb += ub * m + vb * n;
    rb += -irb * ir * ir;
    const double g[4] = {rb, mb, nb, Eb};
    for (int k = 0; k < 4; ++k) { Wlb[k] += 0.5 * g[k]; Wrb[k] += 0.5 * g[k]; }
}

// adjoint of project (Q = L W): Wb += L^T Qb, basis adjoint accumulated
DFK_HD void project_vjp(const CharBasis& B, const double W[4], const double Qb[4], double Wb[4], BasisBar& Bb) {
    double kb = 0.5 * Qb[0] - Qb[1] + 0.5 * Qb[3];
    double mmb = 0.5 * Qb[0] - 0.5 * Qb[3];
    Wb[0] += Qb[1] - B.v * Qb[2];
    Bb.v += -Qb[2] * W[0];
    Wb[2] += Qb[2];
    // mm = (u W0 - W1) ic
    Bb.u += mmb * B.ic * W[0];
    Wb[0] += mmb * B.ic * B.u;
    Wb[1] += -mmb * B.ic;
    Bb.ic += mmb * (B.u * W[0] - W[1]);
    // k = b2 W0 - t
    Bb.b2 += kb * W[0];
    Wb[0] += kb * B.b2;
    double tb = -kb;
    // t = b1 (u W1 + v W2 - W3)
    Bb.b1 += tb * (B.u * W[1] + B.v * W[2] - W[3]);
    Bb.u += tb * B.b1 * W[1];
    Wb[1] += tb * B.b1 * B.u;
    Bb.v += tb * B.b1 * W[2];
    Wb[2] += tb * B.b1 * B.v;
    Wb[3] += -tb * B.b1;
}

// the two halves of the adjoint of back_project (W = R Q): Qb += R^T Wb, which does not depend on
// Q, and the basis adjoint, which is linear in Q
DFK_HD void back_project_T(const CharBasis& B, const double Wb[4], double Qb[4]) {
    double W0b = Wb[0] + Wb[2] * B.v + Wb[1] * B.u;
    double sb = Wb[3] * B.H + W0b, db = Wb[3] * B.u * B.c + Wb[1] * B.c;
    Qb[1] += Wb[3] * B.q2 + W0b;
    Qb[2] += Wb[3] * B.v + Wb[2];
    Qb[0] += sb - db;
    Qb[3] += sb + db;
}

DFK_HD void back_project_basis_vjp(const CharBasis& B, const double Q[4], const double Wb[4], BasisBar& Bb) {
    double s = Q[0] + Q[3], d = Q[3] - Q[0];
    double W0 = s + Q[1];
    Bb.H += Wb[3] * s;
    Bb.u += Wb[3] * B.c * d + Wb[1] * W0;
    Bb.c += Wb[3] * B.u * d + Wb[1] * d;
    Bb.q2 += Wb[3] * Q[1];
    Bb.v += Wb[3] * Q[2] + Wb[2] * W0;
}

// adjoint of back_project (W = R Q): Qb += R^T Wb, basis adjoint accumulated
DFK_HD void back_project_vjp(const CharBasis& B, const double Q[4], const double Wb[4], double Qb[4], BasisBar& Bb) {
    double s = Q[0] + Q[3], d = Q[3] - Q[0];
    double W0 = s + Q[1];
    double sb = 0.0, db = 0.0;
    // W3 = H s + u c d + q2 Q1 + v Q2
    Bb.H += Wb[3] * s;
    sb += Wb[3] * B.H;
    Bb.u += Wb[3] * B.c * d;
    Bb.c += Wb[3] * B.u * d;
    db += Wb[3] * B.u * B.c;
    Bb.q2 += Wb[3] * Q[1];
    Qb[1] += Wb[3] * B.q2;
    Bb.v += Wb[3] * Q[2];
    Qb[2] += Wb[3] * B.v;
    // W2 = v W0 + Q2
    Bb.v += Wb[2] * W0;
    Qb[2] += Wb[2];
    // W1 = u W0 + c d
    Bb.u += Wb[1] * W0;
    Bb.c += Wb[1] * d;
    db += Wb[1] * B.c;
    // W0 = s + Q1, with the uses in W1 and W2
    double W0b = Wb[0] + Wb[2] * B.v + Wb[1] * B.u;
    sb += W0b;
    Qb[1] += W0b;
    Qb[0] += sb - db;
    Qb[3] += sb + db;
}

// ------------------------------------------------------------------------------------------
// WENO-AO(5,3) and the DF quadratic
// ------------------------------------------------------------------------------------------
struct AOBar { double A1, A2, c3a3, c3a4, rmax, rmin; };

DFK_HD void ao_bar_zero(AOBar& b) { b.A1 = b.A2 = b.c3a3 = b.c3a4 = b.rmax = b.rmin = 0.0; }

// The outputs of a taped WENO-AO reconstruction (weno_ao_t), rebuilt from its tape
template <class Tape>
DFK_HD AO ao_from_tape(const Tape& tp, int base, const SchemeConsts& S) {
    const double iw = tp.get(base + AT_IW), c3 = tp.get(base + AT_C3);
    const double c0 = tp.get(base + AT_W) * iw - c3 * S.d[0], c1 = tp.get(base + AT_W + 1) * iw - c3 * S.d[1];
    const double c2 = tp.get(base + AT_W + 2) * iw - c3 * S.d[2];
    AO o;
    o.A1 = c0 * tp.get(base + AT_A1) + c1 * tp.get(base + AT_A1 + 1) + c2 * tp.get(base + AT_A1 + 2) + c3 * tp.get(base + AT_A1 + 3);
    o.A2 = c0 * tp.get(base + AT_A2) + c1 * tp.get(base + AT_A2 + 1) + c2 * tp.get(base + AT_A2 + 2) + c3 * tp.get(base + AT_A2 + 3);
    o.c3a3 = c3 * tp.get(base + AT_A3);
    o.c3a4 = c3 * tp.get(base + AT_A4);
    o.rmax = tp.get(base + AT_R + (int)tp.get(base + AT_KMAX));
    o.rmin = tp.get(base + AT_R + (int)tp.get(base + AT_KMIN));
    o.rs = 1.0;
    return o;
}

// reverse of weno_ao_t from its tape: qb += (d AO / d q)^T ob
template <class Tape>
DFK_HD void weno_ao_rev(const Tape& tp, int base, const SchemeConsts& S, const AOBar& ob, double qb[5]) {
    const double c13_3 = 13.0 / 3.0;
    double a1[4], a2[4], w[4], r[4], ie[4];
    for (int k = 0; k < 4; ++k) {
        a1[k] = tp.get(base + AT_A1 + k); a2[k] = tp.get(base + AT_A2 + k);
        w[k] = tp.get(base + AT_W + k); r[k] = tp.get(base + AT_R + k); ie[k] = tp.get(base + AT_IE + k);
    }
    const double a3 = tp.get(base + AT_A3), a4 = tp.get(base + AT_A4), iw = tp.get(base + AT_IW), c3 = tp.get(base + AT_C3);
    double c[4];
    for (int k = 0; k < 3; ++k) c[k] = w[k] * iw - c3 * S.d[k];
    c[3] = c3;
    double a1b[4], a2b[4], cb[4];
    for (int k = 0; k < 4; ++k) { a1b[k] = ob.A1 * c[k]; a2b[k] = ob.A2 * c[k]; cb[k] = ob.A1 * a1[k] + ob.A2 * a2[k]; }
    cb[3] += ob.c3a3 * a3 + ob.c3a4 * a4;
    double a3b = ob.c3a3 * c3, a4b = ob.c3a4 * c3;
    double wb[4], iwb = 0.0;
    for (int k = 0; k < 3; ++k) { wb[k] = cb[k] * iw; iwb += cb[k] * w[k]; cb[3] -= cb[k] * S.d[k]; }
    wb[3] = cb[3] * iw * S.inv_d3;
    iwb += cb[3] * w[3] * S.inv_d3;
    const double sumb = -iwb * iw * iw;
    double rb[4];
    for (int k = 0; k < 4; ++k) rb[k] = (wb[k] + sumb) * S.d[k] * 2.0 * r[k];
    rb[(int)tp.get(base + AT_KMAX)] += ob.rmax;
    rb[(int)tp.get(base + AT_KMIN)] += ob.rmin;
    double taub = 0.0, bb[4];
    for (int k = 0; k < 4; ++k) { double t = rb[k] * ie[k]; taub += t; bb[k] = -t * r[k]; }
    const double tb3 = taub * (1.0 / 3.0);
    for (int k = 0; k < 3; ++k) { const double sg = tp.get(base + AT_SG + k); bb[3] += tb3 * sg; bb[k] -= tb3 * sg; }
    for (int k = 0; k < 3; ++k) { a1b[k] += bb[k] * 2.0 * a1[k]; a2b[k] += bb[k] * 2.0 * c13_3 * a2[k]; }
    a1b[3] += bb[3] * (2.0 * a1[3] + 0.5 * a3);
    a3b += bb[3] * (0.5 * a1[3] + 2.0 * (3129.0 / 80.0) * a3);
    a2b[3] += bb[3] * (2.0 * c13_3 * a2[3] + (21.0 / 5.0) * a4);
    a4b += bb[3] * ((21.0 / 5.0) * a2[3] + 2.0 * (87617.0 / 140.0) * a4);
    qb[0] += 0.5 * a1b[0] + 0.5 * a2b[0] + (5.0 / 48.0) * a1b[3] - (1.0 / 16.0) * a2b[3] - (1.0 / 12.0) * a3b + (1.0 / 24.0) * a4b;
    qb[1] += -2.0 * a1b[0] - a2b[0] - 0.5 * a1b[1] + 0.5 * a2b[1] - (34.0 / 48.0) * a1b[3] + (12.0 / 16.0) * a2b[3]
           + (2.0 / 12.0) * a3b - (4.0 / 24.0) * a4b;
    qb[2] += 1.5 * a1b[0] + 0.5 * a2b[0] - a2b[1] - 1.5 * a1b[2] + 0.5 * a2b[2] - (22.0 / 16.0) * a2b[3] + (6.0 / 24.0) * a4b;
    qb[3] += 0.5 * a1b[1] + 0.5 * a2b[1] + 2.0 * a1b[2] - a2b[2] + (34.0 / 48.0) * a1b[3] + (12.0 / 16.0) * a2b[3]
           - (2.0 / 12.0) * a3b - (4.0 / 24.0) * a4b;
    qb[4] += -0.5 * a1b[2] + 0.5 * a2b[2] - (5.0 / 48.0) * a1b[3] - (1.0 / 16.0) * a2b[3] + (1.0 / 12.0) * a3b + (1.0 / 24.0) * a4b;
}

// o from a taped reconstruction (ratios unscaled, o.rs = 1)
DFK_HD void limiter_alpha_vjp(const AO& o, double outb, AOBar& ob) {
    double a1 = 1.0 + o.rmax * o.rmax, a2 = 1.0 + o.rmin * o.rmin, D = a1 + a2;
    ob.rmax += outb * (-2.0 * a2 / (D * D)) * 2.0 * o.rmax;
    ob.rmin += outb * (2.0 * a1 / (D * D)) * 2.0 * o.rmin;
}

DFK_HD void ao_at_right_edge_vjp(double valb, double slopeb, double& q0b, AOBar& ob) {
    q0b += valb;
    ob.A1 += 0.5 * valb + slopeb;
    ob.A2 += (1.0 / 6.0) * valb + slopeb;
    ob.c3a3 += 0.125 * valb + 0.75 * slopeb;
    ob.c3a4 += 0.05 * valb + 0.5 * slopeb;
}

DFK_HD void ao_at_gauss_vjp(const double valb[2], const double slopeb[2], double& q0b, AOBar& ob) {
    const double g = kGaussEta;
    double Eb = valb[0] + valb[1], Ob = valb[1] - valb[0], Esb = slopeb[0] + slopeb[1], Osb = slopeb[1] - slopeb[0];
    q0b += Eb;
    ob.c3a4 += -(1.0 / 180.0) * Eb + g * (1.0 / 3.0) * Osb;
    ob.A1 += g * Ob + Esb;
    ob.c3a3 += g * (1.0 / 12.0) * Ob + 0.25 * Esb;
    ob.A2 += 2.0 * g * Osb;
}

// a1 = (q3 - q1)/2, a2 = (q1 - 2 q2 + q3)/2 of the DF quadratic
DFK_HD void df_coeffs_vjp(double a1b, double a2b, double qb[5]) {
    qb[3] += 0.5 * a1b + 0.5 * a2b;
    qb[1] += -0.5 * a1b + 0.5 * a2b;
    qb[2] += -a2b;
}

DFK_HD void df_at_right_edge_vjp(double alpha, double valb, double slopeb, double qb[5]) {
    qb[2] += valb;
    df_coeffs_vjp(alpha * (0.5 * valb + slopeb), alpha * ((1.0 / 6.0) * valb + slopeb), qb);
}

DFK_HD void df_at_gauss_vjp(double alpha, const double valb[2], const double slopeb[2], double qb[5]) {
    const double g = kGaussEta;
    qb[2] += valb[0] + valb[1];
    double Ob = valb[1] - valb[0], Esb = slopeb[0] + slopeb[1], Osb = slopeb[1] - slopeb[0];
    df_coeffs_vjp(alpha * g * Ob + alpha * Esb, 2.0 * alpha * g * Osb, qb);
}

// ------------------------------------------------------------------------------------------
// GKS flux
// ------------------------------------------------------------------------------------------
struct MaxwBar { double rho, ir, U, V, p, tl, il2, f4, qK; };
struct MomBar { double mu[7], mv[6], mx[3]; };

DFK_HD void zero(MaxwBar& b) { b.rho = b.ir = b.U = b.V = b.p = b.tl = b.il2 = b.f4 = b.qK = 0.0; }
DFK_HD void zero(MomBar& b) {
    for (int i = 0; i < 7; ++i) b.mu[i] = 0.0;
    for (int i = 0; i < 6; ++i) b.mv[i] = 0.0;
    for (int i = 0; i < 3; ++i) b.mx[i] = 0.0;
}

DFK_HD void maxw_of_vjp(const double W[4], const SchemeConsts& S, const Maxw& s, const MaxwBar& sb, double Wb[4]) {
    double tlb = sb.tl + sb.f4 * 2.0 * s.tl * S.inv_K2;
    double Ub = sb.U + sb.qK * 2.0 * s.U, Vb = sb.V + sb.qK * 2.0 * s.V;
    double il2b = sb.il2 + sb.qK * (S.K + 2.0);
    double pb = sb.p + il2b * s.ir;
    double irb = sb.ir + il2b * s.p;
    Wb[0] += tlb / s.p;
    pb += -tlb * s.tl / s.p;
    Wb[3] += pb * S.gm1;
    Wb[0] += -pb * S.gm1 * 0.5 * (s.U * s.U + s.V * s.V);
    Ub += -pb * S.gm1 * W[0] * s.U;
    Vb += -pb * S.gm1 * W[0] * s.V;
    Wb[1] += Ub * s.ir;
    Wb[2] += Vb * s.ir;
    irb += Ub * W[1] + Vb * W[2];
    Wb[0] += -irb * s.ir * s.ir + sb.rho;
}

// adjoint of fill_moments; accumulates into the state's U, V, il2 and tl adjoints
template <int HALF>
DFK_HD void fill_moments_vjp(const Maxw& s, double K, const Mom& m, MomBar& mb, MaxwBar& sb) {
    sb.il2 += mb.mx[1] * K + mb.mx[2] * K * (K + 2.0) * 2.0 * s.il2;
    for (int n = 5; n >= 2; --n) {
        double g = mb.mv[n];
        sb.V += g * m.mv[n - 1];
        mb.mv[n - 1] += g * s.V;
        sb.il2 += g * (double)(n - 1) * m.mv[n - 2];
        mb.mv[n - 2] += g * (double)(n - 1) * s.il2;
    }
    sb.V += mb.mv[1];
    for (int n = 6; n >= 2; --n) {
        double g = mb.mu[n];
        sb.U += g * m.mu[n - 1];
        mb.mu[n - 1] += g * s.U;
        sb.il2 += g * (double)(n - 1) * m.mu[n - 2];
        mb.mu[n - 2] += g * (double)(n - 1) * s.il2;
    }
    if (HALF == 0) {
        sb.U += mb.mu[1];
    } else {
        double lam = 0.5 * s.tl;
        double isl = rsqrt(lam);
        double x = lam * isl * s.U;
        double ex = exp(-x * x);
        double e = ex * (0.28209479177387814347 * isl);
        // mu1 = U mu0 +/- e
        sb.U += mb.mu[1] * m.mu[0];
        double mu0b = mb.mu[0] + mb.mu[1] * s.U;
        double eb = HALF > 0 ? mb.mu[1] : -mb.mu[1];
        // mu0 = erfc(-/+ x)/2: d/dx = +/- exp(-x^2)/sqrt(pi)
        double xb = mu0b * (HALF > 0 ? 1.0 : -1.0) * ex * 0.56418958354775628695;
        xb += eb * e * (-2.0 * x);
        double islb = eb * ex * 0.28209479177387814347;
        double lamb = xb * isl * s.U;
        islb += xb * lam * s.U;
        sb.U += xb * lam * isl;
        lamb += -0.5 * islb * isl * isl * isl;
        sb.tl += 0.5 * lamb;
    }
}

template <int k, int l, int c>
DFK_HD void M_vjp(const Mom& m, double g, MomBar& mb) {
    mb.mu[k] += g * m.mv[l] * m.mx[c];
    mb.mv[l] += g * m.mu[k] * m.mx[c];
    mb.mx[c] += g * m.mu[k] * m.mv[l];
}

template <int k, int l, int c>
DFK_HD void psi_mom_vjp(const Mom& m, const double ob[4], MomBar& mb) {
    M_vjp<k, l, c>(m, ob[0], mb);
    M_vjp<k + 1, l, c>(m, ob[1], mb);
    M_vjp<k, l + 1, c>(m, ob[2], mb);
    M_vjp<k + 2, l, c>(m, 0.5 * ob[3], mb);
    M_vjp<k, l + 2, c>(m, 0.5 * ob[3], mb);
    M_vjp<k, l, c + 1>(m, 0.5 * ob[3], mb);
}

// adjoint of the factorised a_mom (see its comment): ab += d out/d a ^T ob, moment adjoints accumulated
template <int k, int l>
DFK_HD void a_mom_vjp(const Mom& m, const double a[4], const double ob[4], MomBar& mb, double ab[4]) {
    const double* mu = m.mu;
    const double* mv = m.mv;
    const double h = 0.5 * a[3], x1 = m.mx[1], x2 = m.mx[2], hx1 = h * x1;
    double P[3], Qp[3];
    for (int j = 0; j < 3; ++j) {
        P[j] = a[0] * mu[k + j] + a[1] * mu[k + j + 1] + h * mu[k + j + 2];
        Qp[j] = a[2] * mv[l + j + 1] + h * mv[l + j + 2] + hx1 * mv[l + j];
    }
    const double Ql = a[2] * mv[l + 1] + h * mv[l + 2];
    const double g0 = ob[0], g1 = ob[1], g2 = ob[2], g3 = 0.5 * ob[3];
    double Pb[3] = {0.0, 0.0, 0.0}, Qpb[3] = {0.0, 0.0, 0.0}, Qlb = 0.0, hb = 0.0;
    // out0 = mv_l P0 + mu_k Qp0, out1 = mv_l P1 + mu_{k+1} Qp0, out2 = mv_{l+1} P0 + mu_k Qp1
    mb.mv[l] += g0 * P[0] + g1 * P[1] + g3 * P[2];
    mb.mu[k] += g0 * Qp[0] + g2 * Qp[1] + g3 * Qp[2];
    mb.mu[k + 1] += g1 * Qp[0];
    mb.mv[l + 1] += g2 * P[0];
    Pb[0] += g0 * mv[l] + g2 * mv[l + 1] + g3 * mv[l + 2];
    Pb[1] += g1 * mv[l];
    Pb[2] += g3 * mv[l];
    Qpb[0] += g0 * mu[k] + g1 * mu[k + 1] + g3 * mu[k + 2];
    Qpb[1] += g2 * mu[k];
    Qpb[2] += g3 * mu[k];
    // out3 / 2 = G(k+2,l,0) + G(k,l+2,0) + G(k,l,1): the first two above, then
    // G(k,l,1) = x1 (mv_l P0 + mu_k Ql) + h mu_k mv_l x2
    mb.mu[k + 2] += g3 * Qp[0];
    mb.mv[l + 2] += g3 * P[0];
    {
        const double gi = g3 * x1, t = g3 * h * x2;
        mb.mx[1] += g3 * (mv[l] * P[0] + mu[k] * Ql);
        mb.mv[l] += gi * P[0] + t * mu[k];
        mb.mu[k] += gi * Ql + t * mv[l];
        mb.mx[2] += g3 * h * mu[k] * mv[l];
        Pb[0] += gi * mv[l];
        Qlb += gi * mu[k];
        hb += g3 * mu[k] * mv[l] * x2;
    }
    // Qp_j = a2 mv_{l+j+1} + h mv_{l+j+2} + h x1 mv_{l+j},  Ql = a2 mv_{l+1} + h mv_{l+2}
    for (int j = 0; j < 3; ++j) {
        ab[2] += Qpb[j] * mv[l + j + 1];
        hb += Qpb[j] * (mv[l + j + 2] + x1 * mv[l + j]);
        mb.mv[l + j + 1] += Qpb[j] * a[2];
        mb.mv[l + j + 2] += Qpb[j] * h;
        mb.mv[l + j] += Qpb[j] * hx1;
        mb.mx[1] += Qpb[j] * h * mv[l + j];
    }
    ab[2] += Qlb * mv[l + 1];
    hb += Qlb * mv[l + 2];
    mb.mv[l + 1] += Qlb * a[2];
    mb.mv[l + 2] += Qlb * h;
    // P_j = a0 mu_{k+j} + a1 mu_{k+j+1} + h mu_{k+j+2}
    for (int j = 0; j < 3; ++j) {
        ab[0] += Pb[j] * mu[k + j];
        ab[1] += Pb[j] * mu[k + j + 1];
        hb += Pb[j] * mu[k + j + 2];
        mb.mu[k + j] += Pb[j] * a[0];
        mb.mu[k + j + 1] += Pb[j] * a[1];
        mb.mu[k + j + 2] += Pb[j] * h;
    }
    ab[3] += 0.5 * hb;
}

// The reverse of several a_mom of one (m, a) at once (the factorised form of a_mom): the output
// adjoints of each out<k, l> are accumulated into the adjoints of the shared P_k, Q_l, Qp_l terms
// (out_vjp), whose own reverse runs once (finish).  Needs KLO <= k, k + 2 <= KHI, LLO <= l,
// l + 2 <= LHI for every output.
template <int KLO, int KHI, int LLO, int LHI>
struct AMomRev {
    double P[KHI - KLO + 1], Q[LHI - LLO + 1], Qp[LHI - LLO + 1], h, x1, x2;
    double Pb[KHI - KLO + 1], Qb[LHI - LLO + 1], Qpb[LHI - LLO + 1], hb;
    DFK_HD AMomRev(const Mom& m, const double a[4]) {
        h = 0.5 * a[3];
        x1 = m.mx[1];
        x2 = m.mx[2];
        const double hx1 = h * x1;
        for (int j = KLO; j <= KHI; ++j) {
            P[j - KLO] = a[0] * m.mu[j] + a[1] * m.mu[j + 1] + h * m.mu[j + 2];
            Pb[j - KLO] = 0.0;
        }
        for (int j = LLO; j <= LHI; ++j) {
            Q[j - LLO] = a[2] * m.mv[j + 1] + h * m.mv[j + 2];
            Qp[j - LLO] = Q[j - LLO] + hx1 * m.mv[j];
            Qb[j - LLO] = 0.0;
            Qpb[j - LLO] = 0.0;
        }
        hb = 0.0;
    }
    template <int k, int l>
    DFK_HD void out_vjp(const Mom& m, const double ob[4], MomBar& mb) {
        const double* mu = m.mu;
        const double* mv = m.mv;
        const double g0 = ob[0], g1 = ob[1], g2 = ob[2], g3 = 0.5 * ob[3];
        const int pk = k - KLO, ql = l - LLO;
        // out0 = mv_l P_k + mu_k Qp_l, out1 = mv_l P_{k+1} + mu_{k+1} Qp_l, out2 = mv_{l+1} P_k + mu_k Qp_{l+1},
        // out3 / 2 = G(k+2,l,0) + G(k,l+2,0) + G(k,l,1)
        mb.mv[l] += g0 * P[pk] + g1 * P[pk + 1] + g3 * P[pk + 2];
        mb.mu[k] += g0 * Qp[ql] + g2 * Qp[ql + 1] + g3 * Qp[ql + 2];
        mb.mu[k + 1] += g1 * Qp[ql];
        mb.mv[l + 1] += g2 * P[pk];
        mb.mu[k + 2] += g3 * Qp[ql];
        mb.mv[l + 2] += g3 * P[pk];
        Pb[pk] += g0 * mv[l] + g2 * mv[l + 1] + g3 * mv[l + 2];
        Pb[pk + 1] += g1 * mv[l];
        Pb[pk + 2] += g3 * mv[l];
        Qpb[ql] += g0 * mu[k] + g1 * mu[k + 1] + g3 * mu[k + 2];
        Qpb[ql + 1] += g2 * mu[k];
        Qpb[ql + 2] += g3 * mu[k];
        // G(k,l,1) = x1 (mv_l P_k + mu_k Q_l) + h mu_k mv_l x2
        const double gi = g3 * x1, t = g3 * h * x2;
        mb.mx[1] += g3 * (mv[l] * P[pk] + mu[k] * Q[ql]);
        mb.mv[l] += gi * P[pk] + t * mu[k];
        mb.mu[k] += gi * Q[ql] + t * mv[l];
        mb.mx[2] += g3 * h * mu[k] * mv[l];
        Pb[pk] += gi * mv[l];
        Qb[ql] += gi * mu[k];
        hb += g3 * mu[k] * mv[l] * x2;
    }
    DFK_HD void finish(const Mom& m, const double a[4], MomBar& mb, double ab[4]) {
        const double* mu = m.mu;
        const double* mv = m.mv;
        const double hx1 = h * x1;
        for (int j = LLO; j <= LHI; ++j) {
            const int q = j - LLO;
            // Qp_j = Q_j + h x1 mv_j, Q_j = a2 mv_{j+1} + h mv_{j+2}
            const double qb = Qb[q] + Qpb[q];
            hb += Qpb[q] * x1 * mv[j] + qb * mv[j + 2];
            mb.mx[1] += Qpb[q] * h * mv[j];
            mb.mv[j] += Qpb[q] * hx1;
            ab[2] += qb * mv[j + 1];
            mb.mv[j + 1] += qb * a[2];
            mb.mv[j + 2] += qb * h;
        }
        for (int j = KLO; j <= KHI; ++j) {
            const double pb = Pb[j - KLO];
            ab[0] += pb * mu[j];
            ab[1] += pb * mu[j + 1];
            hb += pb * mu[j + 2];
            mb.mu[j] += pb * a[0];
            mb.mu[j + 1] += pb * a[1];
            mb.mu[j + 2] += pb * h;
        }
        ab[3] += 0.5 * hb;
    }
};

// adjoint of slope_solve: bb += S^T ab, state adjoints accumulated
DFK_HD void slope_solve_vjp(const Maxw& s, const double b[4], const double abin[4], double bb[4], MaxwBar& sb) {
    double R2 = b[1] - s.U * b[0], R3 = b[2] - s.V * b[0], R4 = 2.0 * b[3] - s.qK * b[0];
    double X = R4 - 2.0 * s.U * R2 - 2.0 * s.V * R3;
    double a3 = s.f4 * X;
    double a2 = s.tl * R3 - s.V * a3;
    double a1 = s.tl * R2 - s.U * a3;
    double ab0 = abin[0], ab1 = abin[1], ab2 = abin[2], ab3 = abin[3];
    // a0 = b0 - U a1 - V a2 - a3 qK / 2
    bb[0] += ab0;
    sb.U += -ab0 * a1;
    ab1 += -ab0 * s.U;
    sb.V += -ab0 * a2;
    ab2 += -ab0 * s.V;
    ab3 += -ab0 * 0.5 * s.qK;
    sb.qK += -ab0 * 0.5 * a3;
    // a1 = tl R2 - U a3
    sb.tl += ab1 * R2;
    double R2b = ab1 * s.tl;
    sb.U += -ab1 * a3;
    ab3 += -ab1 * s.U;
    // a2 = tl R3 - V a3
    sb.tl += ab2 * R3;
    double R3b = ab2 * s.tl;
    sb.V += -ab2 * a3;
    ab3 += -ab2 * s.V;
    // a3 = f4 X
    sb.f4 += ab3 * X;
    double Xb = ab3 * s.f4;
    double R4b = Xb;
    sb.U += -Xb * 2.0 * R2;
    R2b += -Xb * 2.0 * s.U;
    sb.V += -Xb * 2.0 * R3;
    R3b += -Xb * 2.0 * s.V;
    bb[3] += 2.0 * R4b;
    sb.qK += -R4b * b[0];
    bb[0] += -R4b * s.qK;
    bb[2] += R3b;
    sb.V += -R3b * b[0];
    bb[0] += -R3b * s.V;
    bb[1] += R2b;
    sb.U += -R2b * b[0];
    bb[0] += -R2b * s.U;
}

// value and derivative with respect to tau_n/dt of the combined time coefficients of Eq. 27
struct Dual { double v, d; };
DFK_HD Dual dmul(Dual a, Dual b) { return Dual{a.v * b.v, a.d * b.v + a.v * b.d}; }
DFK_HD Dual dadd(Dual a, Dual b) { return Dual{a.v + b.v, a.d + b.d}; }
DFK_HD Dual dsub(Dual a, Dual b) { return Dual{a.v - b.v, a.d - b.d}; }
DFK_HD Dual dscale(double c, Dual a) { return Dual{c * a.v, c * a.d}; }

struct TimeCoeffs { Dual gcF, gcD, acF, acD, AcF, AcD, glrF, glrD, alrF, alrD, AlrF, AlrD; };

DFK_HD TimeCoeffs time_coeffs(double rT, double dt, int tau_reading) {
    Dual r = {rT, 1.0};
    Dual T = dscale(dt, r);
    Dual tau = tau_reading == 1 ? T : Dual{0.0, 0.0};
    Dual E2 = {0.0, 0.0}, rr = {0.0, 0.0};
    if (dbits(rT) > 0) { double e = exp(-0.5 / rT); E2 = Dual{e, e * 0.5 / (rT * rT)}; rr = r; }
    Dual E1 = dmul(E2, E2);
    Dual om = dsub(Dual{1.0, 0.0}, E2);
    Dual S3 = dmul(om, dsub(Dual{3.0, 0.0}, E2));
    double idt = 1.0 / dt;
    TimeCoeffs c;
    c.glrF = dmul(rr, S3);
    c.glrD = dscale(-4.0 * idt, dmul(rr, dmul(om, om)));
    c.gcF = dsub(Dual{1.0, 0.0}, c.glrF);
    c.gcD = dscale(-1.0, c.glrD);
    Dual TT = dadd(dmul(T, T), dmul(T, tau));
    c.acF = dsub(dadd(dsub(dscale(idt, dmul(TT, S3)), dscale(2.0, dmul(T, E2))), dmul(T, E1)), tau);
    c.acD = dscale(4.0 * idt * idt, dadd(dscale(-1.0, dmul(TT, dmul(om, om))), dscale(dt, dmul(T, dmul(E2, om)))));
    c.AcF = dadd(dscale(-1.0, tau), dmul(tau, dmul(rr, S3)));
    c.AcD = dsub(Dual{1.0, 0.0}, dscale(4.0 * idt * idt, dmul(dmul(T, tau), dmul(om, om))));
    c.alrF = dsub(dscale(-1.0, c.acF), tau);
    c.alrD = dscale(-1.0, c.acD);
    c.AlrF = dscale(-idt, dmul(dmul(T, tau), S3));
    c.AlrD = dscale(4.0 * idt * idt, dmul(dmul(T, tau), dmul(om, om)));
    return c;
}

struct GPStateBar { double W[4], Wn[4], Wt[4]; };

template <class Tape>
DFK_HD Maxw tape_get_maxw(const Tape& tp, int b) {
    Maxw s;
    s.rho = tp.get(b); s.ir = tp.get(b + 1); s.U = tp.get(b + 2); s.V = tp.get(b + 3); s.p = tp.get(b + 4);
    s.il2 = tp.get(b + 5); s.tl = tp.get(b + 6); s.f4 = tp.get(b + 7); s.qK = tp.get(b + 8);
    return s;
}
template <class Tape>
DFK_HD void tape_get_mom(const Tape& tp, int b, Mom& m) {
    for (int n = 0; n < 7; ++n) m.mu[n] = tp.get(b + n);
    for (int n = 0; n < 6; ++n) m.mv[n] = tp.get(b + 7 + n);
    for (int n = 0; n < 3; ++n) m.mx[n] = tp.get(b + 13 + n);
}
template <class Tape>
DFK_HD void tape_get_vec(const Tape& tp, int b, double v[4]) {
    for (int i = 0; i < 4; ++i) v[i] = tp.get(b + i);
}

// under the tau = tau_n reading, one side's slope coefficients A of the time derivative of its
// Maxwellian (from the compatibility condition over the full velocity space) and <u A psi> over the
// side's half space, recomputed from the tape.  SIGN +1: left side, -1: right side.
template <int SIGN, class Tape>
DFK_HD void tau_side_terms(const Tape& tp, const Maxw& s, double K, Mom& mF, double bA[4], double A[4]) {
    double ax[4], ay[4], t1[4], t2[4];
    tape_get_vec(tp, SIGN > 0 ? TG_ALX : TG_ARX, ax);
    tape_get_vec(tp, SIGN > 0 ? TG_ALY : TG_ARY, ay);
    fill_moments<0>(s, K, mF);
    a_mom<1, 0>(mF, ax, t1);
    a_mom<0, 1>(mF, ay, t2);
    for (int i = 0; i < 4; ++i) bA[i] = -(t1[i] + t2[i]);
    slope_solve(s, bA, A);
}

// reverse of one side's share of gks_flux (SIGN +1 left, -1 right): its half-space moment sums in
// the flux, in the kinetic weighting of the equilibrium state and in its slopes, its slope
// coefficients and (tau = tau_n) its extra terms; accumulates into the side's Maxwellian adjoint sb
// and the Gauss-point state adjoint Pb.  The sides are reversed one after the other so that only
// one side's moments and their adjoints are live at a time.
template <int SIGN, class Tape>
DFK_HD void gks_side_reverse(const Tape& tp, const GPState& P, const Maxw& s, const SchemeConsts& S,
                             const double Wcb[4], const double Wcxb[4], const double Wcyb[4], const double M0b[4],
                             const double M1b[4], const double M2b[4], MaxwBar& sb, GPStateBar& Pb) {
    constexpr bool left = SIGN > 0;
    Mom m;
    tape_get_mom(tp, left ? TG_ML : TG_MR, m);
    MomBar mb;
    zero(mb);
    double axb[4] = {0, 0, 0, 0}, ayb[4] = {0, 0, 0, 0};
    if (S.tau_reading == 1) {
        Mom mF;
        double bA[4], A[4], Ab[4] = {0, 0, 0, 0}, bAb[4] = {0, 0, 0, 0}, nb[4], ax[4], ay[4];
        tau_side_terms<SIGN>(tp, s, S.K, mF, bA, A);
        a_mom_vjp<1, 0>(m, A, M2b, mb, Ab);
        slope_solve_vjp(s, bA, Ab, bAb, sb);
        for (int i = 0; i < 4; ++i) nb[i] = -bAb[i];
        tape_get_vec(tp, left ? TG_ALX : TG_ARX, ax);
        tape_get_vec(tp, left ? TG_ALY : TG_ARY, ay);
        MomBar mFb;
        zero(mFb);
        a_mom_vjp<1, 0>(mF, ax, nb, mFb, axb);
        a_mom_vjp<0, 1>(mF, ay, nb, mFb, ayb);
        fill_moments_vjp<0>(s, S.K, mF, mFb, sb);
    }
    // flux moments <u psi> of the side's initial distribution
    psi_mom_vjp<1, 0, 0>(m, M0b, mb);
    // kinetic weighting of the equilibrium state and its slopes
    double pb[4], tb[4];
    const int tp0 = left ? TG_PL0 : TG_PR0, tx0 = left ? TG_LX0 : TG_RX0, ty0 = left ? TG_LY0 : TG_RY0;
    for (int i = 0; i < 4; ++i) {
        sb.rho += Wcb[i] * tp.get(tp0 + i) + Wcxb[i] * tp.get(tx0 + i) + Wcyb[i] * tp.get(ty0 + i);
        pb[i] = Wcb[i] * s.rho;
    }
    psi_mom_vjp<0, 0, 0>(m, pb, mb);
    // the side's moment sums of a_x (kinetic weighting, flux moment) and of a_y, each reversed as one
    {
        double ax[4];
        tape_get_vec(tp, left ? TG_ALX : TG_ARX, ax);
        AMomRev<0, 4, 0, 2> X(m, ax);
        for (int i = 0; i < 4; ++i) tb[i] = Wcxb[i] * s.rho;
        X.out_vjp<0, 0>(m, tb, mb);
        X.out_vjp<2, 0>(m, M1b, mb);
        X.finish(m, ax, mb, axb);
    }
    {
        double ay[4];
        tape_get_vec(tp, left ? TG_ALY : TG_ARY, ay);
        AMomRev<0, 3, 0, 3> Y(m, ay);
        for (int i = 0; i < 4; ++i) tb[i] = Wcyb[i] * s.rho;
        Y.out_vjp<0, 0>(m, tb, mb);
        Y.out_vjp<1, 1>(m, M1b, mb);
        Y.finish(m, ay, mb, ayb);
    }
    // slope coefficients from the side's normal and tangential slopes (b = W_n / rho, W_t / rho)
    double b[4], bb[4] = {0, 0, 0, 0};
    for (int i = 0; i < 4; ++i) b[i] = P.Wn[i] * s.ir;
    slope_solve_vjp(s, b, axb, bb, sb);
    for (int i = 0; i < 4; ++i) {
        Pb.Wn[i] += bb[i] * s.ir;
        sb.ir += bb[i] * P.Wn[i];
        bb[i] = 0.0;
        b[i] = P.Wt[i] * s.ir;
    }
    slope_solve_vjp(s, b, ayb, bb, sb);
    for (int i = 0; i < 4; ++i) { Pb.Wt[i] += bb[i] * s.ir; sb.ir += bb[i] * P.Wt[i]; }
    fill_moments_vjp<SIGN>(s, S.K, m, mb, sb);
    maxw_of_vjp(P.W, S, s, sb, Pb.W);
}

// reverse of gks_flux from its taped forward intermediates: given Fb, dFb (local frame) accumulates
// into Lb, Rb.  The tau = tau_n reading's extra terms are recomputed from the tape.  Taped values
// are read where they are used: the reverse holds many adjoint accumulators at once, and values
// kept live from the start would spill.
template <class Tape>
DFK_HD void gks_flux_reverse(const Tape& tp, const GPState& L, const GPState& R, double dt, const SchemeConsts& S,
                             const double Fb[4], const double dFb[4], GPStateBar& Lb, GPStateBar& Rb) {
    const double K = S.K;
    const Maxw sl = tape_get_maxw(tp, TG_SL), sr = tape_get_maxw(tp, TG_SR), sc = tape_get_maxw(tp, TG_SC);
    const double q = tp.get(TG_Q);
    double rT = S.C1 + S.C2 * fabs(q);
    TimeCoeffs tc = time_coeffs(rT, dt, S.tau_reading);
    double Ml2[4] = {0, 0, 0, 0}, Mr2[4] = {0, 0, 0, 0};
    if (S.tau_reading == 1) {
        Mom m, mF;
        double bA[4], A[4];
        tau_side_terms<+1>(tp, sl, K, mF, bA, A);
        tape_get_mom(tp, TG_ML, m);
        a_mom<1, 0>(m, A, Ml2);
        tau_side_terms<-1>(tp, sr, K, mF, bA, A);
        tape_get_mom(tp, TG_MR, m);
        a_mom<1, 0>(m, A, Mr2);
    }
    // ---- reverse of the final combination
    MaxwBar slb, srb, scb;
    zero(slb); zero(srb); zero(scb);
    double Mc0b[4], Mc1b[4], Mc2b[4], Ml0b[4], Mr0b[4], Ml1b[4], Mr1b[4], Ml2b[4], Mr2b[4];
    double rTb = 0.0;
    for (int i = 0; i < 4; ++i) {
        const double Mc0 = tp.get(TG_MC0 + i), Mc1 = tp.get(TG_MC1 + i), Mc2 = tp.get(TG_MC2 + i);
        const double Ml0 = tp.get(TG_ML0 + i), Mr0 = tp.get(TG_MR0 + i);
        const double Ml1 = tp.get(TG_ML1 + i), Mr1 = tp.get(TG_MR1 + i);
        double c0 = sc.rho * Mc0, c1 = sc.rho * Mc1, c2 = sc.rho * Mc2;
        double g0 = sl.rho * Ml0 + sr.rho * Mr0;
        double g1 = sl.rho * Ml1 + sr.rho * Mr1;
        double g2 = sl.rho * Ml2[i] + sr.rho * Mr2[i];
        double c0b = Fb[i] * tc.gcF.v + dFb[i] * tc.gcD.v;
        double c1b = Fb[i] * tc.acF.v + dFb[i] * tc.acD.v;
        double c2b = Fb[i] * tc.AcF.v + dFb[i] * tc.AcD.v;
        double g0b = Fb[i] * tc.glrF.v + dFb[i] * tc.glrD.v;
        double g1b = Fb[i] * tc.alrF.v + dFb[i] * tc.alrD.v;
        double g2b = Fb[i] * tc.AlrF.v + dFb[i] * tc.AlrD.v;
        rTb += Fb[i] * (tc.gcF.d * c0 + tc.acF.d * c1 + tc.AcF.d * c2 + tc.glrF.d * g0 + tc.alrF.d * g1 + tc.AlrF.d * g2)
             + dFb[i] * (tc.gcD.d * c0 + tc.acD.d * c1 + tc.AcD.d * c2 + tc.glrD.d * g0 + tc.alrD.d * g1 + tc.AlrD.d * g2);
        scb.rho += c0b * Mc0 + c1b * Mc1 + c2b * Mc2;
        Mc0b[i] = c0b * sc.rho; Mc1b[i] = c1b * sc.rho; Mc2b[i] = c2b * sc.rho;
        slb.rho += g0b * Ml0 + g1b * Ml1 + g2b * Ml2[i];
        srb.rho += g0b * Mr0 + g1b * Mr1 + g2b * Mr2[i];
        Ml0b[i] = g0b * sl.rho; Ml1b[i] = g1b * sl.rho; Ml2b[i] = g2b * sl.rho;
        Mr0b[i] = g0b * sr.rho; Mr1b[i] = g1b * sr.rho; Mr2b[i] = g2b * sr.rho;
    }
    // tau_n / dt = C1 + C2 |(pl - pr)/(pl + pr)|
    {
        double sg = q >= 0.0 ? 1.0 : -1.0;
        double den = (sl.p + sr.p) * (sl.p + sr.p);
        slb.p += rTb * S.C2 * sg * 2.0 * sr.p / den;
        srb.p += rTb * S.C2 * sg * (-2.0) * sl.p / den;
    }
    // ---- the equilibrium state's part: its flux moments and the compatibility condition of A^c
    // (the moment sums of a_x and of a_y reversed together: their outputs share P, Q terms), its
    // slopes and its Maxwellian
    double Wcb[4] = {0, 0, 0, 0}, Wcxb[4], Wcyb[4];
    {
        Mom mc;
        tape_get_mom(tp, TG_MC, mc);
        MomBar mcb;
        zero(mcb);
        double Acb[4] = {0, 0, 0, 0}, bctb[4] = {0, 0, 0, 0}, acxb[4] = {0, 0, 0, 0}, acyb[4] = {0, 0, 0, 0};
        psi_mom_vjp<1, 0, 0>(mc, Mc0b, mcb);
        {
            double Ac[4];
            tape_get_vec(tp, TG_AC, Ac);
            a_mom_vjp<1, 0>(mc, Ac, Mc2b, mcb, Acb);
        }
        {
            double bct[4];
            tape_get_vec(tp, TG_BCT, bct);
            slope_solve_vjp(sc, bct, Acb, bctb, scb);
        }
        {
            double acx[4], acy[4], nb[4];
            tape_get_vec(tp, TG_ACX, acx);
            tape_get_vec(tp, TG_ACY, acy);
            for (int i = 0; i < 4; ++i) nb[i] = -bctb[i];
            AMomRev<1, 4, 0, 2> Cx(mc, acx);
            AMomRev<0, 3, 0, 3> Cy(mc, acy);
            Cx.out_vjp<2, 0>(mc, Mc1b, mcb);
            Cx.out_vjp<1, 0>(mc, nb, mcb);
            Cx.finish(mc, acx, mcb, acxb);
            Cy.out_vjp<1, 1>(mc, Mc1b, mcb);
            Cy.out_vjp<0, 1>(mc, nb, mcb);
            Cy.finish(mc, acy, mcb, acyb);
        }
        {
            double Wcx[4], Wcy[4], bcx[4], bcy[4], bcxb[4] = {0, 0, 0, 0}, bcyb[4] = {0, 0, 0, 0};
            tape_get_vec(tp, TG_WCX, Wcx);
            tape_get_vec(tp, TG_WCY, Wcy);
            for (int i = 0; i < 4; ++i) { bcx[i] = Wcx[i] * sc.ir; bcy[i] = Wcy[i] * sc.ir; }
            slope_solve_vjp(sc, bcx, acxb, bcxb, scb);
            slope_solve_vjp(sc, bcy, acyb, bcyb, scb);
            for (int i = 0; i < 4; ++i) {
                Wcxb[i] = bcxb[i] * sc.ir;
                Wcyb[i] = bcyb[i] * sc.ir;
                scb.ir += bcxb[i] * Wcx[i] + bcyb[i] * Wcy[i];
            }
        }
        fill_moments_vjp<0>(sc, K, mc, mcb, scb);
        double Wc[4];
        tape_get_vec(tp, TG_WC, Wc);
        maxw_of_vjp(Wc, S, sc, scb, Wcb);
    }
    // ---- the two sides
    gks_side_reverse<+1>(tp, L, sl, S, Wcb, Wcxb, Wcyb, Ml0b, Ml1b, Ml2b, slb, Lb);
    gks_side_reverse<-1>(tp, R, sr, S, Wcb, Wcxb, Wcyb, Mr0b, Mr1b, Mr2b, srb, Rb);
}

// adjoint of gks_flux: the forward recomputed into a local tape, then its reverse
DFK_HD void gks_flux_vjp(const GPState& L, const GPState& R, double dt, const SchemeConsts& S,
                         const double Fb[4], const double dFb[4], GPStateBar& Lb, GPStateBar& Rb) {
    double t[TG_COUNT], F[4], dF[4];
    ArrayTape tp{t};
    gks_flux_t(L, R, dt, S, F, dF, tp);
    gks_flux_reverse(tp, L, R, dt, S, Fb, dFb, Lb, Rb);
}

// ------------------------------------------------------------------------------------------
// Lax-Friedrichs flux
// ------------------------------------------------------------------------------------------
struct EulerBar { double u, v, p, c, H, q; };

DFK_HD void euler_pt_vjp(const double W[4], const SchemeConsts& S, const EulerPt& e, EulerBar eb, double Wb[4]) {
    double ir = 1.0 / W[0];
    double irb = 0.0;
    Wb[3] += eb.H * ir;
    eb.p += eb.H * ir;
    irb += eb.H * (W[3] + e.p);
    double sb = eb.c * 0.5 / e.c;
    eb.p += sb * S.gamma * ir;
    irb += sb * S.gamma * e.p;
    Wb[3] += eb.p * S.gm1;
    Wb[0] += -eb.p * S.gm1 * e.q;
    eb.q += -eb.p * S.gm1 * W[0];
    eb.u += eb.q * e.u;
    eb.v += eb.q * e.v;
    Wb[1] += eb.u * ir;
    Wb[2] += eb.v * ir;
    irb += eb.u * W[1] + eb.v * W[2];
    Wb[0] += -irb * ir * ir;
}

DFK_HD void jac_dp_vjp(const EulerPt& e, double gm1, const double X[4], double dpb, EulerBar& eb, double Xb[4]) {
    Xb[3] += dpb * gm1;
    eb.u += -dpb * gm1 * X[1];
    Xb[1] += -dpb * gm1 * e.u;
    eb.v += -dpb * gm1 * X[2];
    Xb[2] += -dpb * gm1 * e.v;
    eb.q += dpb * gm1 * X[0];
    Xb[0] += dpb * gm1 * e.q;
}

DFK_HD void jac_x_vjp(const EulerPt& e, double gm1, const double X[4], const double Yb[4], EulerBar& eb, double Xb[4]) {
    double dp = gm1 * (X[3] - e.u * X[1] - e.v * X[2] + e.q * X[0]);
    double dpb = 0.0;
    Xb[1] += Yb[0];
    eb.u += Yb[1] * (2.0 * X[1] - 2.0 * e.u * X[0]);
    Xb[1] += Yb[1] * 2.0 * e.u;
    Xb[0] += -Yb[1] * e.u * e.u;
    dpb += Yb[1];
    eb.v += Yb[2] * (X[1] - e.u * X[0]);
    Xb[1] += Yb[2] * e.v;
    eb.u += Yb[2] * (X[2] - e.v * X[0]);
    Xb[2] += Yb[2] * e.u;
    Xb[0] += -Yb[2] * e.u * e.v;
    eb.u += Yb[3] * ((X[3] + dp) - e.H * X[0]);
    Xb[3] += Yb[3] * e.u;
    dpb += Yb[3] * e.u;
    eb.H += Yb[3] * (X[1] - e.u * X[0]);
    Xb[1] += Yb[3] * e.H;
    Xb[0] += -Yb[3] * e.H * e.u;
    jac_dp_vjp(e, gm1, X, dpb, eb, Xb);
}

DFK_HD void jac_y_vjp(const EulerPt& e, double gm1, const double X[4], const double Yb[4], EulerBar& eb, double Xb[4]) {
    double dp = gm1 * (X[3] - e.u * X[1] - e.v * X[2] + e.q * X[0]);
    double dpb = 0.0;
    Xb[2] += Yb[0];
    eb.v += Yb[1] * (X[1] - e.u * X[0]);
    Xb[1] += Yb[1] * e.v;
    eb.u += Yb[1] * (X[2] - e.v * X[0]);
    Xb[2] += Yb[1] * e.u;
    Xb[0] += -Yb[1] * e.u * e.v;
    eb.v += Yb[2] * (2.0 * X[2] - 2.0 * e.v * X[0]);
    Xb[2] += Yb[2] * 2.0 * e.v;
    Xb[0] += -Yb[2] * e.v * e.v;
    dpb += Yb[2];
    eb.v += Yb[3] * ((X[3] + dp) - e.H * X[0]);
    Xb[3] += Yb[3] * e.v;
    dpb += Yb[3] * e.v;
    eb.H += Yb[3] * (X[2] - e.v * X[0]);
    Xb[2] += Yb[3] * e.H;
    Xb[0] += -Yb[3] * e.H * e.v;
    jac_dp_vjp(e, gm1, X, dpb, eb, Xb);
}

DFK_HD void lf_flux_vjp(const GPState& L, const GPState& R, const SchemeConsts& S, const double Fb[4],
                        const double dFb[4], GPStateBar& Lb, GPStateBar& Rb) {
    EulerPt el = euler_pt(L.W, S), er = euler_pt(R.W, S);
    double sL = fabs(el.u) + el.c, sR = fabs(er.u) + er.c;
    bool left = !nn_less(sL, sR);                 // the left speed on a tie (both >= 0)
    double s = left ? sL : sR;
    double t1[4], t2[4], WtL[4], WtR[4];
    jac_x(el, S.gm1, L.Wn, t1); jac_y(el, S.gm1, L.Wt, t2);
    for (int i = 0; i < 4; ++i) WtL[i] = -(t1[i] + t2[i]);
    jac_x(er, S.gm1, R.Wn, t1); jac_y(er, S.gm1, R.Wt, t2);
    for (int i = 0; i < 4; ++i) WtR[i] = -(t1[i] + t2[i]);
    EulerBar elb = {0, 0, 0, 0, 0, 0}, erb = {0, 0, 0, 0, 0, 0};
    double sb = 0.0, WtLb[4] = {0, 0, 0, 0}, WtRb[4] = {0, 0, 0, 0}, AXb[4];
    for (int i = 0; i < 4; ++i) {
        sb += -0.5 * Fb[i] * (R.W[i] - L.W[i]) - 0.5 * dFb[i] * (WtR[i] - WtL[i]);
        Rb.W[i] += -0.5 * s * Fb[i];
        Lb.W[i] += 0.5 * s * Fb[i];
        WtRb[i] += -0.5 * s * dFb[i];
        WtLb[i] += 0.5 * s * dFb[i];
        AXb[i] = 0.5 * dFb[i];
    }
    // A(W_side) W_t,side
    jac_x_vjp(el, S.gm1, WtL, AXb, elb, WtLb);
    jac_x_vjp(er, S.gm1, WtR, AXb, erb, WtRb);
    // W_t = -(A W_n + B W_t)
    double nb[4];
    for (int i = 0; i < 4; ++i) nb[i] = -WtLb[i];
    jac_x_vjp(el, S.gm1, L.Wn, nb, elb, Lb.Wn);
    jac_y_vjp(el, S.gm1, L.Wt, nb, elb, Lb.Wt);
    for (int i = 0; i < 4; ++i) nb[i] = -WtRb[i];
    jac_x_vjp(er, S.gm1, R.Wn, nb, erb, Rb.Wn);
    jac_y_vjp(er, S.gm1, R.Wt, nb, erb, Rb.Wt);
    // the two Euler fluxes, F = (m, m u + p, m v, u (E + p))
    const GPState* sides[2] = {&L, &R};
    EulerPt* es[2] = {&el, &er};
    EulerBar* ebs[2] = {&elb, &erb};
    GPStateBar* bs[2] = {&Lb, &Rb};
    for (int k = 0; k < 2; ++k) {
        const double* W = sides[k]->W;
        const EulerPt& e = *es[k];
        EulerBar& eb = *ebs[k];
        double* Wb = bs[k]->W;
        double g0 = 0.5 * Fb[0], g1 = 0.5 * Fb[1], g2 = 0.5 * Fb[2], g3 = 0.5 * Fb[3];
        Wb[1] += g0 + g1 * e.u + g2 * e.v;
        eb.u += g1 * W[1] + g3 * (W[3] + e.p);
        eb.p += g1 + g3 * e.u;
        eb.v += g2 * W[1];
        Wb[3] += g3 * e.u;
    }
    // wave speed s = max(|u_l| + c_l, |u_r| + c_r)
    if (left) { elb.u += sb * (el.u >= 0.0 ? 1.0 : -1.0); elb.c += sb; }
    else { erb.u += sb * (er.u >= 0.0 ? 1.0 : -1.0); erb.c += sb; }
    euler_pt_vjp(L.W, S, el, elb, Lb.W);
    euler_pt_vjp(R.W, S, er, erb, Rb.W);
}

}  // namespace dfk
