// dfgks_device.cuh -- FP64 device arithmetic of the hybrid DF + WENO-AO finite-volume scheme
// (Zhang, Ji & Xu, arXiv 2402.10914) for sm_103a.  Every routine works on one face line, one
// face side or one Gauss point in that face's local frame (Sect. 2.1); the kernels in
// dfgks_kernels.cu move data between them.
//
// Arithmetic choices (each algebraically identical to the paper's formulas):
//   * characteristic projection L W and back-projection R Q in factored form (12 + 14 flops
//     instead of two 4x4 products);
//   * WENO-AO sub-stencil polynomials kept as cell-centred coefficients a1..a4 (the cell mean
//     fixes a0), so smoothness indicators (Eq. 38) and every evaluation point share them;
//   * S2O4 flux coefficients (Eq. 27) combined analytically per kinetic term before the moments
//     are summed, using E(dt) = E(dt/2)^2, which avoids the cancellation of 4(F(dt)-2F(dt/2));
//   * the GKS slope system <a psi> = b (Sect. 2.2) solved in closed form.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

// every arithmetic routine also compiles for the host, so its derivatives can be checked there
#define DFK_HD __host__ __device__ __forceinline__

namespace dfk {

constexpr int G = 3;                       // ghost layers: the normal stencil spans i-3 .. i+2
constexpr double kGaussEta = 0.28867513459481288225;   // sqrt(3)/6: Gauss points at eta = -/+ this

// Order of doubles on their bit patterns.  Read as signed 64-bit integers, the IEEE encodings of
// +0 .. +inf compare as the values do, and every negative value (-0 included) reads as negative.
// Maxima, minima and tests of quantities that are never negative (WENO ratios and weight sums, DF
// factors, products of positive states) run on the integer units this way, leaving the FP64 units
// (two per SM) to the arithmetic; the results are the same bits as fmax / fmin / < on such values.
DFK_HD long long dbits(double x) {
#ifdef __CUDA_ARCH__
    return __double_as_longlong(x);
#else
    long long b;
    memcpy(&b, &x, sizeof b);
    return b;
#endif
}
DFK_HD double dval(long long b) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double(b);
#else
    double x;
    memcpy(&x, &b, sizeof x);
    return x;
#endif
}
DFK_HD double nn_max(double a, double b) { const long long x = dbits(a), y = dbits(b); return dval(x > y ? x : y); }
DFK_HD double nn_min(double a, double b) { const long long x = dbits(a), y = dbits(b); return dval(x < y ? x : y); }
// a < b for a >= +0 (b of any sign)
DFK_HD bool nn_less(double a, double b) { return dbits(a) < dbits(b); }
// lo < a < hi for lo, hi > 0: false for a negative, -0 or NaN
DFK_HD bool in_range(double a, double lo, double hi) { const long long x = dbits(a); return dbits(lo) < x && x < dbits(hi); }

struct SchemeConsts {
    double gamma, gm1, K, inv_K2;          // gamma, gamma-1, internal degrees of freedom, 1/(K+2)
    double r2g;                            // sqrt(2/gamma): 1/c = sqrt(2/gamma) sqrt(lambda)
    double d[4];                           // WENO-AO linear weights d0..d3 (Sect. 3.1)
    double inv_d3;
    double eps, alpha_thres, C1, C2;
    int time_limiter, tau_reading, gp_fallback;
    int df_states;                         // DF factor from 0: Gauss-point states, 1: the face's two cell averages
};

// ------------------------------------------------------------------------------------------
// Euler state helpers
// ------------------------------------------------------------------------------------------
DFK_HD double pressure_of(const double W[4], double gm1) {
    return gm1 * (W[3] - 0.5 * (W[1] * W[1] + W[2] * W[2]) / W[0]);
}

// rotate a global-frame state into the local frame of a y-face (theta = pi/2): (rho, rhoV, -rhoU, rhoE)
template <int DIR>
DFK_HD void to_local(double W[4]) {
    if (DIR == 1) { double m = W[1]; W[1] = W[2]; W[2] = -m; }
}
// local-frame flux back to the global frame, F = T^{-1} F~
template <int DIR>
DFK_HD void to_global(double F[4]) {
    if (DIR == 1) { double a = F[1]; F[1] = -F[2]; F[2] = a; }
}

// ------------------------------------------------------------------------------------------
// Characteristic basis of the local-frame x-direction Euler Jacobian at W = (W_l + W_r)/2
// ------------------------------------------------------------------------------------------
struct CharBasis { double u, v, c, ic, H, b1, b2, q2; };

DFK_HD CharBasis make_basis(const double Wl[4], const double Wr[4], const SchemeConsts& S) {
    CharBasis B;
    double r = 0.5 * (Wl[0] + Wr[0]), m = 0.5 * (Wl[1] + Wr[1]);
    double n = 0.5 * (Wl[2] + Wr[2]), E = 0.5 * (Wl[3] + Wr[3]);
    double ir = 1.0 / r;
    B.u = m * ir;
    B.v = n * ir;
    B.q2 = 0.5 * (B.u * B.u + B.v * B.v);
    double p = S.gm1 * (E - r * B.q2);
    const double c2 = S.gamma * p * ir;
    B.ic = rsqrt(c2);                  // one reciprocal square root for 1/c and c = c^2 / c
    B.c = c2 * B.ic;
    B.H = (E + p) * ir;
    B.b1 = S.gm1 * B.ic * B.ic;
    B.b2 = B.q2 * B.b1;
    return B;
}

// Q = L W; components ordered by eigenvalue u-c, u (entropy), u (shear), u+c
DFK_HD void project(const CharBasis& B, const double W[4], double Q[4]) {
    double t = B.b1 * (B.u * W[1] + B.v * W[2] - W[3]);
    double k = B.b2 * W[0] - t;
    double m = (B.u * W[0] - W[1]) * B.ic;
    Q[0] = 0.5 * (k + m);
    Q[1] = W[0] - k;
    Q[2] = W[2] - B.v * W[0];
    Q[3] = 0.5 * (k - m);
}

// W = R Q
DFK_HD void back_project(const CharBasis& B, const double Q[4], double W[4]) {
    double s = Q[0] + Q[3], d = Q[3] - Q[0];
    W[0] = s + Q[1];
    W[1] = B.u * W[0] + B.c * d;
    W[2] = B.v * W[0] + Q[2];
    W[3] = B.H * s + B.u * B.c * d + B.q2 * Q[1] + B.v * Q[2];
}

// ------------------------------------------------------------------------------------------
// WENO-AO(5,3) of Sect. 3.1 on Q_{-2..2} (cell-centred xi in [-1/2, 1/2] of the centre cell).
// Each sub-stencil polynomial is written p_k = Q_0 + a1 xi + a2 (xi^2 - 1/12) (+ a3 xi^3 + a4 (xi^4 - 1/80)
// for the quartic), so its cell mean is Q_0 by construction.  The AO polynomial P = sum c_k p_k with
// c3 = wb3/d3 and c_k = wb_k - c3 d_k sums to one, so P = Q_0 + A1 xi + A2 (xi^2-1/12) + c3 (a3 xi^3 + a4 (xi^4-1/80)).
// ------------------------------------------------------------------------------------------
struct AO {
    double A1, A2;          // sum_k c_k a1_k, sum_k c_k a2_k
    double c3a3, c3a4;      // c3 * a3, c3 * a4 of the quartic
    // the time limiter's ratios tau_Z/(beta_min+eps), tau_Z/(beta_max+eps), both multiplied by rs
    // (1 whenever the reconstruction was taped; the product of the four beta_k+eps otherwise)
    double rmax, rmin, rs;
};

// Optional record of a reconstruction's intermediates for its reverse (a "tape"): a sink with
// put(index, value).  NoTape discards everything, so the plain forward compiles to the arithmetic
// alone; ArrayTape writes a local array, PlaneTape one element of SoA planes in global memory.
struct NoTape {
    static constexpr bool active = false;
    DFK_HD void put(int, double) const {}
};
struct ArrayTape {
    static constexpr bool active = true;
    double* t;
    DFK_HD void put(int i, double v) const { t[i] = v; }
    DFK_HD double get(int i) const { return t[i]; }
};
struct PlaneTape {
    static constexpr bool active = true;
    double* p;
    long long s;
    DFK_HD void put(int i, double v) const { p[(long long)i * s] = v; }
    DFK_HD double get(int i) const { return p[(long long)i * s]; }
};

// WENO-AO tape of one reconstruction: sub-stencil coefficients a1[4], a2[4], the quartic's a3, a4,
// 1/(beta_k+eps), the ratios r_k, unnormalised weights w_k, 1/sum w, c_3, sign(beta_3 - beta_k)
// and the indices of max / min r (first attaining)
enum AOTapeField { AT_A1 = 0, AT_A2 = 4, AT_A3 = 8, AT_A4 = 9, AT_IE = 10, AT_R = 14, AT_W = 18, AT_IW = 22,
                   AT_C3 = 23, AT_SG = 24, AT_KMAX = 27, AT_KMIN = 28, AT_COUNT = 29 };

template <class Tape>
DFK_HD AO weno_ao_t(const double q[5], const SchemeConsts& S, const Tape& tp, int base) {
    const double qm2 = q[0], qm1 = q[1], q0 = q[2], q1 = q[3], q2 = q[4];
    // quadratic sub-stencils {i-2,i-1,i}, {i-1,i,i+1}, {i,i+1,i+2}
    double a1_0 = 0.5 * qm2 - 2.0 * qm1 + 1.5 * q0;
    double a2_0 = 0.5 * (qm2 - 2.0 * qm1 + q0);
    double a1_1 = 0.5 * (q1 - qm1);
    double a2_1 = 0.5 * (qm1 - 2.0 * q0 + q1);
    double a1_2 = -1.5 * q0 + 2.0 * q1 - 0.5 * q2;
    double a2_2 = 0.5 * (q0 - 2.0 * q1 + q2);
    // quartic on the full stencil
    double a1_3 = (5.0 * (qm2 - q2) - 34.0 * (qm1 - q1)) * (1.0 / 48.0);
    double a2_3 = (-(qm2 + q2) + 12.0 * (qm1 + q1) - 22.0 * q0) * (1.0 / 16.0);
    double a3_3 = (-(qm2 - q2) + 2.0 * (qm1 - q1)) * (1.0 / 12.0);
    double a4_3 = ((qm2 + q2) - 4.0 * (qm1 + q1) + 6.0 * q0) * (1.0 / 24.0);
    // smoothness indicators, Eq. 38 with dx^{2q-1} absorbed into the cell-centred coordinate
    const double c13_3 = 13.0 / 3.0;
    double b0 = a1_0 * a1_0 + c13_3 * a2_0 * a2_0;
    double b1 = a1_1 * a1_1 + c13_3 * a2_1 * a2_1;
    double b2 = a1_2 * a1_2 + c13_3 * a2_2 * a2_2;
    double b3 = a1_3 * (a1_3 + 0.5 * a3_3) + c13_3 * a2_3 * a2_3 + (21.0 / 5.0) * a2_3 * a4_3
              + (3129.0 / 80.0) * a3_3 * a3_3 + (87617.0 / 140.0) * a4_3 * a4_3;
    // Eq. 37 and the WENO-Z weights.  With P_k = prod_j (beta_j+eps) / (beta_k+eps) the ratios are
    // r_k = tau P_k / prod; scaled by prod^2 the weights d_k (prod^2 + (tau P_k)^2) need one division
    // (their normalisation) instead of two, and the limiter's ratios none (carried scaled by prod).
    double tau = (fabs(b3 - b0) + fabs(b3 - b1) + fabs(b3 - b2)) * (1.0 / 3.0);
    double e0 = b0 + S.eps, e1 = b1 + S.eps, e2 = b2 + S.eps, e3 = b3 + S.eps;
    double p01 = e0 * e1, p23 = e2 * e3, prod = p01 * p23;
    const double P0 = e1 * p23, P1 = e0 * p23, P2 = p01 * e3, P3 = p01 * e2;
    const double t0 = tau * P0, t1 = tau * P1, t2 = tau * P2, t3 = tau * P3;     // prod * r_k
    const double tmax = nn_max(nn_max(t0, t1), nn_max(t2, t3)), tmin = nn_min(nn_min(t0, t1), nn_min(t2, t3));
    AO o;
    double c0, c1, c2, c3;
    double r0, r1, r2, r3;                           // the ratios themselves: tape and fallback only
    if (nn_less(prod, 1e150) && nn_less(tmax, 1e150)) {   // beta+eps >= eps, so prod >= eps^4 > 0
        const double p2 = prod * prod;
        const double v0 = S.d[0] * (p2 + t0 * t0), v1 = S.d[1] * (p2 + t1 * t1);
        const double v2 = S.d[2] * (p2 + t2 * t2), v3 = S.d[3] * (p2 + t3 * t3);
        const double iv = 1.0 / (v0 + v1 + v2 + v3);
        c3 = v3 * iv * S.inv_d3;
        c0 = v0 * iv - c3 * S.d[0]; c1 = v1 * iv - c3 * S.d[1]; c2 = v2 * iv - c3 * S.d[2];
        o.rmax = tmax; o.rmin = tmin; o.rs = prod;
        if constexpr (Tape::active) {                // unscaled quantities for the reverse
            const double ip = 1.0 / prod;
            r0 = t0 * ip; r1 = t1 * ip; r2 = t2 * ip; r3 = t3 * ip;
            tp.put(base + AT_IE, P0 * ip); tp.put(base + AT_IE + 1, P1 * ip);
            tp.put(base + AT_IE + 2, P2 * ip); tp.put(base + AT_IE + 3, P3 * ip);
            o.rmax = tmax * ip; o.rmin = tmin * ip; o.rs = 1.0;
        }
    } else {
        r0 = tau / e0; r1 = tau / e1; r2 = tau / e2; r3 = tau / e3;
        tp.put(base + AT_IE, 1.0 / e0); tp.put(base + AT_IE + 1, 1.0 / e1);
        tp.put(base + AT_IE + 2, 1.0 / e2); tp.put(base + AT_IE + 3, 1.0 / e3);
        const double w0 = S.d[0] * (1.0 + r0 * r0), w1 = S.d[1] * (1.0 + r1 * r1);
        const double w2 = S.d[2] * (1.0 + r2 * r2), w3 = S.d[3] * (1.0 + r3 * r3);
        const double iw = 1.0 / (w0 + w1 + w2 + w3);
        c3 = w3 * iw * S.inv_d3;
        c0 = w0 * iw - c3 * S.d[0]; c1 = w1 * iw - c3 * S.d[1]; c2 = w2 * iw - c3 * S.d[2];
        // tau >= 0, so the ratio is largest at beta_min and smallest at beta_max
        o.rmax = nn_max(nn_max(r0, r1), nn_max(r2, r3)); o.rmin = nn_min(nn_min(r0, r1), nn_min(r2, r3)); o.rs = 1.0;
    }
    if constexpr (Tape::active) {
        // the reverse differentiates w_k = d_k (1 + r_k^2) and c_k = w_k / sum w - c_3 d_k
        const double w0 = S.d[0] * (1.0 + r0 * r0), w1 = S.d[1] * (1.0 + r1 * r1);
        const double w2 = S.d[2] * (1.0 + r2 * r2), w3 = S.d[3] * (1.0 + r3 * r3);
        const double iw = 1.0 / (w0 + w1 + w2 + w3);
        c3 = w3 * iw * S.inv_d3;
        c0 = w0 * iw - c3 * S.d[0]; c1 = w1 * iw - c3 * S.d[1]; c2 = w2 * iw - c3 * S.d[2];
        tp.put(base + AT_R, r0); tp.put(base + AT_R + 1, r1); tp.put(base + AT_R + 2, r2); tp.put(base + AT_R + 3, r3);
        tp.put(base + AT_W, w0); tp.put(base + AT_W + 1, w1); tp.put(base + AT_W + 2, w2); tp.put(base + AT_W + 3, w3);
        tp.put(base + AT_IW, iw); tp.put(base + AT_C3, c3);
        int kmax = 0, kmin = 0;
        const double rr[4] = {r0, r1, r2, r3};
#pragma unroll
        for (int k = 1; k < 4; ++k) { if (nn_less(rr[kmax], rr[k])) kmax = k; if (nn_less(rr[k], rr[kmin])) kmin = k; }
        tp.put(base + AT_KMAX, (double)kmax);
        tp.put(base + AT_KMIN, (double)kmin);
    }
    o.A1 = c0 * a1_0 + c1 * a1_1 + c2 * a1_2 + c3 * a1_3;
    o.A2 = c0 * a2_0 + c1 * a2_1 + c2 * a2_2 + c3 * a2_3;
    o.c3a3 = c3 * a3_3;
    o.c3a4 = c3 * a4_3;
    tp.put(base + AT_A1, a1_0); tp.put(base + AT_A1 + 1, a1_1); tp.put(base + AT_A1 + 2, a1_2); tp.put(base + AT_A1 + 3, a1_3);
    tp.put(base + AT_A2, a2_0); tp.put(base + AT_A2 + 1, a2_1); tp.put(base + AT_A2 + 2, a2_2); tp.put(base + AT_A2 + 3, a2_3);
    tp.put(base + AT_A3, a3_3); tp.put(base + AT_A4, a4_3);
    tp.put(base + AT_SG, (b3 - b0) >= 0.0 ? 1.0 : -1.0);
    tp.put(base + AT_SG + 1, (b3 - b1) >= 0.0 ? 1.0 : -1.0);
    tp.put(base + AT_SG + 2, (b3 - b2) >= 0.0 ? 1.0 : -1.0);
    return o;
}

DFK_HD AO weno_ao(const double q[5], const SchemeConsts& S) { return weno_ao_t(q, S, NoTape{}, 0); }

// The forward sweeps' WENO-AO without a tape, split in two so that two reconstructions can share
// one division: ao_core does everything up to the weights' normaliser, ao_finish applies its
// reciprocal.  Same formulas as weno_ao_t; the second differences are carried multiplied by
// sqrt(13/3) (the smoothness indicators then need one multiply less each), and the AO coefficient
// A2 is scaled back at the end.
constexpr double kS13 = 2.0816659994661326;            // sqrt(13/3)
constexpr double kIS13 = 0.48038446141526137;          // sqrt(3/13)

struct AOCore {
    double a1[4], a2s[4];   // first-derivative coefficients; second ones times sqrt(13/3)
    double a3, a4;          // quartic's cubic and quartic coefficients
    double v[4];            // unnormalised weights (scaled by prod^2 when `scaled`)
    double sum;             // their sum
    double rmax, rmin, rs;  // limiter ratios as in AO
};

// second differences of the three quadratic sub-stencils are shared between the left and right
// reconstructions of a face line; the caller passes them (times sqrt(13/3)/2) in
DFK_HD AOCore ao_core(const double q[5], const double a2s_q[3], const SchemeConsts& S) {
    const double qm2 = q[0], qm1 = q[1], q0 = q[2], q1 = q[3], q2 = q[4];
    AOCore c;
    c.a1[0] = 0.5 * qm2 - 2.0 * qm1 + 1.5 * q0;
    c.a1[1] = 0.5 * (q1 - qm1);
    c.a1[2] = -1.5 * q0 + 2.0 * q1 - 0.5 * q2;
    c.a1[3] = (5.0 * (qm2 - q2) - 34.0 * (qm1 - q1)) * (1.0 / 48.0);
    c.a2s[0] = a2s_q[0]; c.a2s[1] = a2s_q[1]; c.a2s[2] = a2s_q[2];
    c.a2s[3] = (-(qm2 + q2) + 12.0 * (qm1 + q1) - 22.0 * q0) * (kS13 / 16.0);
    c.a3 = (-(qm2 - q2) + 2.0 * (qm1 - q1)) * (1.0 / 12.0);
    c.a4 = ((qm2 + q2) - 4.0 * (qm1 + q1) + 6.0 * q0) * (1.0 / 24.0);
    // Eq. 38 (cell-centred): beta_k = a1^2 + 13/3 a2^2 (+ the quartic's cross and higher terms)
    const double b0 = c.a1[0] * c.a1[0] + c.a2s[0] * c.a2s[0];
    const double b1 = c.a1[1] * c.a1[1] + c.a2s[1] * c.a2s[1];
    const double b2 = c.a1[2] * c.a1[2] + c.a2s[2] * c.a2s[2];
    const double b3 = c.a1[3] * (c.a1[3] + 0.5 * c.a3) + c.a2s[3] * (c.a2s[3] + (21.0 / 5.0) * kIS13 * c.a4)
                    + (3129.0 / 80.0) * c.a3 * c.a3 + (87617.0 / 140.0) * c.a4 * c.a4;
    // Eq. 37 and the WENO-Z weights d_k (1 + r_k^2), r_k = tau / (beta_k + eps), scaled by prod^2
    const double tau = (fabs(b3 - b0) + fabs(b3 - b1) + fabs(b3 - b2)) * (1.0 / 3.0);
    const double e0 = b0 + S.eps, e1 = b1 + S.eps, e2 = b2 + S.eps, e3 = b3 + S.eps;
    const double p01 = e0 * e1, p23 = e2 * e3, prod = p01 * p23;
    const double t0 = tau * (e1 * p23), t1 = tau * (e0 * p23), t2 = tau * (p01 * e3), t3 = tau * (p01 * e2);
    const double tmax = nn_max(nn_max(t0, t1), nn_max(t2, t3)), tmin = nn_min(nn_min(t0, t1), nn_min(t2, t3));
    if (nn_less(prod, 1e150) && nn_less(tmax, 1e150)) {
        const double p2 = prod * prod;
        c.v[0] = S.d[0] * (p2 + t0 * t0); c.v[1] = S.d[1] * (p2 + t1 * t1);
        c.v[2] = S.d[2] * (p2 + t2 * t2); c.v[3] = S.d[3] * (p2 + t3 * t3);
        c.rmax = tmax; c.rmin = tmin; c.rs = prod;
    } else {
        const double r0 = tau / e0, r1 = tau / e1, r2 = tau / e2, r3 = tau / e3;
        c.v[0] = S.d[0] * (1.0 + r0 * r0); c.v[1] = S.d[1] * (1.0 + r1 * r1);
        c.v[2] = S.d[2] * (1.0 + r2 * r2); c.v[3] = S.d[3] * (1.0 + r3 * r3);
        c.rmax = nn_max(nn_max(r0, r1), nn_max(r2, r3)); c.rmin = nn_min(nn_min(r0, r1), nn_min(r2, r3)); c.rs = 1.0;
    }
    c.sum = (c.v[0] + c.v[1]) + (c.v[2] + c.v[3]);
    return c;
}

// second differences of q (times sqrt(13/3)/2) for the three quadratic sub-stencils
DFK_HD void ao_second_differences(const double q[5], double a2s[3]) {
    a2s[0] = (0.5 * kS13) * (q[0] - 2.0 * q[1] + q[2]);
    a2s[1] = (0.5 * kS13) * (q[1] - 2.0 * q[2] + q[3]);
    a2s[2] = (0.5 * kS13) * (q[2] - 2.0 * q[3] + q[4]);
}

// the AO polynomial's coefficients from a core and iv = 1 / c.sum
DFK_HD AO ao_finish(const AOCore& c, double iv, const SchemeConsts& S) {
    AO o;
    const double c3 = c.v[3] * iv * S.inv_d3;
    const double c0 = c.v[0] * iv - c3 * S.d[0], c1 = c.v[1] * iv - c3 * S.d[1], c2 = c.v[2] * iv - c3 * S.d[2];
    o.A1 = c0 * c.a1[0] + c1 * c.a1[1] + c2 * c.a1[2] + c3 * c.a1[3];
    o.A2 = (c0 * c.a2s[0] + c1 * c.a2s[1] + c2 * c.a2s[2] + c3 * c.a2s[3]) * kIS13;
    o.c3a3 = c3 * c.a3;
    o.c3a4 = c3 * c.a4;
    o.rmax = c.rmax; o.rmin = c.rmin; o.rs = c.rs;
    return o;
}

// two reconstructions finished with one division: 1/(sa sb) times sb and sa (both sums lie in
// [1e-50, 1e150] on the scaled branch, so the product neither overflows nor underflows)
DFK_HD void ao_finish_pair(const AOCore& a, const AOCore& b, const SchemeConsts& S, AO& oa, AO& ob) {
    double ia, ib;
    if (nn_less(a.sum, 1e150) && nn_less(b.sum, 1e150)) {
        const double r = 1.0 / (a.sum * b.sum);
        ia = b.sum * r;
        ib = a.sum * r;
    } else {
        ia = 1.0 / a.sum;
        ib = 1.0 / b.sum;
    }
    oa = ao_finish(a, ia, S);
    ob = ao_finish(b, ib, S);
}

// time-limiter ingredient 2 at2 / (at1 + at2) of one reconstruction (Sect. 2.2), as numerator and
// (positive) denominator, so that a minimum over several needs one division at the end
DFK_HD void limiter_fraction(const AO& o, double& num, double& den) {
    // 1 + r^2 scaled by rs^2, which cancels in the ratio
    const double s2 = o.rs * o.rs;
    double a1 = s2 + o.rmax * o.rmax, a2 = s2 + o.rmin * o.rmin;
    num = 2.0 * a2;
    den = a1 + a2;
}

DFK_HD double limiter_alpha(const AO& o) {
    double n, d;
    limiter_fraction(o, n, d);
    return n / d;
}

// value and d/dxi of the AO polynomial at the right cell edge xi = +1/2
DFK_HD void ao_at_right_edge(const AO& o, double q0, double& val, double& slope) {
    val = q0 + 0.5 * o.A1 + (1.0 / 6.0) * o.A2 + 0.125 * o.c3a3 + 0.05 * o.c3a4;
    slope = o.A1 + o.A2 + 0.75 * o.c3a3 + 0.5 * o.c3a4;
}

// zero-mean DF quadratic of Sect. 3.3, p_DF = Q_0 + alpha (p1 - Q_0), at xi = +1/2
DFK_HD void df_at_right_edge(const double q[5], double alpha, double& val, double& slope) {
    double a1 = 0.5 * (q[3] - q[1]);
    double a2 = 0.5 * (q[1] - 2.0 * q[2] + q[3]);
    val = q[2] + alpha * (0.5 * a1 + (1.0 / 6.0) * a2);
    slope = alpha * (a1 + a2);
}

// values and d/deta at the two Gauss points eta = -g (m=1), +g (m=2), g = sqrt(3)/6
DFK_HD void ao_at_gauss(const AO& o, double q0, double val[2], double slope[2]) {
    const double g = kGaussEta;
    double E = q0 - (1.0 / 180.0) * o.c3a4;                 // even part: xi^2 = 1/12, xi^4 = 1/144
    double O = g * (o.A1 + (1.0 / 12.0) * o.c3a3);          // odd part
    double Es = o.A1 + 0.25 * o.c3a3;
    double Os = g * (2.0 * o.A2 + (1.0 / 3.0) * o.c3a4);
    val[0] = E - O; val[1] = E + O;
    slope[0] = Es - Os; slope[1] = Es + Os;
}

DFK_HD void df_at_gauss(const double q[5], double alpha, double val[2], double slope[2]) {
    const double g = kGaussEta;
    double a1 = 0.5 * (q[3] - q[1]);
    double a2 = 0.5 * (q[1] - 2.0 * q[2] + q[3]);
    double O = alpha * g * a1;                               // xi^2 - 1/12 vanishes at the Gauss points
    double Es = alpha * a1, Os = alpha * 2.0 * g * a2;
    val[0] = q[2] - O; val[1] = q[2] + O;
    slope[0] = Es - Os; slope[1] = Es + Os;
}

// ------------------------------------------------------------------------------------------
// Gas-kinetic flux at one Gauss point in the local frame (Sect. 2.2, 3.4; Eqs. 25-27).
// Maxwellian moments are normalised by rho.  <u^k v^l xi^{2c}> = mu[k] mv[l] mx[c].
// ------------------------------------------------------------------------------------------
struct Mom {
    double mu[7];   // <u^n>, full or half-space
    double mv[6];   // <v^n>, full
    double mx[3];   // <1>, <xi^2>, <xi^4>
};

// One Maxwellian: il2 = 1/(2 lambda) = p/rho, tl = 2 lambda, f4 = 4 lambda^2/(K+2),
// qK = U^2 + V^2 + (K+2)/(2 lambda); the slope solves of a state share them.
struct Maxw { double rho, ir, U, V, p, il2, tl, f4, qK, isl; };   // isl = 1/sqrt(lambda)

// velocities and pressure of W given ir = 1/rho
DFK_HD void maxw_velocities(const double W[4], double ir, const SchemeConsts& S, Maxw& s) {
    s.rho = W[0];
    s.ir = ir;
    s.U = W[1] * ir;
    s.V = W[2] * ir;
    s.p = S.gm1 * (W[3] - 0.5 * W[0] * (s.U * s.U + s.V * s.V));
}

// the rest given tl = 2 lambda = rho / p
DFK_HD void maxw_finish(double tl, const SchemeConsts& S, Maxw& s) {
    s.tl = tl;
    s.il2 = s.p * s.ir;
    s.f4 = tl * tl * S.inv_K2;
    s.qK = s.U * s.U + s.V * s.V + (S.K + 2.0) * s.il2;
    s.isl = rsqrt(0.5 * tl);           // the half-space moments and the DF factor's 1/c need it
}

DFK_HD Maxw maxw_of(const double W[4], const SchemeConsts& S) {
    Maxw s;
    maxw_velocities(W, 1.0 / W[0], S, s);
    maxw_finish(W[0] / s.p, S, s);
    return s;
}

// the two sides' Maxwellians with two divisions instead of four: 1/(rho_l rho_r) gives both 1/rho
// and 1/(p_l p_r) both rho/p.  A product outside [1e-150, 1e150] (non-physical or extreme states)
// is divided side by side as in maxw_of.
DFK_HD void maxw_pair(const double WL[4], const double WR[4], const SchemeConsts& S, Maxw& a, Maxw& b) {
    const double rr = WL[0] * WR[0];
    if (in_range(rr, 1e-150, 1e150)) {
        const double r = 1.0 / rr;
        maxw_velocities(WL, WR[0] * r, S, a);
        maxw_velocities(WR, WL[0] * r, S, b);
    } else {
        maxw_velocities(WL, 1.0 / WL[0], S, a);
        maxw_velocities(WR, 1.0 / WR[0], S, b);
    }
    const double pp = a.p * b.p;
    if (in_range(pp, 1e-150, 1e150)) {
        const double r = 1.0 / pp;
        maxw_finish(WL[0] * b.p * r, S, a);
        maxw_finish(WR[0] * a.p * r, S, b);
    } else {
        maxw_finish(WL[0] / a.p, S, a);
        maxw_finish(WR[0] / b.p, S, b);
    }
}

// half: 0 full, +1 u>0, -1 u<0
template <int HALF>
DFK_HD void fill_moments(const Maxw& s, double K, Mom& m) {
    if (HALF == 0) {
        m.mu[0] = 1.0;
        m.mu[1] = s.U;
    } else {
        double lam = 0.5 * s.tl;
        double isl = s.isl;                                   // 1/sqrt(lambda)
        double x = lam * isl * s.U;                           // sqrt(lambda) U
        double G = exp(-x * x);
        double e = G * (0.28209479177387814347 * isl);        // exp(-lambda U^2) / (2 sqrt(pi lambda))
        // erfc(|x|) / 2 from the scaled function erfcx(|x|) = exp(x^2) erfc(|x|) and the Gaussian
        // above (one exponential for both); erfc(-|x|) = 2 - erfc(|x|)
#ifdef __CUDA_ARCH__
        double h = 0.5 * G * erfcx(fabs(x));
#else
        double h = 0.5 * erfc(fabs(x));
#endif
        const bool xpos = dbits(x) >= 0;                      // x >= +0 (at -0 both forms give 1/2)
        if (HALF > 0) { m.mu[0] = xpos ? 1.0 - h : h; m.mu[1] = s.U * m.mu[0] + e; }   // erfc(-x) / 2
        else          { m.mu[0] = xpos ? h : 1.0 - h; m.mu[1] = s.U * m.mu[0] - e; }   // erfc(x) / 2
    }
#pragma unroll
    for (int n = 2; n < 7; ++n) m.mu[n] = s.U * m.mu[n - 1] + (double)(n - 1) * s.il2 * m.mu[n - 2];
    m.mv[0] = 1.0;
    m.mv[1] = s.V;
#pragma unroll
    for (int n = 2; n < 6; ++n) m.mv[n] = s.V * m.mv[n - 1] + (double)(n - 1) * s.il2 * m.mv[n - 2];
    m.mx[0] = 1.0;
    m.mx[1] = K * s.il2;
    m.mx[2] = K * (K + 2.0) * s.il2 * s.il2;
}

template <int k, int l, int c>
DFK_HD double M(const Mom& m) { return m.mu[k] * m.mv[l] * m.mx[c]; }

// <u^k v^l xi^{2c} psi>, psi = (1, u, v, (u^2+v^2+xi^2)/2)
template <int k, int l, int c>
DFK_HD void psi_mom(const Mom& m, double out[4]) {
    out[0] = M<k, l, c>(m);
    out[1] = M<k + 1, l, c>(m);
    out[2] = M<k, l + 1, c>(m);
    out[3] = 0.5 * (M<k + 2, l, c>(m) + M<k, l + 2, c>(m) + M<k, l, c + 1>(m));
}

// <u^k v^l a psi> with a = a0 + a1 u + a2 v + a3 (u^2+v^2+xi^2)/2.  With h = a3/2 and the
// factorised moments <u^k v^l xi^2c> = mu_k mv_l mx_c (mx_0 = 1):
//   G(k,l,c) = <u^k v^l xi^2c a> = mx_c (mv_l P_k + mu_k Q_l) + h mu_k mv_l mx_{c+1},
//   P_k = a0 mu_k + a1 mu_{k+1} + h mu_{k+2},   Q_l = a2 mv_{l+1} + h mv_{l+2},
// and out = (G(k,l,0), G(k+1,l,0), G(k,l+1,0), [G(k+2,l,0) + G(k,l+2,0) + G(k,l,1)] / 2).
// Qp_j = Q_{l+j} + h mx_1 mv_{l+j} folds the xi^2 term into the c = 0 forms.
template <int k, int l>
DFK_HD void a_mom(const Mom& m, const double a[4], double out[4]) {
    const double h = 0.5 * a[3], hx1 = h * m.mx[1];
    double P[3], Qp[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        P[j] = a[0] * m.mu[k + j] + a[1] * m.mu[k + j + 1] + h * m.mu[k + j + 2];
        Qp[j] = a[2] * m.mv[l + j + 1] + h * m.mv[l + j + 2] + hx1 * m.mv[l + j];
    }
    const double Ql = a[2] * m.mv[l + 1] + h * m.mv[l + 2];
    const double G1 = m.mx[1] * (m.mv[l] * P[0] + m.mu[k] * Ql) + h * m.mu[k] * m.mv[l] * m.mx[2];
    out[0] = m.mv[l] * P[0] + m.mu[k] * Qp[0];
    out[1] = m.mv[l] * P[1] + m.mu[k + 1] * Qp[0];
    out[2] = m.mv[l + 1] * P[0] + m.mu[k] * Qp[1];
    out[3] = 0.5 * ((m.mv[l] * P[2] + m.mu[k + 2] * Qp[0]) + (m.mv[l + 2] * P[0] + m.mu[k] * Qp[2]) + G1);
}

// closed-form solution of <a psi> = b for a Maxwellian (U, V, lambda)
DFK_HD void slope_solve(const Maxw& s, const double b[4], double a[4]) {
    double R2 = b[1] - s.U * b[0], R3 = b[2] - s.V * b[0], R4 = 2.0 * b[3] - s.qK * b[0];
    a[3] = s.f4 * (R4 - 2.0 * s.U * R2 - 2.0 * s.V * R3);
    a[2] = s.tl * R3 - s.V * a[3];
    a[1] = s.tl * R2 - s.U * a[3];
    a[0] = b[0] - s.U * a[1] - s.V * a[2] - 0.5 * a[3] * s.qK;
}

struct GPState { double W[4], Wn[4], Wt[4]; };   // one side of one Gauss point, local frame

// Forward intermediates of gks_flux that its reverse reads (the tau = 0 reading's part), as a
// tape of doubles: the three Maxwellians (rho, 1/rho, U, V, p, 1/(2 lambda), 2 lambda, f4, qK),
// their moments (mu[7], mv[6], mx[3]), the slope coefficients, the compatibility right-hand side,
// the equilibrium state and slopes, the kinetic-weighting moments, the flux moments and the
// pressure ratio of tau_n.  A reverse sweep can read them back instead of recomputing the flux.
enum GksTapeField {
    TG_SL = 0, TG_SR = 9, TG_SC = 18, TG_ML = 27, TG_MR = 43, TG_MC = 59,
    TG_ALX = 75, TG_ALY = 79, TG_ARX = 83, TG_ARY = 87, TG_ACX = 91, TG_ACY = 95, TG_AC = 99, TG_BCT = 103,
    TG_WC = 107, TG_WCX = 111, TG_WCY = 115,
    TG_PL0 = 119, TG_PR0 = 123, TG_LX0 = 127, TG_RX0 = 131, TG_LY0 = 135, TG_RY0 = 139,
    TG_MC0 = 143, TG_MC1 = 147, TG_MC2 = 151, TG_ML0 = 155, TG_MR0 = 159, TG_ML1 = 163, TG_MR1 = 167,
    TG_Q = 171, TG_COUNT = 172
};


template <class Tape>
DFK_HD void tape_maxw(const Tape& tp, int b, const Maxw& s) {
    tp.put(b, s.rho); tp.put(b + 1, s.ir); tp.put(b + 2, s.U); tp.put(b + 3, s.V); tp.put(b + 4, s.p);
    tp.put(b + 5, s.il2); tp.put(b + 6, s.tl); tp.put(b + 7, s.f4); tp.put(b + 8, s.qK);
}
template <class Tape>
DFK_HD void tape_mom(const Tape& tp, int b, const Mom& m) {
#pragma unroll
    for (int n = 0; n < 7; ++n) tp.put(b + n, m.mu[n]);
#pragma unroll
    for (int n = 0; n < 6; ++n) tp.put(b + 7 + n, m.mv[n]);
#pragma unroll
    for (int n = 0; n < 3; ++n) tp.put(b + 13 + n, m.mx[n]);
}
template <class Tape>
DFK_HD void tape_vec(const Tape& tp, int b, const double v[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) tp.put(b + i, v[i]);
}

// sl, sr: the Maxwellians of L.W and R.W (maxw_pair)
template <class Tape>
DFK_HD void gks_flux_t(const GPState& L, const GPState& R, const Maxw& sl, const Maxw& sr, double dt,
                       const SchemeConsts& S, double F[4], double dF[4], const Tape& tp) {
    const double K = S.K;
    Mom ml, mr;
    fill_moments<+1>(sl, K, ml);
    fill_moments<-1>(sr, K, mr);
    double b[4], alx[4], aly[4], arx[4], ary[4];
    const double irl = sl.ir, irr = sr.ir;
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = L.Wn[i] * irl;
    slope_solve(sl, b, alx);
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = L.Wt[i] * irl;
    slope_solve(sl, b, aly);
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = R.Wn[i] * irr;
    slope_solve(sr, b, arx);
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = R.Wt[i] * irr;
    slope_solve(sr, b, ary);
    tape_maxw(tp, TG_SL, sl); tape_maxw(tp, TG_SR, sr);
    tape_mom(tp, TG_ML, ml); tape_mom(tp, TG_MR, mr);
    tape_vec(tp, TG_ALX, alx); tape_vec(tp, TG_ALY, aly); tape_vec(tp, TG_ARX, arx); tape_vec(tp, TG_ARY, ary);
    // Sect. 3.4: equilibrium state and slopes by kinetic weighting
    double Wc[4], Wcx[4], Wcy[4], t1[4], t2[4];
    psi_mom<0, 0, 0>(ml, t1); psi_mom<0, 0, 0>(mr, t2);
    tape_vec(tp, TG_PL0, t1); tape_vec(tp, TG_PR0, t2);
#pragma unroll
    for (int i = 0; i < 4; ++i) Wc[i] = sl.rho * t1[i] + sr.rho * t2[i];
    a_mom<0, 0>(ml, alx, t1); a_mom<0, 0>(mr, arx, t2);
    tape_vec(tp, TG_LX0, t1); tape_vec(tp, TG_RX0, t2);
#pragma unroll
    for (int i = 0; i < 4; ++i) Wcx[i] = sl.rho * t1[i] + sr.rho * t2[i];
    a_mom<0, 0>(ml, aly, t1); a_mom<0, 0>(mr, ary, t2);
    tape_vec(tp, TG_LY0, t1); tape_vec(tp, TG_RY0, t2);
#pragma unroll
    for (int i = 0; i < 4; ++i) Wcy[i] = sl.rho * t1[i] + sr.rho * t2[i];
    tape_vec(tp, TG_WC, Wc); tape_vec(tp, TG_WCX, Wcx); tape_vec(tp, TG_WCY, Wcy);
    // the equilibrium state's Maxwellian: 1/rho_c shares a division with 1/dt, and rho_c / p_c one
    // with 1/(p_l + p_r) of the pressure ratio in tau_n (products outside [1e-150, 1e150] are
    // divided separately)
    Maxw sc;
    double idt, ips;
    {
        const double a = Wc[0] * dt;
        if (in_range(a, 1e-150, 1e150)) {
            const double r = 1.0 / a;
            maxw_velocities(Wc, dt * r, S, sc);
            idt = Wc[0] * r;
        } else {
            maxw_velocities(Wc, 1.0 / Wc[0], S, sc);
            idt = 1.0 / dt;
        }
        const double ps = sl.p + sr.p, b = sc.p * ps;
        if (in_range(b, 1e-150, 1e150)) {
            const double r = 1.0 / b;
            maxw_finish(Wc[0] * ps * r, S, sc);
            ips = sc.p * r;
        } else {
            maxw_finish(Wc[0] / sc.p, S, sc);
            ips = 1.0 / ps;
        }
    }
    Mom mc;
    fill_moments<0>(sc, K, mc);
    tape_maxw(tp, TG_SC, sc); tape_mom(tp, TG_MC, mc);
    double acx[4], acy[4], Ac[4];
    const double irc = sc.ir;
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = Wcx[i] * irc;
    slope_solve(sc, b, acx);
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = Wcy[i] * irc;
    slope_solve(sc, b, acy);
    // compatibility <A + a_x u + a_y v> = 0
    a_mom<1, 0>(mc, acx, t1); a_mom<0, 1>(mc, acy, t2);
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = -(t1[i] + t2[i]);
    slope_solve(sc, b, Ac);
    tape_vec(tp, TG_ACX, acx); tape_vec(tp, TG_ACY, acy); tape_vec(tp, TG_AC, Ac); tape_vec(tp, TG_BCT, b);
    // moments entering the flux
    double Mc0[4], Mc1[4], Mc2[4], Ml0[4], Mr0[4], Ml1[4], Mr1[4];
    psi_mom<1, 0, 0>(mc, Mc0);
    a_mom<2, 0>(mc, acx, t1); a_mom<1, 1>(mc, acy, t2);
#pragma unroll
    for (int i = 0; i < 4; ++i) Mc1[i] = t1[i] + t2[i];
    a_mom<1, 0>(mc, Ac, Mc2);
    psi_mom<1, 0, 0>(ml, Ml0);
    psi_mom<1, 0, 0>(mr, Mr0);
    a_mom<2, 0>(ml, alx, t1); a_mom<1, 1>(ml, aly, t2);
#pragma unroll
    for (int i = 0; i < 4; ++i) Ml1[i] = t1[i] + t2[i];
    a_mom<2, 0>(mr, arx, t1); a_mom<1, 1>(mr, ary, t2);
#pragma unroll
    for (int i = 0; i < 4; ++i) Mr1[i] = t1[i] + t2[i];
    tape_vec(tp, TG_MC0, Mc0); tape_vec(tp, TG_MC1, Mc1); tape_vec(tp, TG_MC2, Mc2);
    tape_vec(tp, TG_ML0, Ml0); tape_vec(tp, TG_MR0, Mr0); tape_vec(tp, TG_ML1, Ml1); tape_vec(tp, TG_MR1, Mr1);
    // numerical collision time (Sect. 2.2) and the combined time coefficients of Eq. 27
    const double q = (sl.p - sr.p) * ips;
    tp.put(TG_Q, q);
    double rT = S.C1 + S.C2 * fabs(q);   // tau_n / dt
    double T = rT * dt;
    double tau = (S.tau_reading == 1) ? T : 0.0;
    double E2 = 0.0, r = 0.0;
    if (dbits(rT) > 0) { E2 = exp(-0.5 / rT); r = rT; }   // rT >= 0
    double E1 = E2 * E2;
    double om = 1.0 - E2;
    double S3 = om * (3.0 - E2);                       // 3 - 4 E2 + E1
    // F-coefficients (4 G(dt/2) - G(dt)) / dt and dF-coefficients 4 (G(dt) - 2 G(dt/2)) / dt^2
    double glrF = r * S3, glrD = -4.0 * r * om * om * idt;
    double gcF = 1.0 - glrF, gcD = -glrD;
    double TT = T * T + T * tau;
    double acF = TT * S3 * idt - 2.0 * T * E2 + T * E1 - tau;
    double acD = 4.0 * (-TT * om * om + T * dt * E2 * om) * idt * idt;
    double AcF = -tau + tau * r * S3;
    double AcD = 1.0 - 4.0 * T * tau * om * om * idt * idt;
    double alrF = -acF - tau, alrD = -acD;
    double AlrF = -T * tau * S3 * idt, AlrD = 4.0 * T * tau * om * om * idt * idt;
    double Ml2[4] = {0, 0, 0, 0}, Mr2[4] = {0, 0, 0, 0};
    if (S.tau_reading == 1) {
        Mom mlF, mrF;
        fill_moments<0>(sl, K, mlF);
        fill_moments<0>(sr, K, mrF);
        double Al[4], Ar[4];
        a_mom<1, 0>(mlF, alx, t1); a_mom<0, 1>(mlF, aly, t2);
#pragma unroll
        for (int i = 0; i < 4; ++i) b[i] = -(t1[i] + t2[i]);
        slope_solve(sl, b, Al);
        a_mom<1, 0>(mrF, arx, t1); a_mom<0, 1>(mrF, ary, t2);
#pragma unroll
        for (int i = 0; i < 4; ++i) b[i] = -(t1[i] + t2[i]);
        slope_solve(sr, b, Ar);
        a_mom<1, 0>(ml, Al, Ml2);
        a_mom<1, 0>(mr, Ar, Mr2);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        double c0 = sc.rho * Mc0[i], c1 = sc.rho * Mc1[i], c2 = sc.rho * Mc2[i];
        double g0 = sl.rho * Ml0[i] + sr.rho * Mr0[i];
        double g1 = sl.rho * Ml1[i] + sr.rho * Mr1[i];
        double g2 = sl.rho * Ml2[i] + sr.rho * Mr2[i];
        F[i] = gcF * c0 + acF * c1 + AcF * c2 + glrF * g0 + alrF * g1 + AlrF * g2;
        dF[i] = gcD * c0 + acD * c1 + AcD * c2 + glrD * g0 + alrD * g1 + AlrD * g2;
    }
}

template <class Tape>
DFK_HD void gks_flux_t(const GPState& L, const GPState& R, double dt, const SchemeConsts& S,
                       double F[4], double dF[4], const Tape& tp) {
    Maxw sl, sr;
    maxw_pair(L.W, R.W, S, sl, sr);
    gks_flux_t(L, R, sl, sr, dt, S, F, dF, tp);
}

DFK_HD void gks_flux(const GPState& L, const GPState& R, double dt, const SchemeConsts& S, double F[4], double dF[4]) {
    gks_flux_t(L, R, dt, S, F, dF, NoTape{});
}

// ------------------------------------------------------------------------------------------
// Lax-Friedrichs flux (Sect. 2.3) and its time derivative with frozen wave speed and
// W_t = -(A W_n + B W_t) on each side (Cauchy-Kovalevskaya)
// ------------------------------------------------------------------------------------------
struct EulerPt { double u, v, p, c, H, q; };

DFK_HD EulerPt euler_pt(const double W[4], const SchemeConsts& S) {
    EulerPt e;
    double ir = 1.0 / W[0];
    e.u = W[1] * ir;
    e.v = W[2] * ir;
    e.q = 0.5 * (e.u * e.u + e.v * e.v);
    e.p = S.gm1 * (W[3] - W[0] * e.q);
    e.c = sqrt(S.gamma * e.p * ir);
    e.H = (W[3] + e.p) * ir;
    return e;
}

// A X (x-flux Jacobian) and B X (y-flux Jacobian) at a state
DFK_HD void jac_x(const EulerPt& e, double gm1, const double X[4], double Y[4]) {
    double dp = gm1 * (X[3] - e.u * X[1] - e.v * X[2] + e.q * X[0]);
    Y[0] = X[1];
    Y[1] = 2.0 * e.u * X[1] - e.u * e.u * X[0] + dp;
    Y[2] = e.v * X[1] + e.u * X[2] - e.u * e.v * X[0];
    Y[3] = e.u * (X[3] + dp) + e.H * (X[1] - e.u * X[0]);
}
DFK_HD void jac_y(const EulerPt& e, double gm1, const double X[4], double Y[4]) {
    double dp = gm1 * (X[3] - e.u * X[1] - e.v * X[2] + e.q * X[0]);
    Y[0] = X[2];
    Y[1] = e.v * X[1] + e.u * X[2] - e.u * e.v * X[0];
    Y[2] = 2.0 * e.v * X[2] - e.v * e.v * X[0] + dp;
    Y[3] = e.v * (X[3] + dp) + e.H * (X[2] - e.v * X[0]);
}

DFK_HD void lf_flux(const GPState& L, const GPState& R, const SchemeConsts& S,
                                        double F[4], double dF[4]) {
    EulerPt el = euler_pt(L.W, S), er = euler_pt(R.W, S);
    double FL[4] = {L.W[1], L.W[1] * el.u + el.p, L.W[1] * el.v, el.u * (L.W[3] + el.p)};
    double FR[4] = {R.W[1], R.W[1] * er.u + er.p, R.W[1] * er.v, er.u * (R.W[3] + er.p)};
    double s = nn_max(fabs(el.u) + el.c, fabs(er.u) + er.c);
    double t1[4], t2[4], WtL[4], WtR[4], AL[4], AR[4];
    jac_x(el, S.gm1, L.Wn, t1); jac_y(el, S.gm1, L.Wt, t2);
#pragma unroll
    for (int i = 0; i < 4; ++i) WtL[i] = -(t1[i] + t2[i]);
    jac_x(er, S.gm1, R.Wn, t1); jac_y(er, S.gm1, R.Wt, t2);
#pragma unroll
    for (int i = 0; i < 4; ++i) WtR[i] = -(t1[i] + t2[i]);
    jac_x(el, S.gm1, WtL, AL);
    jac_x(er, S.gm1, WtR, AR);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        F[i] = 0.5 * (FL[i] + FR[i]) - 0.5 * s * (R.W[i] - L.W[i]);
        dF[i] = 0.5 * (AL[i] + AR[i]) - 0.5 * s * (WtR[i] - WtL[i]);
    }
}

// DF factor of one Gauss point (Sect. 3.2, Eq. 33) from the Maxwellians of its two local-frame
// states (maxw_pair, which the GKS flux shares): reciprocal square roots for the sound speeds, one
// division at the end
DFK_HD double df_alpha_maxw(const Maxw& l, const Maxw& r, const SchemeConsts& S) {
    // 1/c = sqrt(rho / (gamma p)) = sqrt(2/gamma) lambda / sqrt(lambda) on each side
    const double icl = S.r2g * (0.5 * l.tl) * l.isl, icr = S.r2g * (0.5 * r.tl) * r.isl;
    const double dn = l.U * icl - r.U * icr, dtg = l.V * icl - r.V * icr;
    // |p_l - p_r| (p_l + p_r) / (p_l p_r) = |p_l - p_r| (1/p_l + 1/p_r), 1/p = (rho/p) (1/rho)
    const double D = fabs(l.p - r.p) * (l.tl * l.ir + r.tl * r.ir) + dn * dn + dtg * dtg;
    return 1.0 / (1.0 + D * D);
}

DFK_HD double df_alpha(const double WL[4], const double WR[4], const SchemeConsts& S) {
    Maxw l, r;
    maxw_pair(WL, WR, S, l, r);
    return df_alpha_maxw(l, r, S);
}

// 0 < x <= +inf on the bit pattern (false for negatives, zeros and NaN)
DFK_HD bool positive_bits(double x) { const long long b = dbits(x); return b > 0 && b <= 0x7FF0000000000000LL; }

DFK_HD bool physical_state(const double W[4], double gm1) {
    if (!positive_bits(W[0])) return false;
    // p > 0 tested as rho p = (gamma - 1) (rho E - |rho u|^2 / 2) > 0: the same sign for rho > 0,
    // without a division
    double rp = gm1 * (W[0] * W[3] - 0.5 * (W[1] * W[1] + W[2] * W[2]));
    return positive_bits(rp);
}

}  // namespace dfk
