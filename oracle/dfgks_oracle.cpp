// ============================================================================================
// dfgks_oracle.cpp -- TEST INFRASTRUCTURE, not part of the product path.
//
// A plain, slow, CPU-only FP64 restatement of the hybrid DF + WENO-AO high-order finite-volume
// scheme of Zhang, Ji & Xu, "A robustness-enhanced reconstruction based on discontinuity
// feedback factor for high-order finite volume scheme" (arXiv 2402.10914):
//   Sect. 2.1  finite-volume form (Eq. 2), two-point Gauss quadrature, local frame T / T^-1
//   Sect. 2.2  BGK gas-kinetic flux, Maxwellian, slope/time coefficients, tau_n, Eqs. 25-27,
//              S2O4 (Eq. 24) and its non-linear time limiter
//   Sect. 2.3  Euler equations, Lax-Friedrichs flux, SSP-RK3
//   Sect. 3.1  WENO-AO(5,3): sub-stencil polynomials, linear weights, WENO-Z weights,
//              tau_Z (Eq. 37), smoothness indicators (Eq. 38)
//   Sect. 3.2  discontinuity feedback factor alpha_{p,m}, alpha_ij
//   Sect. 3.3  hybrid switch (Eq. 34) and the zero-mean DF quadratic; Remark 1; Algorithm 1
//   Sect. 3.4  equilibrium state by kinetic weighting
//
// Everything is done the obvious way, in the paper's order: sub-stencil polynomials come from
// solving the cell-average interpolation conditions, smoothness indicators from Gauss-Legendre
// quadrature of Eq. 38, the characteristic basis from inverting the right-eigenvector matrix,
// the GKS slope coefficients from solving the 4x4 moment system <a psi> = b, and every
// Maxwellian moment from a generic polynomial-in-(u, v, xi^2) expansion.  No blocking, no
// fusion.  Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may load this
// library; the CUDA path shares no code with it.
//
// Readings of points the paper leaves open (each is a switch in oracle_cfg where it has an
// alternative):
//   R-dt   dt = CFL * min over cells of min(dx/(|U|+c), dy/(|V|+c)); last step clipped to t_end.
//   R-char one characteristic basis per face line, the Euler x-eigensystem of the local-frame
//          state 0.5*(W_left + W_right); the same basis serves both sides and the tangential step.
//   R-eps  the WENO-Z epsilon is 1e-6, the value the paper gives for the time limiter.
//   R-tau  (tau_reading=0) the physical collision time is 0 outside the exponentials and tau_n
//          inside them; the printed exponent e^{t/tau_n} is read as e^{-t/tau_n}; the
//          Maxwellian normalisation is (lambda/pi)^{(K+2)/2}.  tau_reading=1: tau = tau_n.
//   R-LF   the L-F time derivative for S2O4 freezes the wave speed s and uses the
//          Cauchy-Kovalevskaya relation W_t = -(A W_n + B W_t) on each side.
//   R-alpha alpha^{n+1} is the product of the alpha_{p,m} of the last stage's Gauss-point
//          states; alpha^0 comes from a reconstruction of W^0 with alpha = 1.
//   R-tl   omega^t of a face is the minimum over both sides and the four characteristic
//          components of 2*at2/(at1+at2), built from beta_0..beta_3 of the face line's normal
//          reconstruction (computed whether or not the DF branch is taken).
//   R-bc   "free"/"non-reflecting" = zero-gradient copy; reflecting walls mirror with the
//          normal momentum negated; alpha ghosts use the same index map without sign change.
//   R-fb   (gp_fallback=1) a Gauss-point side state with rho<=0 or p<=0 is replaced by its
//          cell average with zero slopes.
//   R-eq34 strict "<" in Eq. 34; no extra condition beyond the if/else of Algorithm 1.
// ============================================================================================
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <cstdlib>
#include <vector>
#include <algorithm>
#include <limits>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {
typedef struct {
    int nx, ny;
    double x0, x1, y0, y1;
    double gamma, cfl;
    int bc[4];            // x-low, x-high, y-low, y-high: 0 periodic, 1 outflow (zero gradient), 2 reflecting wall
    double alpha_thres, dH, dL, eps, C1, C2;
    int flux;             // 0 gas-kinetic, 1 Lax-Friedrichs
    int time_limiter;     // 1: non-linear time limiter on the S2O4 update
    int tau_reading;      // 0: physical tau = 0 outside exponentials; 1: tau = tau_n everywhere
    int gp_fallback;      // 1: non-physical Gauss-point states fall back to the cell average
    int time_scheme;      // 0: S2O4, 1: SSP-RK3
    int dt_rule;          // 0: per-direction minimum, 1: CFL / max((|U|+c)/dx + (|V|+c)/dy)
    int df_states;        // left/right states of a Gauss point's DF factor: 0 the reconstructed
                          // Gauss-point states, 1 the cell averages beside the face
    int alpha_source;     // alpha^{n+1}: 0 from the last stage's Gauss points, 1 from a reconstruction
                          // of W^{n+1} itself with alpha^n deciding its DF branches
} oracle_cfg;

typedef struct {
    long fallbacks;       // Gauss-point side states replaced by the cell average
    long df_normal;       // normal reconstructions that took the DF branch
    long df_tangential;   // tangential reconstructions that took the DF branch
    long fail_step;       // step index of a positivity failure, -1 if none
    int fail_i, fail_j;   // first failing cell
} oracle_stats;
}

// ------------------------------------------------------------------------------------------
// Reverse-mode scalar for the oracle's own adjoint: every operation on `ad::Var` appends a node
// (up to two parents and the local partial derivatives) to a tape; a reverse sweep over the tape
// accumulates adjoints.  Branches are taken on values, so the forward pass fixes every decision.
// ------------------------------------------------------------------------------------------
namespace ad {
struct Tape {
    std::vector<int> pa, pb;
    std::vector<double> da, db;
    int push(int a, double ga, int b, double gb) {
        pa.push_back(a); da.push_back(ga); pb.push_back(b); db.push_back(gb);
        return (int)pa.size() - 1;
    }
    void clear() { pa.clear(); pb.clear(); da.clear(); db.clear(); }
};
static Tape* g_tape = nullptr;

struct Var {
    double v;
    int id;                        // -1: a constant
    Var() : v(0.0), id(-1) {}
    Var(double x) : v(x), id(-1) {}
    static Var leaf(double x) { Var r(x); r.id = g_tape->push(-1, 0.0, -1, 0.0); return r; }
};
inline Var mk(double v, int a, double ga, int b, double gb) {
    Var r(v);
    if (a >= 0 || b >= 0) r.id = g_tape->push(a, ga, b, gb);
    return r;
}
inline Var operator+(const Var& x, const Var& y) { return mk(x.v + y.v, x.id, 1.0, y.id, 1.0); }
inline Var operator-(const Var& x, const Var& y) { return mk(x.v - y.v, x.id, 1.0, y.id, -1.0); }
inline Var operator*(const Var& x, const Var& y) { return mk(x.v * y.v, x.id, y.v, y.id, x.v); }
inline Var operator/(const Var& x, const Var& y) { double q = x.v / y.v; return mk(q, x.id, 1.0 / y.v, y.id, -q / y.v); }
inline Var operator-(const Var& x) { return mk(-x.v, x.id, -1.0, -1, 0.0); }
inline Var operator+(const Var& x, double c) { return mk(x.v + c, x.id, 1.0, -1, 0.0); }
inline Var operator+(double c, const Var& x) { return mk(c + x.v, x.id, 1.0, -1, 0.0); }
inline Var operator-(const Var& x, double c) { return mk(x.v - c, x.id, 1.0, -1, 0.0); }
inline Var operator-(double c, const Var& x) { return mk(c - x.v, x.id, -1.0, -1, 0.0); }
inline Var operator*(const Var& x, double c) { return mk(x.v * c, x.id, c, -1, 0.0); }
inline Var operator*(double c, const Var& x) { return mk(c * x.v, x.id, c, -1, 0.0); }
inline Var operator/(const Var& x, double c) { return mk(x.v / c, x.id, 1.0 / c, -1, 0.0); }
inline Var operator/(double c, const Var& x) { double q = c / x.v; return mk(q, x.id, -q / x.v, -1, 0.0); }
inline bool operator<(const Var& x, const Var& y) { return x.v < y.v; }
inline bool operator>(const Var& x, const Var& y) { return x.v > y.v; }
inline bool operator<(const Var& x, double c) { return x.v < c; }
inline bool operator>(const Var& x, double c) { return x.v > c; }
inline bool operator<=(const Var& x, double c) { return x.v <= c; }
inline bool operator>=(const Var& x, double c) { return x.v >= c; }
inline Var fabs(const Var& x) { return x.v >= 0.0 ? mk(x.v, x.id, 1.0, -1, 0.0) : mk(-x.v, x.id, -1.0, -1, 0.0); }
inline Var sqrt(const Var& x) { double r = std::sqrt(x.v); return mk(r, x.id, 0.5 / r, -1, 0.0); }
inline Var exp(const Var& x) { double r = std::exp(x.v); return mk(r, x.id, r, -1, 0.0); }
inline Var erfc(const Var& x) {
    return mk(std::erfc(x.v), x.id, -2.0 / std::sqrt(M_PI) * std::exp(-x.v * x.v), -1, 0.0);
}
}  // namespace ad

namespace orc {
template <class R> struct Parallel { static const bool ok = true; };
template <> struct Parallel<ad::Var> { static const bool ok = false; };
}

namespace orc {

static const int G = 3;                 // ghost layers: the normal stencil reaches i-3 .. i+2
using std::fabs;
using std::sqrt;
using std::exp;
using std::erfc;

// ------------------------------------------------------------------------------------------
// Small dense linear algebra (Gauss-Jordan with partial pivoting)
// ------------------------------------------------------------------------------------------
template <class R>
static void solve_dense(int n, R* A /* n*n row-major, destroyed */, R* b /* n, in/out */) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
        if (piv != c) {
            for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
            std::swap(b[c], b[piv]);
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            R f = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; ++k) A[r * n + k] = A[r * n + k] - f * A[c * n + k];
            b[r] = b[r] - f * b[c];
        }
    }
    for (int r = 0; r < n; ++r) b[r] = b[r] / A[r * n + r];
}

template <class R>
static void invert4(const R M[4][4], R Inv[4][4]) {
    for (int col = 0; col < 4; ++col) {
        R A[16], e[4];
        for (int r = 0; r < 4; ++r) {
            for (int k = 0; k < 4; ++k) A[r * 4 + k] = M[r][k];
            e[r] = (r == col) ? R(1.0) : R(0.0);
        }
        solve_dense(4, A, e);
        for (int r = 0; r < 4; ++r) Inv[r][col] = e[r];
    }
}

// ------------------------------------------------------------------------------------------
// Sect. 3.1: WENO-AO tables.  Polynomials are in the cell-centred coordinate xi = (x - x_i)/dx,
// cell i = [-1/2, 1/2]; p_k is fixed by "its average over every cell of its sub-stencil equals
// that cell's value".  p0: cells i-2..i, p1: i-1..i+1, p2: i..i+2 (quadratics), p3: i-2..i+2.
// ------------------------------------------------------------------------------------------
struct Tables {
    double A[4][5][5];     // A[k][c][s]: coefficient of xi^c in p_k contributed by Q_{s-2}
    int deg[4];
    double d[4];           // linear weights d0..d3
    double glx[5], glw[5]; // 5-point Gauss-Legendre on [-1/2, 1/2]
};

static double cell_avg_monomial(int s, int c) {   // average of xi^c over [s-1/2, s+1/2]
    double hi = s + 0.5, lo = s - 0.5;
    return (std::pow(hi, c + 1) - std::pow(lo, c + 1)) / (c + 1);
}

static void gauss_legendre5(double* x, double* w) {
    // roots of the Legendre polynomial P5 by Newton iteration from the Chebyshev guesses
    const int n = 5;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) { double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp; z -= dz;
            if (fabs(dz) < 1e-17) break;
        }
        x[i] = 0.5 * z;                                  // map [-1,1] -> [-1/2,1/2]
        w[i] = 0.5 * 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

static Tables make_tables(double dH, double dL) {
    Tables T;
    std::memset(&T, 0, sizeof(T));
    const int lo[4] = {-2, -1, 0, -2};
    const int np[4] = {3, 3, 3, 5};
    for (int k = 0; k < 4; ++k) {
        int n = np[k];
        T.deg[k] = n - 1;
        for (int m = 0; m < n; ++m) {           // column m of the inverse: response to Q_{lo+m} = 1
            double M[25], e[5];
            for (int r = 0; r < n; ++r) {
                for (int c = 0; c < n; ++c) M[r * n + c] = cell_avg_monomial(lo[k] + r, c);
                e[r] = (r == m) ? 1.0 : 0.0;
            }
            solve_dense<double>(n, M, e);
            for (int c = 0; c < n; ++c) T.A[k][c][lo[k] + m + 2] = e[c];
        }
    }
    // linear weights (Sect. 3.1)
    T.d[3] = dH;
    T.d[0] = (1.0 - dH) * (1.0 - dL) / 2.0;
    T.d[1] = (1.0 - dH) * dL;
    T.d[2] = T.d[0];
    gauss_legendre5(T.glx, T.glw);
    return T;
}

template <class R>
struct PolyK { R a[5]; int deg; };

template <class R>
static PolyK<R> sub_poly(const Tables& T, int k, const R Q[5]) {
    PolyK<R> p;
    p.deg = T.deg[k];
    for (int c = 0; c < 5; ++c) {
        R s = R(0.0);
        for (int m = 0; m < 5; ++m)
            if (T.A[k][c][m] != 0.0) s = s + T.A[k][c][m] * Q[m];
        p.a[c] = s;
    }
    return p;
}

// q-th derivative (d/dxi)^q of p at xi
template <class R>
static R poly_deriv(const PolyK<R>& p, int q, double xi) {
    R s = R(0.0);
    for (int c = p.deg; c >= q; --c) {
        double f = 1.0;
        for (int t = 0; t < q; ++t) f *= (c - t);
        s = s + f * p.a[c] * std::pow(xi, c - q);
    }
    return s;
}

// Eq. 38 in the cell-centred coordinate: beta = sum_q int_{-1/2}^{1/2} (d^q p / dxi^q)^2 dxi
template <class R>
static R smoothness(const Tables& T, const PolyK<R>& p) {
    R b = R(0.0);
    for (int q = 1; q <= p.deg; ++q)
        for (int g = 0; g < 5; ++g) {
            R v = poly_deriv(p, q, T.glx[g]);
            b = b + T.glw[g] * (v * v);
        }
    return b;
}

// Result of one 1-D hybrid reconstruction of one characteristic component.
template <class R>
struct Recon1D {
    R val[2], slope[2];    // at up to two evaluation points; slope is d/dxi (divide by the cell size)
    R beta[4];             // beta_0..beta_3 (Eq. 38)
    bool df;               // the DF branch was taken
};

// WENO-AO (Sect. 3.1) or, when the hybrid switch holds (Eq. 34), the zero-mean DF quadratic:
// p1 in zero-mean form scaled by the cell's alpha (Sect. 3.3).
template <class R>
static Recon1D<R> recon1d(const Tables& T, const R Q[5], int neval, const double* xi_eval,
                          bool use_df, double alpha_cell, double eps) {
    Recon1D<R> out;
    PolyK<R> p[4];
    for (int k = 0; k < 4; ++k) p[k] = sub_poly(T, k, Q);
    for (int k = 0; k < 4; ++k) out.beta[k] = smoothness(T, p[k]);
    out.df = use_df;
    if (use_df) {
        // p_DF = Q_i + alpha_i * (p1 - mean(p1)), and mean(p1) = Q_i by construction
        for (int e = 0; e < neval; ++e) {
            out.val[e] = Q[2] + alpha_cell * (poly_deriv(p[1], 0, xi_eval[e]) - Q[2]);
            out.slope[e] = alpha_cell * poly_deriv(p[1], 1, xi_eval[e]);
        }
        return out;
    }
    // Eq. 37: global smoothness indicator
    R tauZ = (fabs(out.beta[3] - out.beta[0]) + fabs(out.beta[3] - out.beta[1]) +
              fabs(out.beta[3] - out.beta[2])) / 3.0;
    // WENO-Z non-linear weights and their normalisation
    R w[4], wsum = R(0.0);
    for (int k = 0; k < 4; ++k) {
        R r = tauZ / (out.beta[k] + eps);
        w[k] = T.d[k] * (1.0 + r * r);
        wsum = wsum + w[k];
    }
    R wb[4];
    for (int k = 0; k < 4; ++k) wb[k] = w[k] / wsum;
    // P = wb3 * (p3/d3 - sum_k d_k/d3 p_k) + sum_k wb_k p_k
    for (int e = 0; e < neval; ++e)
        for (int q = 0; q <= 1; ++q) {
            R pv[4];
            for (int k = 0; k < 4; ++k) pv[k] = poly_deriv(p[k], q, xi_eval[e]);
            R hi = pv[3] / T.d[3];
            for (int k = 0; k < 3; ++k) hi = hi - (T.d[k] / T.d[3]) * pv[k];
            R P = wb[3] * hi;
            for (int k = 0; k < 3; ++k) P = P + wb[k] * pv[k];
            if (q == 0) out.val[e] = P; else out.slope[e] = P;
        }
    return out;
}

// Time-limiter ingredient of one side (Sect. 2.2): 2*at2/(at1+at2)
template <class R>
static R limiter_alpha(const R beta[4], double eps) {
    R bmin = beta[0], bmax = beta[0];
    for (int k = 1; k < 4; ++k) { if (beta[k] < bmin) bmin = beta[k]; if (beta[k] > bmax) bmax = beta[k]; }
    R tauZ = (fabs(beta[3] - beta[0]) + fabs(beta[3] - beta[1]) + fabs(beta[3] - beta[2])) / 3.0;
    R r1 = tauZ / (bmin + eps), r2 = tauZ / (bmax + eps);
    R a1 = 1.0 + r1 * r1, a2 = 1.0 + r2 * r2;
    return 2.0 * a2 / (a1 + a2);
}

// ------------------------------------------------------------------------------------------
// Euler state helpers (Sect. 2.2, 2.3): W = (rho, rho U, rho V, rho E)
// ------------------------------------------------------------------------------------------
template <class R>
struct Prim { R rho, U, V, p, lam; };

template <class R>
static Prim<R> prim_of(const R W[4], double gamma) {
    Prim<R> s;
    s.rho = W[0];
    s.U = W[1] / W[0];
    s.V = W[2] / W[0];
    s.p = (gamma - 1.0) * (W[3] - 0.5 * s.rho * (s.U * s.U + s.V * s.V));
    s.lam = s.rho / (2.0 * s.p);
    return s;
}

// Characteristic basis: right eigenvectors of the Euler x-flux Jacobian at a state, and their inverse
template <class R>
struct Basis { R L[4][4], Rm[4][4]; };

template <class R>
static Basis<R> char_basis(const R Wbar[4], double gamma) {
    Prim<R> s = prim_of(Wbar, gamma);
    R c = sqrt(gamma * s.p / s.rho);
    R H = (Wbar[3] + s.p) / s.rho;
    R q2 = 0.5 * (s.U * s.U + s.V * s.V);
    Basis<R> B;
    // columns: u-c, u (entropy), u (shear), u+c
    R cols[4][4] = {{R(1.0), s.U - c, s.V, H - s.U * c},
                    {R(1.0), s.U, s.V, q2},
                    {R(0.0), R(0.0), R(1.0), s.V},
                    {R(1.0), s.U + c, s.V, H + s.U * c}};
    for (int r = 0; r < 4; ++r)
        for (int k = 0; k < 4; ++k) B.Rm[r][k] = cols[k][r];
    invert4(B.Rm, B.L);
    return B;
}

template <class R>
static void matvec4(const R M[4][4], const R x[4], R y[4]) {
    for (int r = 0; r < 4; ++r) {
        R s = R(0.0);
        for (int k = 0; k < 4; ++k) s = s + M[r][k] * x[k];
        y[r] = s;
    }
}

// Euler normal flux and the x/y flux Jacobians (Sect. 2.3)
template <class R>
static void euler_flux_x(const R W[4], double gamma, R F[4]) {
    Prim<R> s = prim_of(W, gamma);
    F[0] = W[1];
    F[1] = W[1] * s.U + s.p;
    F[2] = W[1] * s.V;
    F[3] = s.U * (W[3] + s.p);
}

template <class R>
static void euler_jacobians(const R W[4], double gamma, R A[4][4], R B[4][4]) {
    Prim<R> s = prim_of(W, gamma);
    R u = s.U, v = s.V, H = (W[3] + s.p) / s.rho, g1 = gamma - 1.0;
    R phi = 0.5 * g1 * (u * u + v * v);
    R a[4][4] = {{R(0.0), R(1.0), R(0.0), R(0.0)},
                 {phi - u * u, (3.0 - gamma) * u, -g1 * v, R(g1)},
                 {-u * v, v, u, R(0.0)},
                 {u * (phi - H), H - g1 * u * u, -g1 * u * v, gamma * u}};
    R b[4][4] = {{R(0.0), R(0.0), R(1.0), R(0.0)},
                 {-u * v, v, u, R(0.0)},
                 {phi - v * v, -g1 * u, (3.0 - gamma) * v, R(g1)},
                 {v * (phi - H), -g1 * u * v, H - g1 * v * v, gamma * v}};
    for (int r = 0; r < 4; ++r)
        for (int k = 0; k < 4; ++k) { A[r][k] = a[r][k]; B[r][k] = b[r][k]; }
}

// ------------------------------------------------------------------------------------------
// Sect. 2.2: Maxwellian moments.  A polynomial in (u, v, xi^2) is a list of terms
// coef * u^a v^b (xi^2)^k.  <P> is its normalised moment (1/rho) int P g dXi over all
// velocities, or over the half-space u>0 (half=+1) / u<0 (half=-1).
// ------------------------------------------------------------------------------------------
template <class R>
struct Term { R c; int a, b, k; };

template <class R>
struct Poly {
    Term<R> t[64];
    int n = 0;
    void add(const R& c, int a, int b, int k) {
        if (n >= 64 || a > 7 || b > 7 || k > 2) { std::fprintf(stderr, "oracle: polynomial overflow\n"); std::abort(); }
        t[n].c = c; t[n].a = a; t[n].b = b; t[n].k = k; ++n;
    }
};

// a = a1 + a2 u + a3 v + a4 * (u^2 + v^2 + xi^2)/2
template <class R>
static Poly<R> poly_from_coeffs(const R a[4]) {
    Poly<R> P;
    P.add(a[0], 0, 0, 0);
    P.add(a[1], 1, 0, 0);
    P.add(a[2], 0, 1, 0);
    P.add(R(0.5 * a[3]), 2, 0, 0);
    P.add(R(0.5 * a[3]), 0, 2, 0);
    P.add(R(0.5 * a[3]), 0, 0, 1);
    return P;
}

// P * u^i v^j
template <class R>
static Poly<R> poly_shift(const Poly<R>& P, int i, int j) {
    Poly<R> Q;
    for (int q = 0; q < P.n; ++q) Q.add(P.t[q].c, P.t[q].a + i, P.t[q].b + j, P.t[q].k);
    return Q;
}

template <class R>
static Poly<R> poly_add(const Poly<R>& P, const Poly<R>& Q) {
    Poly<R> S = P;
    for (int q = 0; q < Q.n; ++q) S.add(Q.t[q].c, Q.t[q].a, Q.t[q].b, Q.t[q].k);
    return S;
}

template <class R>
struct Moments { R u[10], v[10], x[4]; };

// <u^n>: full moments by the Gaussian recursion; half-space moments start from erfc and exp
template <class R>
static Moments<R> moments(const Prim<R>& s, int half, double K) {
    Moments<R> m;
    R inv2l = 1.0 / (2.0 * s.lam);
    if (half == 0) {
        m.u[0] = R(1.0);
        m.u[1] = s.U;
    } else {
        R sl = sqrt(s.lam);
        R e = exp(-s.lam * s.U * s.U) / (2.0 * sqrt(M_PI * s.lam));
        if (half > 0) { m.u[0] = 0.5 * erfc(-sl * s.U); m.u[1] = s.U * m.u[0] + e; }
        else          { m.u[0] = 0.5 * erfc(sl * s.U);  m.u[1] = s.U * m.u[0] - e; }
    }
    for (int n = 2; n < 10; ++n) m.u[n] = s.U * m.u[n - 1] + (double)(n - 1) * inv2l * m.u[n - 2];
    m.v[0] = R(1.0);
    m.v[1] = s.V;
    for (int n = 2; n < 10; ++n) m.v[n] = s.V * m.v[n - 1] + (double)(n - 1) * inv2l * m.v[n - 2];
    m.x[0] = R(1.0);
    m.x[1] = K * inv2l;                                  // <|xi|^2> = K/(2 lambda)
    m.x[2] = K * (K + 2.0) * inv2l * inv2l;              // <|xi|^4> = K(K+2)/(4 lambda^2)
    m.x[3] = K * (K + 2.0) * (K + 4.0) * inv2l * inv2l * inv2l;   // <|xi|^6>, reached only by guards
    return m;
}

template <class R>
static R avg(const Poly<R>& P, const Moments<R>& m) {
    R s = R(0.0);
    for (int q = 0; q < P.n; ++q) s = s + P.t[q].c * (m.u[P.t[q].a] * m.v[P.t[q].b] * m.x[P.t[q].k]);
    return s;
}

// <P psi>, psi = (1, u, v, (u^2+v^2+xi^2)/2)
template <class R>
static void avg_psi(const Poly<R>& P, const Moments<R>& m, R out[4]) {
    out[0] = avg(P, m);
    out[1] = avg(poly_shift(P, 1, 0), m);
    out[2] = avg(poly_shift(P, 0, 1), m);
    R s = R(0.0);
    for (int q = 0; q < P.n; ++q) {
        const Term<R>& t = P.t[q];
        R e = m.u[t.a + 2] * m.v[t.b] * m.x[t.k] + m.u[t.a] * m.v[t.b + 2] * m.x[t.k] + m.u[t.a] * m.v[t.b] * m.x[t.k + 1];
        s = s + 0.5 * t.c * e;
    }
    out[3] = s;
}

// <a psi> = b for the coefficients a of a = a1 + a2 u + a3 v + a4 (u^2+v^2+xi^2)/2 (Sect. 2.2)
template <class R>
static void slope_solve(const Moments<R>& mfull, const R b[4], R a[4]) {
    R M[16];
    for (int j = 0; j < 4; ++j) {
        R e[4] = {R(0.0), R(0.0), R(0.0), R(0.0)};
        e[j] = R(1.0);
        Poly<R> Pj = poly_from_coeffs(e);
        R col[4];
        avg_psi(Pj, mfull, col);
        for (int i = 0; i < 4; ++i) M[i * 4 + j] = col[i];
    }
    for (int i = 0; i < 4; ++i) a[i] = b[i];
    solve_dense(4, M, a);
}

// Time integrals over [0, delta] of the coefficients of the second-order interface
// distribution (Sect. 2.2), T = tau_n in the exponentials, tau elsewhere.
template <class R>
struct Gammas { R gc, ac, Ac, glr, alr, Alr; };

template <class R>
static Gammas<R> time_integrals(R T, R tau, double delta) {
    Gammas<R> g;
    R E, oneE;
    if (T > 0.0) { E = exp(-delta / T); oneE = 1.0 - E; }
    else         { E = R(0.0); oneE = R(1.0); }
    g.gc  = delta - T * oneE;                               // int (1 - e^{-t/T})
    g.ac  = (T * T + T * tau) * oneE - T * delta * E - tau * delta;   // int ((t+tau) e^{-t/T} - tau)
    g.Ac  = 0.5 * delta * delta - tau * delta + T * tau * oneE;      // int (t - tau + tau e^{-t/T})
    g.glr = T * oneE;                                       // int e^{-t/T}
    g.alr = -((T * T + T * tau) * oneE - T * delta * E);    // int -(tau + t) e^{-t/T}
    g.Alr = -T * tau * oneE;                                // int -tau e^{-t/T}
    return g;
}

struct FluxParams { double gamma, K, C1, C2, dt; int tau_reading; };

// Gas-kinetic flux at one Gauss point in the local frame (Sect. 2.2, Sect. 3.4, Eqs. 25-27).
// Inputs: left/right conserved states with normal (x) and tangential (y) slopes.
template <class R>
static void gks_point(const FluxParams& P, const R WL[4], const R WLx[4], const R WLy[4],
                      const R WR[4], const R WRx[4], const R WRy[4], R F[4], R dtF[4]) {
    Prim<R> sl = prim_of(WL, P.gamma), sr = prim_of(WR, P.gamma);
    Moments<R> mlF = moments(sl, 0, P.K), mrF = moments(sr, 0, P.K);
    Moments<R> mlH = moments(sl, +1, P.K), mrH = moments(sr, -1, P.K);
    // slope coefficients of the initial left/right Maxwellians: <a psi> = W'/rho
    R bl[4], br[4], alx[4], aly[4], arx[4], ary[4];
    for (int k = 0; k < 4; ++k) bl[k] = WLx[k] / sl.rho;
    slope_solve(mlF, bl, alx);
    for (int k = 0; k < 4; ++k) bl[k] = WLy[k] / sl.rho;
    slope_solve(mlF, bl, aly);
    for (int k = 0; k < 4; ++k) br[k] = WRx[k] / sr.rho;
    slope_solve(mrF, br, arx);
    for (int k = 0; k < 4; ++k) br[k] = WRy[k] / sr.rho;
    slope_solve(mrF, br, ary);
    Poly<R> one; one.add(R(1.0), 0, 0, 0);
    Poly<R> Palx = poly_from_coeffs(alx), Paly = poly_from_coeffs(aly);
    Poly<R> Parx = poly_from_coeffs(arx), Pary = poly_from_coeffs(ary);
    // Sect. 3.4: equilibrium state and its slopes by kinetic weighting
    R Wc[4], Wcx[4], Wcy[4], tl[4], tr[4];
    avg_psi(one, mlH, tl); avg_psi(one, mrH, tr);
    for (int k = 0; k < 4; ++k) Wc[k] = sl.rho * tl[k] + sr.rho * tr[k];
    avg_psi(Palx, mlH, tl); avg_psi(Parx, mrH, tr);
    for (int k = 0; k < 4; ++k) Wcx[k] = sl.rho * tl[k] + sr.rho * tr[k];
    avg_psi(Paly, mlH, tl); avg_psi(Pary, mrH, tr);
    for (int k = 0; k < 4; ++k) Wcy[k] = sl.rho * tl[k] + sr.rho * tr[k];
    Prim<R> sc = prim_of(Wc, P.gamma);
    Moments<R> mc = moments(sc, 0, P.K);
    R b[4], acx[4], acy[4], Ac[4];
    for (int k = 0; k < 4; ++k) b[k] = Wcx[k] / sc.rho;
    slope_solve(mc, b, acx);
    for (int k = 0; k < 4; ++k) b[k] = Wcy[k] / sc.rho;
    slope_solve(mc, b, acy);
    Poly<R> Pacx = poly_from_coeffs(acx), Pacy = poly_from_coeffs(acy);
    // compatibility <A + a_x u + a_y v> = 0
    Poly<R> adv_c = poly_add(poly_shift(Pacx, 1, 0), poly_shift(Pacy, 0, 1));
    avg_psi(adv_c, mc, b);
    for (int k = 0; k < 4; ++k) b[k] = -b[k];
    slope_solve(mc, b, Ac);
    Poly<R> PAc = poly_from_coeffs(Ac);
    // numerical collision time
    R dp = fabs((sl.p - sr.p) / (sl.p + sr.p));
    R T = P.C1 * P.dt + P.C2 * dp * P.dt;
    R tau = (P.tau_reading == 1) ? T : R(0.0);
    // flux moments
    Poly<R> u1 = poly_shift(one, 1, 0);
    R Mc0[4], Mc1[4], Mc2[4], Ml0[4], Mr0[4], Ml1[4], Mr1[4], Ml2[4], Mr2[4];
    avg_psi(u1, mc, Mc0);
    avg_psi(poly_shift(adv_c, 1, 0), mc, Mc1);
    avg_psi(poly_shift(PAc, 1, 0), mc, Mc2);
    avg_psi(u1, mlH, Ml0);
    avg_psi(u1, mrH, Mr0);
    Poly<R> adv_l = poly_add(poly_shift(Palx, 1, 0), poly_shift(Paly, 0, 1));
    Poly<R> adv_r = poly_add(poly_shift(Parx, 1, 0), poly_shift(Pary, 0, 1));
    avg_psi(poly_shift(adv_l, 1, 0), mlH, Ml1);
    avg_psi(poly_shift(adv_r, 1, 0), mrH, Mr1);
    for (int k = 0; k < 4; ++k) { Ml2[k] = R(0.0); Mr2[k] = R(0.0); }
    if (P.tau_reading == 1) {
        // time-derivative coefficients of the left/right states (needed only when tau != 0)
        R Al[4], Ar[4];
        avg_psi(adv_l, mlF, b);
        for (int k = 0; k < 4; ++k) b[k] = -b[k];
        slope_solve(mlF, b, Al);
        avg_psi(adv_r, mrF, b);
        for (int k = 0; k < 4; ++k) b[k] = -b[k];
        slope_solve(mrF, b, Ar);
        avg_psi(poly_shift(poly_from_coeffs(Al), 1, 0), mlH, Ml2);
        avg_psi(poly_shift(poly_from_coeffs(Ar), 1, 0), mrH, Mr2);
    }
    // Eq. 25 for delta = dt and dt/2, then Eq. 27
    R Fd[2][4];
    for (int h = 0; h < 2; ++h) {
        double delta = (h == 0) ? P.dt : 0.5 * P.dt;
        Gammas<R> g = time_integrals(T, tau, delta);
        for (int k = 0; k < 4; ++k)
            Fd[h][k] = sc.rho * (g.gc * Mc0[k] + g.ac * Mc1[k] + g.Ac * Mc2[k])
                     + g.glr * (sl.rho * Ml0[k] + sr.rho * Mr0[k])
                     + g.alr * (sl.rho * Ml1[k] + sr.rho * Mr1[k])
                     + g.Alr * (sl.rho * Ml2[k] + sr.rho * Mr2[k]);
    }
    for (int k = 0; k < 4; ++k) {
        F[k] = (4.0 * Fd[1][k] - Fd[0][k]) / P.dt;
        dtF[k] = 4.0 * (Fd[0][k] - 2.0 * Fd[1][k]) / (P.dt * P.dt);
    }
}

// Lax-Friedrichs flux at one Gauss point in the local frame (Sect. 2.3) and its time
// derivative (reading R-LF: frozen s, Cauchy-Kovalevskaya W_t = -(A W_x + B W_y)).
template <class R>
static void lf_point(double gamma, const R WL[4], const R WLx[4], const R WLy[4],
                     const R WR[4], const R WRx[4], const R WRy[4], R F[4], R dtF[4]) {
    Prim<R> sl = prim_of(WL, gamma), sr = prim_of(WR, gamma);
    R FL[4], FR[4];
    euler_flux_x(WL, gamma, FL);
    euler_flux_x(WR, gamma, FR);
    R cl = sqrt(gamma * sl.p / sl.rho), cr = sqrt(gamma * sr.p / sr.rho);
    R s = std::max(fabs(sl.U) + cl, fabs(sr.U) + cr);
    for (int k = 0; k < 4; ++k) F[k] = 0.5 * (FL[k] + FR[k]) - 0.5 * s * (WR[k] - WL[k]);
    R Al[4][4], Bl[4][4], Ar[4][4], Br[4][4];
    euler_jacobians(WL, gamma, Al, Bl);
    euler_jacobians(WR, gamma, Ar, Br);
    R t1[4], t2[4], Wtl[4], Wtr[4], AWl[4], AWr[4];
    matvec4(Al, WLx, t1); matvec4(Bl, WLy, t2);
    for (int k = 0; k < 4; ++k) Wtl[k] = -(t1[k] + t2[k]);
    matvec4(Ar, WRx, t1); matvec4(Br, WRy, t2);
    for (int k = 0; k < 4; ++k) Wtr[k] = -(t1[k] + t2[k]);
    matvec4(Al, Wtl, AWl); matvec4(Ar, Wtr, AWr);
    for (int k = 0; k < 4; ++k) dtF[k] = 0.5 * (AWl[k] + AWr[k]) - 0.5 * s * (Wtr[k] - Wtl[k]);
}

// Sect. 3.2: DF factor of one Gauss point from its left/right states in the local frame
template <class R>
static R df_alpha_point(const R WL[4], const R WR[4], double gamma) {
    Prim<R> l = prim_of(WL, gamma), r = prim_of(WR, gamma);
    R cl = sqrt(gamma * l.p / l.rho), cr = sqrt(gamma * r.p / r.rho);
    R jp = fabs(l.p - r.p);
    R dn = l.U / cl - r.U / cr, dtn = l.V / cl - r.V / cr;
    R D = jp / l.p + jp / r.p + dn * dn + dtn * dtn;
    return 1.0 / (1.0 + D * D);
}

// ------------------------------------------------------------------------------------------
// Mesh with ghost layers; direction-generic face addressing in the local frame of each face
// (Sect. 2.1): x-faces use the global frame; y-faces rotate by theta = pi/2, so the local
// normal is +y and the local tangential axis is -x.
// ------------------------------------------------------------------------------------------
template <class R>
struct Field {
    int nx, ny, NX, NY;
    std::vector<R> w[4];
    std::vector<double> alpha;
    void init(int nx_, int ny_) {
        nx = nx_; ny = ny_; NX = nx + 2 * G; NY = ny + 2 * G;
        for (int k = 0; k < 4; ++k) w[k].assign((size_t)NX * NY, R(0.0));
        alpha.assign((size_t)NX * NY, 1.0);
    }
    size_t id(int i, int j) const { return (size_t)(j + G) * NX + (i + G); }
};

struct Ctx {
    oracle_cfg cfg;
    Tables T;
    double dx, dy, K;
};

// ghost source index for a coordinate outside [0, n): returns interior index and whether it mirrors
static int ghost_map(int k, int n, int bc_lo, int bc_hi, bool& mirrored) {
    mirrored = false;
    if (k < 0) {
        if (bc_lo == 0) return k + n;
        if (bc_lo == 1) return 0;
        mirrored = true; return -1 - k;
    }
    if (k >= n) {
        if (bc_hi == 0) return k - n;
        if (bc_hi == 1) return n - 1;
        mirrored = true; return 2 * n - 1 - k;
    }
    return k;
}

// Boundary condition (Algorithm 1, "update boundary condition"): x pass over interior rows,
// then y pass over all columns, so corners are filled too.
template <class R>
static void fill_ghosts(const Ctx& C, Field<R>& F, bool with_alpha) {
    const int nx = F.nx, ny = F.ny;
    for (int j = 0; j < ny; ++j)
        for (int i = -G; i < nx + G; ++i) {
            if (i >= 0 && i < nx) continue;
            bool mir;
            int s = ghost_map(i, nx, C.cfg.bc[0], C.cfg.bc[1], mir);
            for (int k = 0; k < 4; ++k) F.w[k][F.id(i, j)] = F.w[k][F.id(s, j)];
            if (mir) F.w[1][F.id(i, j)] = -F.w[1][F.id(i, j)];
            if (with_alpha) F.alpha[F.id(i, j)] = F.alpha[F.id(s, j)];
        }
    for (int j = -G; j < ny + G; ++j) {
        if (j >= 0 && j < ny) continue;
        for (int i = -G; i < nx + G; ++i) {
            bool mir;
            int s = ghost_map(j, ny, C.cfg.bc[2], C.cfg.bc[3], mir);
            for (int k = 0; k < 4; ++k) F.w[k][F.id(i, j)] = F.w[k][F.id(i, s)];
            if (mir) F.w[2][F.id(i, j)] = -F.w[2][F.id(i, j)];
            if (with_alpha) F.alpha[F.id(i, j)] = F.alpha[F.id(i, s)];
        }
    }
}

// Direction descriptor: dir 0 = x-faces, dir 1 = y-faces
struct Dir {
    int dir, nn, nt;      // cells along the normal / tangential direction
    double dn, dt;        // cell sizes along the normal / tangential direction
    int sigma;            // global tangential index step per local +y~ step
};
static Dir make_dir(const Ctx& C, int dir) {
    Dir d;
    d.dir = dir;
    if (dir == 0) { d.nn = C.cfg.nx; d.nt = C.cfg.ny; d.dn = C.dx; d.dt = C.dy; d.sigma = +1; }
    else          { d.nn = C.cfg.ny; d.nt = C.cfg.nx; d.dn = C.dy; d.dt = C.dx; d.sigma = -1; }
    return d;
}
// cell (normal index n, tangential index t) in the local frame of a face of direction d
template <class R>
static void cell_local(const Field<R>& F, const Dir& d, int n, int t, R W[4]) {
    size_t id = (d.dir == 0) ? F.id(n, t) : F.id(t, n);
    if (d.dir == 0) { for (int k = 0; k < 4; ++k) W[k] = F.w[k][id]; }
    else { W[0] = F.w[0][id]; W[1] = F.w[2][id]; W[2] = -F.w[1][id]; W[3] = F.w[3][id]; }   // W~ = T W
}
template <class R>
static double alpha_at(const Field<R>& F, const Dir& d, int n, int t) {
    return (d.dir == 0) ? F.alpha[F.id(n, t)] : F.alpha[F.id(t, n)];
}

// Per-face-line results of the normal reconstruction (Algorithm 1, normal step)
template <class R>
struct LineRec { R WL[4], WLn[4], WR[4], WRn[4]; R tl_alpha; bool dfL[4], dfR[4]; };

// Normal reconstruction on face line (f, t): face f sits between normal cells f-1 (left) and f.
template <class R>
static LineRec<R> normal_line(const Ctx& C, const Field<R>& F, const Dir& d, int f, int t) {
    const oracle_cfg& cf = C.cfg;
    R W[6][4];
    double al[6];
    for (int s = 0; s < 6; ++s) { cell_local(F, d, f - 3 + s, t, W[s]); al[s] = alpha_at(F, d, f - 3 + s, t); }
    R Wbar[4];
    for (int k = 0; k < 4; ++k) Wbar[k] = 0.5 * (W[2][k] + W[3][k]);
    Basis<R> B = char_basis(Wbar, cf.gamma);
    R Q[6][4];
    for (int s = 0; s < 6; ++s) matvec4(B.L, W[s], Q[s]);
    bool dfL = std::max(std::max(al[1], al[2]), al[3]) < cf.alpha_thres;    // Eq. 34, cell f-1
    bool dfR = std::max(std::max(al[2], al[3]), al[4]) < cf.alpha_thres;    // Eq. 34, cell f
    R qL[4], qLn[4], qR[4], qRn[4];
    R tlL = R(1.0), tlR = R(1.0);
    LineRec<R> rec;
    const double xiL = 0.5, xiR = -0.5;
    for (int k = 0; k < 4; ++k) {
        R sL[5], sR[5];
        for (int m = 0; m < 5; ++m) { sL[m] = Q[m][k]; sR[m] = Q[m + 1][k]; }
        Recon1D<R> rl = recon1d(C.T, sL, 1, &xiL, dfL, al[2], cf.eps);
        Recon1D<R> rr = recon1d(C.T, sR, 1, &xiR, dfR, al[3], cf.eps);
        qL[k] = rl.val[0]; qLn[k] = rl.slope[0] / d.dn;
        qR[k] = rr.val[0]; qRn[k] = rr.slope[0] / d.dn;
        R aLk = limiter_alpha(rl.beta, cf.eps), aRk = limiter_alpha(rr.beta, cf.eps);
        if (aLk < tlL) tlL = aLk;
        if (aRk < tlR) tlR = aRk;
        rec.dfL[k] = dfL; rec.dfR[k] = dfR;
    }
    matvec4(B.Rm, qL, rec.WL); matvec4(B.Rm, qLn, rec.WLn);
    matvec4(B.Rm, qR, rec.WR); matvec4(B.Rm, qRn, rec.WRn);
    rec.tl_alpha = (tlL < tlR) ? tlL : tlR;
    return rec;
}

// Gauss-point states of one side of a face after the tangential reconstruction
template <class R>
struct GPSide { R W[2][4], Wn[2][4], Wt[2][4]; bool fallback[2]; bool df; };

// Per-face results
template <class R>
struct FaceRec { R F[4], dtF[4]; R omega; R alpha_gp[2]; int nfallback; };

struct Counters { long fallbacks = 0, df_n = 0, df_t = 0; };

template <class R>
static bool physical(const R W[4], double gamma) {
    if (!(W[0] > 0.0)) return false;
    R p = (gamma - 1.0) * (W[3] - 0.5 * (W[1] * W[1] + W[2] * W[2]) / W[0]);
    return p > 0.0;
}

// Tangential reconstruction and flux of face (f, t) (Algorithm 1, tangential step and flux loop)
template <class R>
static FaceRec<R> face_flux(const Ctx& C, const Field<R>& F, const Dir& d, int f, int t,
                            const std::vector<LineRec<R>>& lines, int line_stride,
                            double dt, bool want_flux, Counters& cnt, GPSide<R>* sides_out) {
    const oracle_cfg& cf = C.cfg;
    FaceRec<R> fr;
    GPSide<R> sides[2];
    // basis of face line (f, t): the same one its normal step used
    R W2[4], W3[4], Wbar[4];
    cell_local(F, d, f - 1, t, W2);
    cell_local(F, d, f, t, W3);
    for (int k = 0; k < 4; ++k) Wbar[k] = 0.5 * (W2[k] + W3[k]);
    Basis<R> B = char_basis(Wbar, cf.gamma);
    const double eta[2] = {-std::sqrt(3.0) / 6.0, std::sqrt(3.0) / 6.0};   // Gauss points m = 1, 2
    auto line_at = [&](int b) -> const LineRec<R>& { return lines[(size_t)(t + d.sigma * b + 2) * line_stride + f]; };
    for (int side = 0; side < 2; ++side) {
        int ncell = (side == 0) ? f - 1 : f;
        double al[3];
        for (int b = -1; b <= 1; ++b) al[b + 1] = alpha_at(F, d, ncell, t + d.sigma * b);
        bool df = std::max(std::max(al[0], al[1]), al[2]) < cf.alpha_thres;   // Eq. 34, tangential
        GPSide<R>& S = sides[side];
        S.df = df;
        R Q[5][4];
        for (int b = -2; b <= 2; ++b) {
            const LineRec<R>& L = line_at(b);
            matvec4(B.L, side == 0 ? L.WL : L.WR, Q[b + 2]);
        }
        R qv[2][4], qt[2][4];
        for (int k = 0; k < 4; ++k) {
            R s[5];
            for (int m = 0; m < 5; ++m) s[m] = Q[m][k];
            Recon1D<R> r = recon1d(C.T, s, 2, eta, df, al[1], cf.eps);
            for (int m = 0; m < 2; ++m) { qv[m][k] = r.val[m]; qt[m][k] = r.slope[m] / d.dt; }
        }
        const LineRec<R>& L0 = line_at(0);
        for (int m = 0; m < 2; ++m) {
            matvec4(B.Rm, qv[m], S.W[m]);
            matvec4(B.Rm, qt[m], S.Wt[m]);
            for (int k = 0; k < 4; ++k) S.Wn[m][k] = side == 0 ? L0.WLn[k] : L0.WRn[k];
            S.fallback[m] = false;
            if (cf.gp_fallback && !physical(S.W[m], cf.gamma)) {
                R Wc[4];
                cell_local(F, d, ncell, t, Wc);
                for (int k = 0; k < 4; ++k) { S.W[m][k] = Wc[k]; S.Wn[m][k] = R(0.0); S.Wt[m][k] = R(0.0); }
                S.fallback[m] = true;
            }
        }
        if (df) cnt.df_t += 1;
    }
    fr.nfallback = 0;
    for (int s = 0; s < 2; ++s) for (int m = 0; m < 2; ++m) fr.nfallback += sides[s].fallback[m] ? 1 : 0;
    if (sides_out) { sides_out[0] = sides[0]; sides_out[1] = sides[1]; }
    for (int m = 0; m < 2; ++m) fr.alpha_gp[m] = df_alpha_point(sides[0].W[m], sides[1].W[m], cf.gamma);
    if (cf.df_states == 1) {
        // the alternative reading: the states on either side of the Gauss point are the cell averages
        R Wl[4], Wr[4];
        cell_local(F, d, f - 1, t, Wl);
        cell_local(F, d, f, t, Wr);
        for (int m = 0; m < 2; ++m) fr.alpha_gp[m] = df_alpha_point(Wl, Wr, cf.gamma);
    }
    for (int k = 0; k < 4; ++k) { fr.F[k] = R(0.0); fr.dtF[k] = R(0.0); }
    fr.omega = cf.time_limiter ? lines[(size_t)(t + 2) * line_stride + f].tl_alpha : R(1.0);
    if (!want_flux) return fr;
    FluxParams P;
    P.gamma = cf.gamma; P.K = C.K; P.C1 = cf.C1; P.C2 = cf.C2; P.dt = dt; P.tau_reading = cf.tau_reading;
    for (int m = 0; m < 2; ++m) {
        const GPSide<R>& l = sides[0];
        const GPSide<R>& r = sides[1];
        R Fl[4], dFl[4];
        if (cf.flux == 0) gks_point(P, l.W[m], l.Wn[m], l.Wt[m], r.W[m], r.Wn[m], r.Wt[m], Fl, dFl);
        else lf_point(cf.gamma, l.W[m], l.Wn[m], l.Wt[m], r.W[m], r.Wn[m], r.Wt[m], Fl, dFl);
        // rotate back to the global frame: F = T^{-1} F~
        R Fg[4], dFg[4];
        if (d.dir == 0) { for (int k = 0; k < 4; ++k) { Fg[k] = Fl[k]; dFg[k] = dFl[k]; } }
        else {
            Fg[0] = Fl[0]; Fg[1] = -Fl[2]; Fg[2] = Fl[1]; Fg[3] = Fl[3];
            dFg[0] = dFl[0]; dFg[1] = -dFl[2]; dFg[2] = dFl[1]; dFg[3] = dFl[3];
        }
        // two-point Gauss quadrature, A_1 = A_2 = 1/2
        for (int k = 0; k < 4; ++k) { fr.F[k] = fr.F[k] + 0.5 * Fg[k]; fr.dtF[k] = fr.dtF[k] + 0.5 * dFg[k]; }
    }
    return fr;
}

// One stage operator (Eq. 2 with Gauss quadrature): L, dL/dt, limited dL/dt, and the DF factor
// alpha_ij = prod over the 8 Gauss points of the cell (Sect. 3.2).  F must have ghosts filled.
template <class R>
struct StageOut { std::vector<R> L[4], dtL[4], dtLt[4]; std::vector<R> alpha_next; Counters cnt;
                  std::vector<FaceRec<R>> faces[2]; std::vector<LineRec<R>> lines[2];
                  std::vector<GPSide<R>> sides[2]; };

template <class R>
static void stage_operator(const Ctx& C, const Field<R>& F, double dt, bool want_flux, StageOut<R>& out,
                           bool keep_faces = false) {
    const int nx = C.cfg.nx, ny = C.cfg.ny;
    std::vector<FaceRec<R>> faces[2];
    Counters total;
    for (int dir = 0; dir < 2; ++dir) {
        Dir d = make_dir(C, dir);
        const int nf = d.nn + 1, nl = d.nt + 4;
        std::vector<LineRec<R>> lines((size_t)nf * nl);
        long dfn = 0;
        #pragma omp parallel for schedule(static) reduction(+:dfn) if(Parallel<R>::ok)
        for (int tl = 0; tl < nl; ++tl)
            for (int f = 0; f < nf; ++f) {
                lines[(size_t)tl * nf + f] = normal_line(C, F, d, f, tl - 2);
                dfn += (lines[(size_t)tl * nf + f].dfL[0] ? 1 : 0) + (lines[(size_t)tl * nf + f].dfR[0] ? 1 : 0);
            }
        total.df_n += dfn;
        faces[dir].resize((size_t)nf * d.nt);
        if (keep_faces) out.sides[dir].resize((size_t)nf * d.nt * 2);
        long fb = 0, dft = 0;
        #pragma omp parallel for schedule(static) reduction(+:fb,dft) if(Parallel<R>::ok)
        for (int t = 0; t < d.nt; ++t)
            for (int f = 0; f < nf; ++f) {
                Counters c;
                GPSide<R>* so = keep_faces ? &out.sides[dir][((size_t)t * nf + f) * 2] : nullptr;
                FaceRec<R> fr = face_flux(C, F, d, f, t, lines, nf, dt, want_flux, c, so);
                fb += fr.nfallback;
                dft += c.df_t;
                faces[dir][(size_t)t * nf + f] = fr;
            }
        total.fallbacks += fb;
        total.df_t += dft;
        if (keep_faces) out.lines[dir] = lines;
    }
    for (int k = 0; k < 4; ++k) { out.L[k].assign((size_t)nx * ny, R(0.0)); out.dtL[k].assign((size_t)nx * ny, R(0.0)); out.dtLt[k].assign((size_t)nx * ny, R(0.0)); }
    out.alpha_next.assign((size_t)nx * ny, R(1.0));
    #pragma omp parallel for schedule(static) if(Parallel<R>::ok)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const FaceRec<R>& Wf = faces[0][(size_t)j * (nx + 1) + i];
            const FaceRec<R>& Ef = faces[0][(size_t)j * (nx + 1) + i + 1];
            const FaceRec<R>& Sf = faces[1][(size_t)i * (ny + 1) + j];
            const FaceRec<R>& Nf = faces[1][(size_t)i * (ny + 1) + j + 1];
            size_t c = (size_t)j * nx + i;
            for (int k = 0; k < 4; ++k) {
                out.L[k][c] = -(Ef.F[k] - Wf.F[k]) / C.dx - (Nf.F[k] - Sf.F[k]) / C.dy;
                out.dtL[k][c] = -(Ef.dtF[k] - Wf.dtF[k]) / C.dx - (Nf.dtF[k] - Sf.dtF[k]) / C.dy;
                out.dtLt[k][c] = -(Ef.omega * Ef.dtF[k] - Wf.omega * Wf.dtF[k]) / C.dx
                               - (Nf.omega * Nf.dtF[k] - Sf.omega * Sf.dtF[k]) / C.dy;
            }
            R a = R(1.0);
            const FaceRec<R>* order[4] = {&Wf, &Ef, &Sf, &Nf};
            for (int p = 0; p < 4; ++p) for (int m = 0; m < 2; ++m) a = a * order[p]->alpha_gp[m];
            out.alpha_next[c] = a;
        }
    out.cnt = total;
    if (keep_faces) { out.faces[0] = faces[0]; out.faces[1] = faces[1]; }
}

// Layout helpers: external arrays are SoA [4][ny][nx] (interior cells, x fastest)
template <class R>
static void load_field(const Ctx& C, Field<R>& F, const double* W, const double* alpha) {
    F.init(C.cfg.nx, C.cfg.ny);
    const size_t N = (size_t)C.cfg.nx * C.cfg.ny;
    for (int j = 0; j < C.cfg.ny; ++j)
        for (int i = 0; i < C.cfg.nx; ++i) {
            for (int k = 0; k < 4; ++k) F.w[k][F.id(i, j)] = R(W[k * N + (size_t)j * C.cfg.nx + i]);
            F.alpha[F.id(i, j)] = alpha ? alpha[(size_t)j * C.cfg.nx + i] : 1.0;
        }
}

static bool make_ctx(const oracle_cfg* cfg, Ctx& C) {
    if (!cfg || cfg->nx < 1 || cfg->ny < 1) return false;
    C.cfg = *cfg;
    C.T = make_tables(cfg->dH, cfg->dL);
    C.dx = (cfg->x1 - cfg->x0) / cfg->nx;
    C.dy = (cfg->y1 - cfg->y0) / cfg->ny;
    C.K = (4.0 - 2.0 * cfg->gamma) / (cfg->gamma - 1.0);      // internal degrees of freedom, 2-D
    // periodic wrap and wall mirror both need G interior cells to copy from (outflow copies one)
    if ((cfg->bc[0] != 1 || cfg->bc[1] != 1) && cfg->nx < G) return false;
    if ((cfg->bc[2] != 1 || cfg->bc[3] != 1) && cfg->ny < G) return false;
    return true;
}

// Algorithm 1, "calculate time increment": reading R-dt
static double cfl_dt(const Ctx& C, const Field<double>& F) {
    double best = std::numeric_limits<double>::infinity();
    for (int j = 0; j < C.cfg.ny; ++j)
        for (int i = 0; i < C.cfg.nx; ++i) {
            double W[4];
            for (int k = 0; k < 4; ++k) W[k] = F.w[k][F.id(i, j)];
            Prim<double> s = prim_of(W, C.cfg.gamma);
            double c = std::sqrt(C.cfg.gamma * s.p / s.rho);
            double v;
            if (C.cfg.dt_rule == 0) v = std::min(C.dx / (std::fabs(s.U) + c), C.dy / (std::fabs(s.V) + c));
            else v = 1.0 / ((std::fabs(s.U) + c) / C.dx + (std::fabs(s.V) + c) / C.dy);
            best = std::min(best, v);
        }
    return C.cfg.cfl * best;
}

static bool check_state(const Ctx& C, const Field<double>& F, int& fi, int& fj) {
    for (int j = 0; j < C.cfg.ny; ++j)
        for (int i = 0; i < C.cfg.nx; ++i) {
            double W[4];
            for (int k = 0; k < 4; ++k) W[k] = F.w[k][F.id(i, j)];
            bool ok = std::isfinite(W[0]) && std::isfinite(W[1]) && std::isfinite(W[2]) && std::isfinite(W[3]) &&
                      physical(W, C.cfg.gamma);
            if (!ok) { fi = i; fj = j; return false; }
        }
    return true;
}

}  // namespace orc

using namespace orc;

extern "C" {

int oracle_abi_version(void) { return 1; }

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

// ---- unit-level entry points (pins) ------------------------------------------------------

// coefficients (in xi) of p0..p3 for Q_{-2..2}: out[k*5 + c]
int oracle_sub_polys(const double* Q, double* out) {
    Tables T = make_tables(0.85, 0.85);
    for (int k = 0; k < 4; ++k) {
        PolyK<double> p = sub_poly(T, k, Q);
        for (int c = 0; c < 5; ++c) out[k * 5 + c] = p.a[c];
    }
    return 0;
}

int oracle_smoothness(const double* Q, double* beta4) {
    Tables T = make_tables(0.85, 0.85);
    for (int k = 0; k < 4; ++k) beta4[k] = smoothness(T, sub_poly(T, k, Q));
    return 0;
}

// 1-D hybrid reconstruction of one component at n <= 2 points xi (cell-centred)
int oracle_recon1d(const double* Q, int n, const double* xi, int use_df, double alpha_cell,
                   double dH, double dL, double eps, double* val, double* slope, double* beta4) {
    if (n < 1 || n > 2) return 1;
    Tables T = make_tables(dH, dL);
    Recon1D<double> r = recon1d(T, Q, n, xi, use_df != 0, alpha_cell, eps);
    for (int e = 0; e < n; ++e) { val[e] = r.val[e]; slope[e] = r.slope[e]; }
    if (beta4) for (int k = 0; k < 4; ++k) beta4[k] = r.beta[k];
    return 0;
}

int oracle_limiter_alpha(const double* beta4, double eps, double* out) { *out = limiter_alpha(beta4, eps); return 0; }

int oracle_char_basis(const double* W, double gamma, double* L16, double* R16) {
    Basis<double> B = char_basis(W, gamma);
    for (int r = 0; r < 4; ++r) for (int k = 0; k < 4; ++k) { L16[r * 4 + k] = B.L[r][k]; R16[r * 4 + k] = B.Rm[r][k]; }
    return 0;
}

int oracle_jacobians(const double* W, double gamma, double* A16, double* B16) {
    double A[4][4], B[4][4];
    euler_jacobians(W, gamma, A, B);
    for (int r = 0; r < 4; ++r) for (int k = 0; k < 4; ++k) { A16[r * 4 + k] = A[r][k]; B16[r * 4 + k] = B[r][k]; }
    return 0;
}

// normalised moments <u^n> (n < 10) of the Maxwellian with (U, V, lambda): half 0 / +1 / -1
int oracle_moments_u(double U, double V, double lam, int half, double K, double* mu10) {
    Prim<double> s; s.rho = 1.0; s.U = U; s.V = V; s.lam = lam; s.p = 0.5 / lam;
    Moments<double> m = moments(s, half, K);
    for (int n = 0; n < 10; ++n) mu10[n] = m.u[n];
    return 0;
}

int oracle_slope_solve(const double* W, double gamma, const double* b, double* a) {
    Prim<double> s = prim_of(W, gamma);
    double K = (4.0 - 2.0 * gamma) / (gamma - 1.0);
    slope_solve(moments(s, 0, K), b, a);
    return 0;
}

// <P psi> for P = a1 + a2 u + a3 v + a4 (u^2+v^2+xi^2)/2 times u^i v^j (full moments of W's Maxwellian)
int oracle_avg_psi(const double* W, double gamma, const double* a, int i, int j, double* out) {
    Prim<double> s = prim_of(W, gamma);
    double K = (4.0 - 2.0 * gamma) / (gamma - 1.0);
    avg_psi(poly_shift(poly_from_coeffs(a), i, j), moments(s, 0, K), out);
    return 0;
}

int oracle_gks_point(double gamma, double C1, double C2, double dt, int tau_reading,
                     const double* WL, const double* WLx, const double* WLy,
                     const double* WR, const double* WRx, const double* WRy, double* F, double* dtF) {
    FluxParams P;
    P.gamma = gamma; P.K = (4.0 - 2.0 * gamma) / (gamma - 1.0); P.C1 = C1; P.C2 = C2; P.dt = dt; P.tau_reading = tau_reading;
    gks_point(P, WL, WLx, WLy, WR, WRx, WRy, F, dtF);
    return 0;
}

int oracle_lf_point(double gamma, const double* WL, const double* WLx, const double* WLy,
                    const double* WR, const double* WRx, const double* WRy, double* F, double* dtF) {
    lf_point(gamma, WL, WLx, WLy, WR, WRx, WRy, F, dtF);
    return 0;
}

int oracle_df_alpha_point(double gamma, const double* WL, const double* WR, double* out) {
    *out = df_alpha_point(WL, WR, gamma);
    return 0;
}

int oracle_time_integrals(double T, double tau, double delta, double* g6) {
    Gammas<double> g = time_integrals(T, tau, delta);
    g6[0] = g.gc; g6[1] = g.ac; g6[2] = g.Ac; g6[3] = g.glr; g6[4] = g.alr; g6[5] = g.Alr;
    return 0;
}

// ---- scheme-level entry points -----------------------------------------------------------

int oracle_fill_ghosts(const oracle_cfg* cfg, const double* W, const double* alpha, double* Wg, double* alphag) {
    Ctx C;
    if (!make_ctx(cfg, C)) return 1;
    Field<double> F;
    load_field(C, F, W, alpha);
    fill_ghosts(C, F, true);
    const size_t NG = (size_t)F.NX * F.NY;
    for (int k = 0; k < 4; ++k) std::memcpy(Wg + k * NG, F.w[k].data(), NG * sizeof(double));
    if (alphag) std::memcpy(alphag, F.alpha.data(), NG * sizeof(double));
    return 0;
}

int oracle_cfl_dt(const oracle_cfg* cfg, const double* W, double* dt) {
    Ctx C;
    if (!make_ctx(cfg, C)) return 1;
    Field<double> F;
    load_field(C, F, W, nullptr);
    *dt = cfl_dt(C, F);
    return 0;
}

// One stage operator at (W, alpha) with ghosts filled by the configured boundary conditions.
// Outputs [4][ny][nx]: L, dL/dt, limited dL/dt; alpha_next [ny][nx]; any output may be NULL.
int oracle_residual(const oracle_cfg* cfg, const double* W, const double* alpha, double dt,
                    double* L, double* dtL, double* dtLt, double* alpha_next, oracle_stats* st) {
    Ctx C;
    if (!make_ctx(cfg, C)) return 1;
    Field<double> F;
    load_field(C, F, W, alpha);
    fill_ghosts(C, F, true);
    StageOut<double> o;
    stage_operator(C, F, dt, true, o);
    const size_t N = (size_t)cfg->nx * cfg->ny;
    for (int k = 0; k < 4; ++k) {
        if (L) std::memcpy(L + k * N, o.L[k].data(), N * sizeof(double));
        if (dtL) std::memcpy(dtL + k * N, o.dtL[k].data(), N * sizeof(double));
        if (dtLt) std::memcpy(dtLt + k * N, o.dtLt[k].data(), N * sizeof(double));
    }
    if (alpha_next) std::memcpy(alpha_next, o.alpha_next.data(), N * sizeof(double));
    if (st) { st->fallbacks = o.cnt.fallbacks; st->df_normal = o.cnt.df_n; st->df_tangential = o.cnt.df_t; st->fail_step = -1; }
    return 0;
}

// Per-face intermediates of one stage (for kernel-by-kernel comparison).  dir 0: x-faces
// [ny][nx+1], dir 1: y-faces [nx][ny+1] (face index fastest).  Per face: F[4], dtF[4], omega,
// alpha_gp[2], then Gauss-point states side(L,R) x m(1,2) x {W, Wn, Wt}[4] in the local frame.
// Line records: [nt+4][nf] x {WL, WLn, WR, WRn}[4] + limiter alpha (17 doubles).
int oracle_face_records(const oracle_cfg* cfg, const double* W, const double* alpha, double dt, int dir,
                        double* face_out /* nfaces*59 */, double* line_out /* nlines*17, may be NULL */) {
    Ctx C;
    if (!make_ctx(cfg, C)) return 1;
    Field<double> F;
    load_field(C, F, W, alpha);
    fill_ghosts(C, F, true);
    StageOut<double> o;
    stage_operator(C, F, dt, true, o, true);
    const std::vector<FaceRec<double>>& fr = o.faces[dir];
    for (size_t n = 0; n < fr.size(); ++n) {
        double* p = face_out + n * 59;
        for (int k = 0; k < 4; ++k) { p[k] = fr[n].F[k]; p[4 + k] = fr[n].dtF[k]; }
        p[8] = fr[n].omega; p[9] = fr[n].alpha_gp[0]; p[10] = fr[n].alpha_gp[1];
        int q = 11;
        const GPSide<double>* sd = &o.sides[dir][n * 2];
        for (int s = 0; s < 2; ++s) for (int m = 0; m < 2; ++m) {
            for (int k = 0; k < 4; ++k) p[q++] = sd[s].W[m][k];
            for (int k = 0; k < 4; ++k) p[q++] = sd[s].Wn[m][k];
            for (int k = 0; k < 4; ++k) p[q++] = sd[s].Wt[m][k];
        }
    }
    if (line_out) {
        const std::vector<LineRec<double>>& lr = o.lines[dir];
        for (size_t n = 0; n < lr.size(); ++n) {
            double* p = line_out + n * 17;
            for (int k = 0; k < 4; ++k) { p[k] = lr[n].WL[k]; p[4 + k] = lr[n].WLn[k]; p[8 + k] = lr[n].WR[k]; p[12 + k] = lr[n].WRn[k]; }
            p[16] = lr[n].tl_alpha;
        }
    }
    return 0;
}

// Vector-Jacobian product of the stage operator by reverse-mode differentiation of the same code:
// W_bar = (dL/dW)^T L_bar + (d dtL/dW)^T dtL_bar + (d dtLt/dW)^T dtLt_bar, with alpha, dt and every
// branch decision fixed by the forward pass (any of the three bars may be NULL).
int oracle_residual_vjp(const oracle_cfg* cfg, const double* W, const double* alpha, double dt,
                        const double* L_bar, const double* dtL_bar, const double* dtLt_bar, double* W_bar) {
    Ctx C;
    if (!make_ctx(cfg, C)) return 1;
    ad::Tape tape;
    ad::g_tape = &tape;
    const int nx = cfg->nx, ny = cfg->ny;
    const size_t N = (size_t)nx * ny;
    Field<ad::Var> F;
    F.init(nx, ny);
    std::vector<int> leaf((size_t)4 * N);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            for (int k = 0; k < 4; ++k) {
                ad::Var x = ad::Var::leaf(W[k * N + (size_t)j * nx + i]);
                F.w[k][F.id(i, j)] = x;
                leaf[k * N + (size_t)j * nx + i] = x.id;
            }
            F.alpha[F.id(i, j)] = alpha[(size_t)j * nx + i];
        }
    fill_ghosts(C, F, true);
    StageOut<ad::Var> o;
    stage_operator(C, F, dt, true, o);
    std::vector<double> adj(tape.pa.size(), 0.0);
    for (int k = 0; k < 4; ++k)
        for (size_t c = 0; c < N; ++c) {
            if (L_bar && o.L[k][c].id >= 0) adj[o.L[k][c].id] += L_bar[k * N + c];
            if (dtL_bar && o.dtL[k][c].id >= 0) adj[o.dtL[k][c].id] += dtL_bar[k * N + c];
            if (dtLt_bar && o.dtLt[k][c].id >= 0) adj[o.dtLt[k][c].id] += dtLt_bar[k * N + c];
        }
    for (long n = (long)tape.pa.size() - 1; n >= 0; --n) {
        const double g = adj[n];
        if (g == 0.0) continue;
        if (tape.pa[n] >= 0) adj[tape.pa[n]] += tape.da[n] * g;
        if (tape.pb[n] >= 0) adj[tape.pb[n]] += tape.db[n] * g;
    }
    for (size_t q = 0; q < 4 * N; ++q) W_bar[q] = adj[leaf[q]];
    ad::g_tape = nullptr;
    return 0;
}

// alpha^0: product of the Gauss-point DF factors of a reconstruction of W with alpha = 1 (R-alpha)
int oracle_alpha0(const oracle_cfg* cfg, const double* W, double* alpha_out) {
    Ctx C;
    if (!make_ctx(cfg, C)) return 1;
    Field<double> F;
    load_field(C, F, W, nullptr);
    fill_ghosts(C, F, true);
    StageOut<double> o;
    stage_operator(C, F, 1.0, false, o);
    std::memcpy(alpha_out, o.alpha_next.data(), (size_t)cfg->nx * cfg->ny * sizeof(double));
    return 0;
}

// Advance up to nsteps steps in place (W [4][ny][nx], alpha [ny][nx], *t).  dt_fixed > 0 fixes dt,
// otherwise R-dt.  t_end > 0 clips the last step and stops there.  dts_out (nsteps) may be NULL.
// Returns 0, or 5 on a positivity failure (W, alpha, t left at the last good step).
int oracle_run(const oracle_cfg* cfg, double* W, double* alpha, double* t, int nsteps, double dt_fixed,
               double t_end, double* dts_out, int* steps_done, oracle_stats* st) {
    Ctx C;
    if (!make_ctx(cfg, C)) return 1;
    const int nx = cfg->nx, ny = cfg->ny;
    const size_t N = (size_t)nx * ny;
    Field<double> Fn;
    load_field(C, Fn, W, alpha);
    oracle_stats local{0, 0, 0, -1, -1, -1};
    int done = 0, rc = 0;
    for (int s = 0; s < nsteps; ++s) {
        if (t_end > 0.0 && *t >= t_end) break;
        fill_ghosts(C, Fn, true);
        double dt = (dt_fixed > 0.0) ? dt_fixed : cfl_dt(C, Fn);
        bool clipped = false;
        // last step: clip to t_end; a remainder below 1e-12 relative is absorbed into this step
        if (t_end > 0.0 && *t + dt >= t_end - 1e-12 * std::fabs(t_end)) { dt = t_end - *t; clipped = true; }
        Field<double> Fs = Fn, Fnext = Fn;
        std::vector<double> a_next;
        bool fail = false;
        int fi = -1, fj = -1;
        if (cfg->time_scheme == 0) {
            // Eq. 24 with the time limiter: stage 1 at W^n, stage 2 at W*
            StageOut<double> o1;
            stage_operator(C, Fn, dt, true, o1);
            for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) {
                size_t c = (size_t)j * nx + i, g = Fn.id(i, j);
                for (int k = 0; k < 4; ++k)
                    Fs.w[k][g] = Fn.w[k][g] + 0.5 * dt * o1.L[k][c] + 0.125 * dt * dt * o1.dtL[k][c];
            }
            local.fallbacks += o1.cnt.fallbacks; local.df_normal += o1.cnt.df_n; local.df_tangential += o1.cnt.df_t;
            if (!check_state(C, Fs, fi, fj)) fail = true;
            if (!fail) {
                fill_ghosts(C, Fs, true);
                StageOut<double> o2;
                stage_operator(C, Fs, dt, true, o2);
                for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) {
                    size_t c = (size_t)j * nx + i, g = Fn.id(i, j);
                    for (int k = 0; k < 4; ++k)
                        Fnext.w[k][g] = Fn.w[k][g] + dt * o1.L[k][c] + 0.5 * dt * dt * o1.dtL[k][c]
                                      - (1.0 / 3.0) * dt * dt * o1.dtLt[k][c] + (1.0 / 3.0) * dt * dt * o2.dtLt[k][c];
                }
                a_next = o2.alpha_next;
                local.fallbacks += o2.cnt.fallbacks; local.df_normal += o2.cnt.df_n; local.df_tangential += o2.cnt.df_t;
                if (!check_state(C, Fnext, fi, fj)) fail = true;
            }
        } else {
            // SSP-RK3 (Sect. 2.3)
            StageOut<double> o1, o2, o3;
            stage_operator(C, Fn, dt, true, o1);
            Field<double> F1 = Fn, F2 = Fn;
            for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) {
                size_t c = (size_t)j * nx + i, g = Fn.id(i, j);
                for (int k = 0; k < 4; ++k) F1.w[k][g] = Fn.w[k][g] + dt * o1.L[k][c];
            }
            if (!check_state(C, F1, fi, fj)) fail = true;
            if (!fail) {
                fill_ghosts(C, F1, true);
                stage_operator(C, F1, dt, true, o2);
                for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) {
                    size_t c = (size_t)j * nx + i, g = Fn.id(i, j);
                    for (int k = 0; k < 4; ++k) F2.w[k][g] = 0.75 * Fn.w[k][g] + 0.25 * F1.w[k][g] + 0.25 * dt * o2.L[k][c];
                }
                if (!check_state(C, F2, fi, fj)) fail = true;
            }
            if (!fail) {
                fill_ghosts(C, F2, true);
                stage_operator(C, F2, dt, true, o3);
                for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) {
                    size_t c = (size_t)j * nx + i, g = Fn.id(i, j);
                    for (int k = 0; k < 4; ++k)
                        Fnext.w[k][g] = (1.0 / 3.0) * Fn.w[k][g] + (2.0 / 3.0) * F2.w[k][g] + (2.0 / 3.0) * dt * o3.L[k][c];
                }
                a_next = o3.alpha_next;
                if (!check_state(C, Fnext, fi, fj)) fail = true;
            }
            const Counters* cs[3] = {&o1.cnt, &o2.cnt, &o3.cnt};
            for (const Counters* c : cs) { local.fallbacks += c->fallbacks; local.df_normal += c->df_n; local.df_tangential += c->df_t; }
        }
        // alpha_source = 1: Algorithm 1's "update DF" read as one more reconstruction after the
        // stages, of W^{n+1} itself, its DF branches (Eq. 34) decided by alpha^n; alpha^{n+1} is
        // the product of that reconstruction's Gauss-point factors (Sect. 3.2).  Its branches and
        // fallbacks are not counted: no flux comes from it.
        if (!fail && cfg->alpha_source == 1) {
            Field<double> Fp = Fnext;                  // Fnext kept alpha^n from its copy of Fn
            fill_ghosts(C, Fp, true);
            StageOut<double> op;
            stage_operator(C, Fp, dt, false, op);
            a_next = op.alpha_next;
        }
        if (fail) { local.fail_step = done; local.fail_i = fi; local.fail_j = fj; rc = 5; break; }
        for (int k = 0; k < 4; ++k) Fn.w[k] = Fnext.w[k];
        for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) Fn.alpha[Fn.id(i, j)] = a_next[(size_t)j * nx + i];
        *t = clipped ? t_end : *t + dt;
        if (dts_out) dts_out[done] = dt;
        ++done;
    }
    for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) {
        for (int k = 0; k < 4; ++k) W[k * N + (size_t)j * nx + i] = Fn.w[k][Fn.id(i, j)];
        alpha[(size_t)j * nx + i] = Fn.alpha[Fn.id(i, j)];
    }
    if (steps_done) *steps_done = done;
    if (st) *st = local;
    return rc;
}

}  // extern "C"
