// Host-side check of the hand-written reverse products in dfgks_adjoint.cuh: each is compared with
// central finite differences of its forward counterpart in dfgks_device.cuh (the same source the
// GPU kernels compile), on random inputs.  Prints one line per block and exits non-zero on failure.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>

#include "dfgks_adjoint.cuh"

using namespace dfk;

static std::mt19937_64 rng(12345);
static double U(double a, double b) { return std::uniform_real_distribution<double>(a, b)(rng); }
static int failures = 0;

static void report(const char* name, double err, double tol) {
    bool ok = err <= tol;
    if (!ok) ++failures;
    std::printf("%-28s max rel err %.3e  %s\n", name, err, ok ? "ok" : "FAIL");
}

static SchemeConsts consts(int tau_reading) {
    SchemeConsts S{};
    S.gamma = 1.4; S.gm1 = 0.4; S.K = 3.0; S.inv_K2 = 0.2; S.r2g = sqrt(2.0 / 1.4);
    S.d[3] = 0.85; S.d[0] = 0.15 * 0.15 / 2; S.d[1] = 0.15 * 0.85; S.d[2] = S.d[0]; S.inv_d3 = 1.0 / 0.85;
    S.eps = 1e-6; S.alpha_thres = 0.5; S.C1 = 0.01; S.C2 = 5.0;
    S.time_limiter = 1; S.tau_reading = tau_reading; S.gp_fallback = 1; S.df_states = 0;
    return S;
}

static void state(double W[4]) {
    double rho = U(0.3, 2.0), u = U(-1, 1), v = U(-1, 1), p = U(0.2, 2.0);
    W[0] = rho; W[1] = rho * u; W[2] = rho * v; W[3] = p / 0.4 + 0.5 * rho * (u * u + v * v);
}

// generic check: f maps x[n] -> y[m]; vjp gives xb from yb
template <class F, class V>
static double check(int n, int m, double* x, F f, V vjp) {
    double yb[64], xb[64], y1[64], y2[64];
    for (int i = 0; i < m; ++i) yb[i] = U(-1, 1);
    for (int i = 0; i < n; ++i) xb[i] = 0.0;
    vjp(x, yb, xb);
    double worst = 0.0, scale = 1e-30;
    for (int i = 0; i < n; ++i) scale = std::fmax(scale, std::fabs(xb[i]));
    for (int i = 0; i < n; ++i) {
        double h = 1e-6 * std::fmax(1.0, std::fabs(x[i])), keep = x[i];
        x[i] = keep + h; f(x, y1);
        x[i] = keep - h; f(x, y2);
        x[i] = keep;
        double fd = 0.0;
        for (int k = 0; k < m; ++k) fd += yb[k] * (y1[k] - y2[k]) / (2 * h);
        worst = std::fmax(worst, std::fabs(fd - xb[i]) / std::fmax(std::fabs(fd), 1e-3 * scale));
    }
    return worst;
}

int main() {
    const SchemeConsts S = consts(0);
    double worst;
    // make_basis: (Wl, Wr) -> 8 basis scalars
    worst = 0;
    for (int t = 0; t < 5; ++t) {
        double x[8];
        state(x); state(x + 4);
        auto f = [&](const double* x, double* y) {
            CharBasis B = make_basis(x, x + 4, S);
            double v[8] = {B.u, B.v, B.c, B.ic, B.H, B.b1, B.b2, B.q2};
            for (int i = 0; i < 8; ++i) y[i] = v[i];
        };
        auto g = [&](const double* x, const double* yb, double* xb) {
            BasisBar Bb = {yb[0], yb[1], yb[2], yb[3], yb[4], yb[5], yb[6], yb[7]};
            make_basis_vjp(x, x + 4, S, Bb, xb, xb + 4);
        };
        worst = std::fmax(worst, check(8, 8, x, f, g));
    }
    report("make_basis", worst, 1e-6);
    // project and back_project as functions of (basis scalars, vector)
    worst = 0;
    double worst2 = 0;
    for (int t = 0; t < 5; ++t) {
        double Wl[4], Wr[4], x[12];
        state(Wl); state(Wr);
        CharBasis B0 = make_basis(Wl, Wr, S);
        double b0[8] = {B0.u, B0.v, B0.c, B0.ic, B0.H, B0.b1, B0.b2, B0.q2};
        for (int i = 0; i < 8; ++i) x[i] = b0[i];
        state(x + 8);
        auto mk = [](const double* x) { CharBasis B; B.u = x[0]; B.v = x[1]; B.c = x[2]; B.ic = x[3]; B.H = x[4]; B.b1 = x[5]; B.b2 = x[6]; B.q2 = x[7]; return B; };
        auto fp = [&](const double* x, double* y) { project(mk(x), x + 8, y); };
        auto gp = [&](const double* x, const double* yb, double* xb) {
            BasisBar Bb; basis_bar_zero(Bb);
            project_vjp(mk(x), x + 8, yb, xb + 8, Bb);
            double v[8] = {Bb.u, Bb.v, Bb.c, Bb.ic, Bb.H, Bb.b1, Bb.b2, Bb.q2};
            for (int i = 0; i < 8; ++i) xb[i] += v[i];
        };
        worst = std::fmax(worst, check(12, 4, x, fp, gp));
        for (int i = 8; i < 12; ++i) x[i] = U(-1, 1);
        auto fb = [&](const double* x, double* y) { back_project(mk(x), x + 8, y); };
        auto gb = [&](const double* x, const double* yb, double* xb) {
            BasisBar Bb; basis_bar_zero(Bb);
            back_project_vjp(mk(x), x + 8, yb, xb + 8, Bb);
            double v[8] = {Bb.u, Bb.v, Bb.c, Bb.ic, Bb.H, Bb.b1, Bb.b2, Bb.q2};
            for (int i = 0; i < 8; ++i) xb[i] += v[i];
        };
        worst2 = std::fmax(worst2, check(12, 4, x, fb, gb));
    }
    report("project", worst, 1e-6);
    report("back_project", worst2, 1e-6);
    // back_project_T + back_project_basis_vjp = back_project_vjp
    {
        double split = 0;
        for (int t = 0; t < 5; ++t) {
            double Wl[4], Wr[4], q[4], wb[4];
            state(Wl); state(Wr);
            CharBasis B = make_basis(Wl, Wr, S);
            for (int i = 0; i < 4; ++i) { q[i] = U(-1, 1); wb[i] = U(-1, 1); }
            double qa[4] = {0, 0, 0, 0}, qc[4] = {0, 0, 0, 0};
            BasisBar A, C; basis_bar_zero(A); basis_bar_zero(C);
            back_project_vjp(B, q, wb, qa, A);
            back_project_T(B, wb, qc);
            back_project_basis_vjp(B, q, wb, C);
            double av[12] = {qa[0], qa[1], qa[2], qa[3], A.u, A.v, A.c, A.ic, A.H, A.b1, A.b2, A.q2};
            double cv[12] = {qc[0], qc[1], qc[2], qc[3], C.u, C.v, C.c, C.ic, C.H, C.b1, C.b2, C.q2};
            for (int i = 0; i < 12; ++i) split = std::fmax(split, std::fabs(av[i] - cv[i]) / std::fmax(std::fabs(av[i]), 1e-12));
        }
        report("back_project split", split, 1e-13);
    }
    // WENO-AO and its evaluations: q[5] -> (edge value, edge slope, gauss values/slopes, limiter)
    worst = 0;
    double worst_tape = 0;
    for (int t = 0; t < 40; ++t) {
        double x[5];
        double amp = (t % 4 == 0) ? 1e-3 : (t % 4 == 1 ? 1.0 : 0.1);
        for (int i = 0; i < 5; ++i) x[i] = U(0.5, 1.5) + amp * U(-1, 1) * (t % 3 == 0 ? (i > 2 ? 5.0 : 0.0) : 1.0);
        auto f = [&](const double* q, double* y) {
            AO o = weno_ao(q, S);
            ao_at_right_edge(o, q[2], y[0], y[1]);
            ao_at_gauss(o, q[2], y + 2, y + 4);
            y[6] = limiter_alpha(o);
        };
        auto g = [&](const double* q, const double* yb, double* qb) {
            double t[AT_COUNT];
            const ArrayTape T{t};
            AO o = weno_ao_t(q, S, T, 0);
            AOBar ob; ao_bar_zero(ob);
            ao_at_right_edge_vjp(yb[0], yb[1], qb[2], ob);
            ao_at_gauss_vjp(yb + 2, yb + 4, qb[2], ob);
            limiter_alpha_vjp(o, yb[6], ob);
            weno_ao_rev(T, 0, S, ob, qb);
        };
        worst = std::fmax(worst, check(5, 7, x, f, g));
        // the outputs rebuilt from the tape are those of weno_ao
        double tt[AT_COUNT];
        const ArrayTape T{tt};
        weno_ao_t(x, S, T, 0);
        AO a = weno_ao(x, S), b = ao_from_tape(T, 0, S);
        // (weno_ao carries the limiter's ratios scaled; compare the limiter weight they give)
        const double av[6] = {a.A1, a.A2, a.c3a3, a.c3a4, limiter_alpha(a), 0.0};
        const double bv[6] = {b.A1, b.A2, b.c3a3, b.c3a4, limiter_alpha(b), 0.0};
        for (int i = 0; i < 6; ++i) worst_tape = std::fmax(worst_tape, std::fabs(av[i] - bv[i]) / std::fmax(std::fabs(av[i]), 1e-300));
    }
    report("weno_ao + evaluations", worst, 1e-5);
    report("weno_ao from its tape", worst_tape, 1e-12);
    // DF quadratic
    worst = 0;
    for (int t = 0; t < 5; ++t) {
        double x[5];
        for (int i = 0; i < 5; ++i) x[i] = U(-1, 1);
        double al = U(0, 1);
        auto f = [&](const double* q, double* y) { df_at_right_edge(q, al, y[0], y[1]); df_at_gauss(q, al, y + 2, y + 4); };
        auto g = [&](const double* q, const double* yb, double* qb) { df_at_right_edge_vjp(al, yb[0], yb[1], qb); df_at_gauss_vjp(al, yb + 2, yb + 4, qb); };
        worst = std::fmax(worst, check(5, 6, x, f, g));
    }
    report("df quadratic", worst, 1e-7);
    // Gauss-point fluxes: 24 inputs -> F, dF
    for (int tr = 0; tr < 2; ++tr) {
        const SchemeConsts St = consts(tr);
        double wg = 0, wl = 0;
        for (int t = 0; t < 6; ++t) {
            double x[24];
            state(x); state(x + 12);
            for (int i = 4; i < 12; ++i) x[i] = 0.3 * U(-1, 1);
            for (int i = 16; i < 24; ++i) x[i] = 0.3 * U(-1, 1);
            const double dt = 0.004;
            auto unpack = [](const double* x, GPState& L, GPState& R) {
                for (int i = 0; i < 4; ++i) { L.W[i] = x[i]; L.Wn[i] = x[4 + i]; L.Wt[i] = x[8 + i]; R.W[i] = x[12 + i]; R.Wn[i] = x[16 + i]; R.Wt[i] = x[20 + i]; }
            };
            auto pack = [](const GPStateBar& Lb, const GPStateBar& Rb, double* xb) {
                for (int i = 0; i < 4; ++i) { xb[i] += Lb.W[i]; xb[4 + i] += Lb.Wn[i]; xb[8 + i] += Lb.Wt[i]; xb[12 + i] += Rb.W[i]; xb[16 + i] += Rb.Wn[i]; xb[20 + i] += Rb.Wt[i]; }
            };
            auto fg = [&](const double* x, double* y) { GPState L, R; unpack(x, L, R); gks_flux(L, R, dt, St, y, y + 4); };
            auto gg = [&](const double* x, const double* yb, double* xb) {
                GPState L, R; unpack(x, L, R);
                GPStateBar Lb = {}, Rb = {};
                gks_flux_vjp(L, R, dt, St, yb, yb + 4, Lb, Rb);
                pack(Lb, Rb, xb);
            };
            wg = std::fmax(wg, check(24, 8, x, fg, gg));
            if (tr == 0) {
                auto fl = [&](const double* x, double* y) { GPState L, R; unpack(x, L, R); lf_flux(L, R, St, y, y + 4); };
                auto gl = [&](const double* x, const double* yb, double* xb) {
                    GPState L, R; unpack(x, L, R);
                    GPStateBar Lb = {}, Rb = {};
                    lf_flux_vjp(L, R, St, yb, yb + 4, Lb, Rb);
                    pack(Lb, Rb, xb);
                };
                wl = std::fmax(wl, check(24, 8, x, fl, gl));
            }
        }
        report(tr ? "gks_flux (tau = tau_n)" : "gks_flux (tau = 0)", wg, 1e-5);
        if (tr == 0) report("lf_flux", wl, 1e-6);
    }
    return failures ? 1 : 0;
}
