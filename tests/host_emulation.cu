// Host build of the CUDA path's per-thread bodies: the stage operator (ghost fill, both sweeps,
// residual) and its reverse sweep, run one body invocation at a time on the CPU exactly as the
// kernels call them.  Reads a problem from argv[1] (the In header, then W, alpha, L_bar, dtL_bar,
// dtLt_bar as dense doubles) and writes L, dL/dt, limited dL/dt, W_bar, and W_bar once more with the
// reverse sweep reading the tapes of the forward intermediates, to argv[2].  Used by
// tests/test_host_emulation.py, which compares the results with the oracle.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <vector>
#include "dfgks_adjoint.cu"
using namespace dfk;

static void rd(void* p, size_t size, size_t n, FILE* f) {
    if (fread(p, size, n, f) != n) { fprintf(stderr, "short input\n"); exit(2); }
}

struct In {
    int nx, ny, bc[4], flux, time_limiter, tau_reading, gp_fallback;
    double x0, x1, y0, y1, gamma, alpha_thres, dH, dL, eps, C1, C2, dt;
};

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    In in;
    rd(&in, sizeof(In), 1, f);
    const long long N = (long long)in.nx * in.ny;
    std::vector<double> Wd(4 * N), ad(N), Lb(4 * N), dLb(4 * N), dLtb(4 * N);
    rd(Wd.data(), 8, 4 * N, f); rd(ad.data(), 8, N, f);
    rd(Lb.data(), 8, 4 * N, f); rd(dLb.data(), 8, 4 * N, f); rd(dLtb.data(), 8, 4 * N, f);
    fclose(f);
    Mesh m;
    m.nx = in.nx; m.ny = in.ny; m.P = (in.nx + 2 * G + 3) & ~3; m.NYg = in.ny + 2 * G; m.plane = (long long)m.P * m.NYg;
    m.dx = (in.x1 - in.x0) / in.nx; m.dy = (in.y1 - in.y0) / in.ny;
    m.rdx = 1.0 / m.dx; m.rdy = 1.0 / m.dy;
    for (int q = 0; q < 4; ++q) m.bc[q] = in.bc[q];
    m.dt_rule = 0; m.gi0 = 0; m.gj0 = 0; m.gnx = in.nx;
    SchemeConsts S;
    S.gamma = in.gamma; S.gm1 = in.gamma - 1.0; S.K = (4.0 - 2.0 * in.gamma) / (in.gamma - 1.0); S.inv_K2 = 1.0 / (S.K + 2.0);
    S.r2g = sqrt(2.0 / S.gamma);
    S.d[3] = in.dH; S.d[0] = (1.0 - in.dH) * (1.0 - in.dL) / 2.0; S.d[1] = (1.0 - in.dH) * in.dL; S.d[2] = S.d[0];
    S.inv_d3 = 1.0 / in.dH; S.eps = in.eps; S.alpha_thres = in.alpha_thres; S.C1 = in.C1; S.C2 = in.C2;
    S.time_limiter = in.time_limiter; S.tau_reading = in.tau_reading; S.gp_fallback = in.gp_fallback;
    S.df_states = 0;
    const long long nfx = (long long)(m.nx + 1) * m.ny, nfy = (long long)(m.ny + 1) * m.nx;
    const long long nlx = (long long)(m.nx + 1) * (m.ny + 4), nly = (long long)(m.ny + 1) * (m.nx + 4);
    SweepBuffers B;
    B.line_stride = (std::max(nlx, nly) + 3) & ~3LL;
    B.gp_stride = (2 * std::max(nfx, nfy) + 3) & ~3LL;
    B.flux_stride[0] = (2 * nfx + 3) & ~3LL; B.flux_stride[1] = (2 * nfy + 3) & ~3LL;
    std::vector<double> Wg(4 * m.plane, 1.0), Ag(m.plane, 1.0), lines(LR_COUNT * B.line_stride, -7.0),
        gp(GP_COUNT * B.gp_stride, -7.0), fr0(FR_COUNT * B.flux_stride[0], -7.0), fr1(FR_COUNT * B.flux_stride[1], -7.0),
        lb(LR_COUNT * B.line_stride), gb(GP_COUNT * B.gp_stride), Wbg(4 * m.plane, 0.0), out(4 * N, 0.0),
        L(4 * N), dL(4 * N), dLt(4 * N);
    B.lines = lines.data(); B.gp = gp.data(); B.flux[0] = fr0.data(); B.flux[1] = fr1.data();
    for (int k = 0; k < 4; ++k) for (int j = 0; j < m.ny; ++j) for (int i = 0; i < m.nx; ++i)
        Wg[k * m.plane + gid(m, i, j)] = Wd[k * N + (long long)j * m.nx + i];
    for (int j = 0; j < m.ny; ++j) for (int i = 0; i < m.nx; ++i) Ag[gid(m, i, j)] = ad[(long long)j * m.nx + i];
    for (int j = 0; j < m.ny; ++j) for (int gc = 0; gc < 2 * G; ++gc) ghost_x_body(m, Wg.data(), Ag.data(), gc, j);
    for (int gr = 0; gr < 2 * G; ++gr) for (int i = -G; i < m.nx + G; ++i) ghost_y_body(m, Wg.data(), Ag.data(), i, gr);
    AdjointArgs a = {Lb.data(), dLb.data(), dLtb.data()};
    // every thread of the kernels' 1-D grids, padded tail included (the bodies must reject it)
    auto grid = [&](int lx, int ly, auto body) {
        const long long n = (long long)sweep_blocks(lx, ly) * 128;
        for (long long i = 0; i < n; ++i) body((int)(i % lx), (int)(i / lx));
    };
    auto sweep = [&](auto dirc) {
        constexpr int DIR = decltype(dirc)::value;
        const int lx = lines_lx<DIR>(m), ly = lines_ly<DIR>(m), fx = faces_lx<DIR>(m), fy = faces_ly<DIR>(m);
        grid(lx, ly, [&](int x, int y) {
            if (B.ltape) lines_body<DIR, true>(m, S, Wg.data(), Ag.data(), B.lines, B.line_stride, x, y, B.ltape);
            else lines_body<DIR>(m, S, Wg.data(), Ag.data(), B.lines, B.line_stride, x, y);
        });
        for (int z = 0; z < 2; ++z) grid(fx, fy, [&](int x, int y) {
            int nfb;
            if (B.ftape) faces_body<DIR, true>(m, S, Wg.data(), Ag.data(), B.lines, B.line_stride, B.gp, B.gp_stride, x, y, z, nfb, B.ftape);
            else faces_body<DIR>(m, S, Wg.data(), Ag.data(), B.lines, B.line_stride, B.gp, B.gp_stride, x, y, z, nfb);
        });
        for (int z = 0; z < 2; ++z) grid(fx, fy, [&](int x, int y) {
            if (in.flux == 0 && B.tape[DIR]) flux_body<DIR, 0, false, true>(m, S, B.lines, B.line_stride, B.gp, B.gp_stride, B.flux[DIR], B.flux_stride[DIR], in.dt, x, y, z, B.tape[DIR]);
            else if (in.flux == 0) flux_body<DIR, 0, false>(m, S, B.lines, B.line_stride, B.gp, B.gp_stride, B.flux[DIR], B.flux_stride[DIR], in.dt, x, y, z);
            else flux_body<DIR, 1, false>(m, S, B.lines, B.line_stride, B.gp, B.gp_stride, B.flux[DIR], B.flux_stride[DIR], in.dt, x, y, z);
        });
    };
    auto reverse = [&](auto dirc) {
        constexpr int DIR = decltype(dirc)::value;
        const int lx = lines_lx<DIR>(m), ly = lines_ly<DIR>(m), fx = faces_lx<DIR>(m), fy = faces_ly<DIR>(m);
        std::fill(lb.begin(), lb.end(), 0.0);
        std::fill(gb.begin(), gb.end(), -9.0);
        for (int z = 0; z < 2; ++z) grid(fx, fy, [&](int x, int y) {
            if (in.flux == 0 && B.tape[DIR]) ka_flux_body<DIR, 0, true>(m, S, a, B.gp, B.gp_stride, B.flux[DIR], B.flux_stride[DIR], in.dt, lb.data(), B.line_stride, gb.data(), x, y, z, B.tape[DIR]);
            else if (in.flux == 0) ka_flux_body<DIR, 0>(m, S, a, B.gp, B.gp_stride, B.flux[DIR], B.flux_stride[DIR], in.dt, lb.data(), B.line_stride, gb.data(), x, y, z);
            else ka_flux_body<DIR, 1>(m, S, a, B.gp, B.gp_stride, B.flux[DIR], B.flux_stride[DIR], in.dt, lb.data(), B.line_stride, gb.data(), x, y, z);
        });
        for (int z = 0; z < 2; ++z) grid(fx, fy, [&](int x, int y) {
            if (B.ftape) ka_faces_body<DIR, true>(m, S, Ag.data(), B.lines, B.line_stride, B.gp, gb.data(), B.gp_stride, lb.data(), Wbg.data(), x, y, z, B.ftape);
            else ka_faces_body<DIR>(m, S, Ag.data(), B.lines, B.line_stride, B.gp, gb.data(), B.gp_stride, lb.data(), Wbg.data(), x, y, z);
        });
        grid(lx, ly, [&](int x, int y) {
            if (B.ltape) ka_lines_body<DIR, true>(m, S, Wg.data(), Ag.data(), B.lines, lb.data(), B.line_stride, Wbg.data(), x, y, B.ltape);
            else ka_lines_body<DIR>(m, S, Wg.data(), Ag.data(), B.lines, lb.data(), B.line_stride, Wbg.data(), x, y);
        });
    };
    // forward residual (both directions), for a sanity check of the emulation
    sweep(std::integral_constant<int, 0>());
    sweep(std::integral_constant<int, 1>());
    UpdateArgs ua{};
    ua.L = L.data(); ua.dtL = dL.data(); ua.dtLt = dLt.data();
    for (int j = 0; j < m.ny; ++j) for (int i = 0; i < m.nx; ++i)
        update_body<UM_RESIDUAL>(m, S, ua, B.flux[0], B.flux_stride[0], B.flux[1], B.flux_stride[1], 0.0, nullptr, i, j);
    // reverse
    auto adjoint = [&](std::vector<double>& res) {
        std::fill(Wbg.begin(), Wbg.end(), 0.0);
        std::fill(res.begin(), res.end(), 0.0);
        sweep(std::integral_constant<int, 0>()); reverse(std::integral_constant<int, 0>());
        sweep(std::integral_constant<int, 1>()); reverse(std::integral_constant<int, 1>());
        for (int i = -G; i < m.nx + G; ++i) ka_fold_y_body(m, Wbg.data(), i);
        for (int j = 0; j < m.ny; ++j) ka_fold_x_body(m, Wbg.data(), j);
        for (int j = 0; j < m.ny; ++j) for (int i = 0; i < m.nx; ++i) ka_accumulate_body(m, Wbg.data(), res.data(), i, j);
    };
    adjoint(out);
    // the same with the reconstructions' and the GKS flux's intermediates taped by the forward sweep
    std::vector<double> tape0(TG_COUNT * B.flux_stride[0], -7.0), tape1(TG_COUNT * B.flux_stride[1], -7.0), out2(4 * N, 0.0);
    std::vector<double> ltape(8 * AT_COUNT * B.line_stride, -7.0), ftape(4 * AT_COUNT * B.gp_stride, -7.0);
    B.tape[0] = tape0.data(); B.tape[1] = tape1.data();
    B.ltape = ltape.data(); B.ftape = ftape.data();
    adjoint(out2);
    f = fopen(argv[2], "wb");
    if (!f) return 2;
    fwrite(L.data(), 8, 4 * N, f); fwrite(dL.data(), 8, 4 * N, f); fwrite(dLt.data(), 8, 4 * N, f); fwrite(out.data(), 8, 4 * N, f); fwrite(out2.data(), 8, 4 * N, f);
    fclose(f);
    return 0;
}
