// dfgks_internal.h -- structures shared by the host side of the C ABI and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <vector>
#include "dfgks_device.cuh"

namespace dfk {

// Optional per-kernel timing on the handle's stream: a pair of CUDA events around every launch
// of a kernel class, harvested after the stream is synchronised.  Also counts launches.
enum KernelKind { KK_LINES = 0, KK_FACES, KK_FLUX, KK_UPDATE, KK_OTHER, KK_COUNT };

struct KernelTimer {
    bool on = false;
    cudaStream_t stream = nullptr;
    std::vector<cudaEvent_t> ev;       // 2 per slot
    std::vector<int> kind;
    int used = 0;
    double total_ms[KK_COUNT] = {0, 0, 0, 0, 0};
    long long timed[KK_COUNT] = {0, 0, 0, 0, 0};
    long long launches[KK_COUNT] = {0, 0, 0, 0, 0};   // counted whether or not timing is on
    int open_slot = -1;

    void begin(int k) {
        if (!on) return;
        if (used >= (int)kind.size()) harvest_sync();
        open_slot = used++;
        kind[open_slot] = k;
        cudaEventRecord(ev[2 * open_slot], stream);
    }
    void end(int k, int nlaunch) {
        launches[k] += nlaunch;
        if (!on || open_slot < 0) return;
        cudaEventRecord(ev[2 * open_slot + 1], stream);
        open_slot = -1;
    }
    void harvest() {           // call with the stream synchronised
        for (int q = 0; q < used; ++q) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[2 * q], ev[2 * q + 1]) == cudaSuccess) {
                total_ms[kind[q]] += ms;
                timed[kind[q]] += 1;
            }
        }
        used = 0;
    }
    void harvest_sync() { cudaStreamSynchronize(stream); harvest(); }
};

// Ghosted SoA field: component k of cell (i, j), i in [-G, nx+G), j in [-G, ny+G), lives at
// base + k*plane + (j+G)*P + (i+G).  The row pitch P is a multiple of 4 doubles (32 B).
struct Mesh {
    int nx, ny;
    int P;              // row pitch in doubles
    int NYg;            // ny + 2G
    long long plane;    // P * NYg
    double dx, dy;
    double rdx, rdy;    // 1/dx and 1/dy, divided once on the host (the same correctly rounded values)
    int bc[4];          // x-low, x-high, y-low, y-high; BC_EXTERNAL: ghosts written by a halo copy
    int dt_rule;        // CFL bound per cell: 0 per-direction minimum, 1 summed inverse
    int gi0, gj0, gnx;  // a block of a larger mesh: its first cell there and that mesh's nx
                        // (0, 0, nx for a whole mesh); positivity failures report that mesh's index
};

// boundary code of a block side whose ghost layers a neighbouring block's halo copy fills
constexpr int BC_EXTERNAL = 3;

__host__ __device__ __forceinline__ long long gid(const Mesh& m, int i, int j) {
    return (long long)(j + G) * m.P + (i + G);
}

// Device-resident step state (one per handle).  Every kernel of a step returns at once when
// `halt` is set (final time reached or positivity lost), so a queue of launched steps drains
// without work and the state stays at the last good step.
struct DevState {
    double dt;                      // dt of the current step
    double t;                       // physical time
    unsigned long long dtmin_bits;  // CFL minimum of the current step, as the bits of a positive double
    long long step;                 // steps completed since set_ic/set_state
    int halt;                       // 1: skip the remaining kernels
    int err;                        // 0 or DFGKS_ENONPOS
    int clipped;                    // the current step was clipped to t_end
    int par;                        // batched path: which of the two state buffers is current
    long long fail_step;
    unsigned long long fail_key;    // smallest failing linear cell index j*nx + i
    unsigned long long fallbacks, df_normal, df_tangential;
};

// Per-face-line record of the normal reconstruction (Algorithm 1, normal step), SoA planes
// (LR_TLK: which of the face's eight reconstructions set the limiter weight, 2k + side, or -1;
// LR_DFC: the DF factor of the face's two cell averages, written when df_states = 1)
enum LineField { LR_WL = 0, LR_WLN = 4, LR_WR = 8, LR_WRN = 12, LR_TL = 16,
                 LR_U = 17, LR_V, LR_C, LR_IC, LR_H, LR_B1, LR_B2, LR_Q2, LR_TLK, LR_DFC, LR_COUNT };
// Per-(face, side) Gauss-point record of the tangential step: m=1 {W, Wn, Wt}, m=2 {W, Wn, Wt},
// then GP_FB: bit m set if Gauss point m fell back to the cell average
constexpr int GP_FB = 24;
constexpr int GP_COUNT = 25;
// Per-(face, Gauss point) flux record: F[4], dF[4] (global frame), alpha_{p,m}, omega^t
enum FluxField { FR_F = 0, FR_DF = 4, FR_ALPHA = 8, FR_OMEGA = 9, FR_COUNT = 10 };

struct SweepBuffers {
    double* lines;          // LR_COUNT planes of line_stride
    long long line_stride;
    double* gp;             // GP_COUNT planes of gp_stride (2 sides x faces)
    long long gp_stride;
    double* flux[2];        // per direction: FR_COUNT planes of flux_stride[dir] (2 Gauss points x faces)
    long long flux_stride[2];
    // optional, per direction: the GKS flux's forward intermediates (TG_COUNT planes of
    // flux_stride[dir]), written by the forward sweep when set and read by the reverse sweep
    double* tape[2] = {nullptr, nullptr};
    // optional: the WENO-AO intermediates of the face lines' 8 reconstructions (8 x AT_COUNT planes
    // of line_stride, reconstruction 2k + side) and of the face sides' 4 tangential ones (4 x AT_COUNT
    // planes of gp_stride), written by the forward sweep when set and read by the reverse sweep
    double* ltape = nullptr;
    double* ftape = nullptr;
};

enum UpdateMode { UM_RESIDUAL = 0, UM_S2O4_1, UM_S2O4_2, UM_RK_1, UM_RK_2, UM_RK_3, UM_ALPHA };

struct UpdateArgs {
    const double* Win;      // ghosted: the stage's input state (read for W^n / stage states)
    const double* Wn;       // ghosted: W^n (SSP-RK3 combinations)
    double* Wout;           // ghosted output state (stage result)
    double* acc;            // dense [4][ny][nx]: S2O4 accumulator
    double* L; double* dtL; double* dtLt;   // dense outputs (residual mode), may be null
    double* alpha_out;      // ghosted or dense alpha output, may be null
    int alpha_dense;        // 1: alpha_out is dense [ny][nx]
};

struct AdjointArgs { const double* Lb; const double* dtLb; const double* dtLtb; };   // dense, may be null

// ---- launchers (dfgks_kernels.cu) -----------------------------------------------------------
void launch_fill_ghosts(const Mesh& m, double* W, double* alpha, const int* halt, cudaStream_t s, KernelTimer* T = nullptr);
// one pass of the ghost fill: 0 = ghost columns of the interior rows, 1 = ghost rows of all columns
void launch_ghost_pass(int dir, const Mesh& m, double* W, double* alpha, const int* halt, cudaStream_t s);
void launch_cfl_min(const Mesh& m, const double* W, double gamma, DevState* st, cudaStream_t s, KernelTimer* T = nullptr);
void launch_begin_step(DevState* st, double cfl, double dt_fixed, double t_end, double* dts, int idx, cudaStream_t s,
                       KernelTimer* T = nullptr);
void launch_end_step(DevState* st, double t_end, cudaStream_t s, KernelTimer* T = nullptr);
void launch_sweep(int dir, const Mesh& m, const SchemeConsts& S, int flux, bool alpha_only,
                  const double* W, const double* alpha, const double* dtp, const SweepBuffers& B,
                  DevState* st, const int* halt, cudaStream_t s, KernelTimer* T = nullptr);
// both directions in one launch per kernel class: the x-faces use Bx's face-line and Gauss-point
// records, flux[0] and tapes, the y-faces By's records, flux[1] and tapes (with tapes in both or
// in neither)
void launch_sweep_xy(const Mesh& m, const SchemeConsts& S, int flux, bool alpha_only, const double* W,
                     const double* alpha, const double* dtp, const SweepBuffers& Bx, const SweepBuffers& By,
                     DevState* st, const int* halt, cudaStream_t s, KernelTimer* T = nullptr);
void launch_update(int mode, const Mesh& m, const SchemeConsts& S, const UpdateArgs& a, const SweepBuffers& B,
                   const double* dtp, DevState* st, const int* halt, cudaStream_t s, KernelTimer* T = nullptr);
void launch_dense_to_ghosted(const Mesh& m, const double* dense, int ncomp, double* ghosted, cudaStream_t s);
void launch_ghosted_to_dense(const Mesh& m, const double* ghosted, int ncomp, double* dense, cudaStream_t s);
void launch_fill_value(double* p, long long n, double v, cudaStream_t s);
void launch_check_state(const Mesh& m, const double* W, double gm1, int* bad, cudaStream_t s);
void launch_set_scalar(double* p, double v, cudaStream_t s);
void launch_pack_faces(int dir, const Mesh& m, const SweepBuffers& B, double* out, cudaStream_t s);

// ---- reverse sweep (dfgks_adjoint.cu) -------------------------------------------------------
void launch_adjoint_dir(int dir, const Mesh& m, const SchemeConsts& S, int flux, const AdjointArgs& a,
                        const double* W, const double* alpha, const double* dtp, const SweepBuffers& B,
                        double* lb, double* gbuf, double* Wb, cudaStream_t s, KernelTimer* T = nullptr);
void launch_adjoint_finish(const Mesh& m, double* Wbg, double* Wb_dense, cudaStream_t s);
void launch_axpby(long long n, double a, const double* x, double b, double* y, cudaStream_t s);

}  // namespace dfk
