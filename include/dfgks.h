/*
 * dfgks.h -- C ABI of the GB300 (sm_103a) FP64 solver for the hybrid DF + WENO-AO
 * high-order finite-volume scheme of Zhang, Ji & Xu, "A robustness-enhanced reconstruction
 * based on discontinuity feedback factor for high-order finite volume scheme"
 * (arXiv 2402.10914).
 *
 * One handle = one 2-D structured-mesh Euler problem on one GPU and one CUDA stream.
 * Every call returns a dfgks_status; nothing throws or aborts across this boundary.
 *
 * Conventions used throughout:
 *   - All floating-point data is IEEE binary64 (double).
 *   - Conserved variables W = (rho, rho U, rho V, rho E) (Sect. 2.1) are stored SoA as
 *     [4][ny][nx], row-major, x fastest, interior cells only (no ghost layers).  Component k of
 *     cell (i, j) is W[k*nx*ny + j*nx + i].
 *   - The discontinuity feedback factor alpha (Sect. 3.2) is stored [ny][nx] the same way.
 *   - Pointer arguments are borrowed for the duration of the call.  "device" pointers must be
 *     CUDA device (or managed) memory of the current device; work is ordered on the handle's
 *     stream, and calls that return data to host memory synchronise that stream.
 *   - A handle is not thread-safe; use one handle per stream.
 *   - Cell (i, j) has centre (x0 + (i+1/2) dx, y0 + (j+1/2) dy), dx = (x1-x0)/nx, dy = (y1-y0)/ny.
 */
#ifndef DFGKS_H
#define DFGKS_H

#if defined(__GNUC__)
#define DFGKS_API __attribute__((visibility("default")))
#else
#define DFGKS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DFGKS_OK = 0,
    DFGKS_EINVAL = 1,      /* bad argument: null handle/pointer, size out of range, unknown enum */
    DFGKS_ENOMEM = 2,      /* a device or pinned allocation failed */
    DFGKS_ECUDA = 3,       /* a CUDA runtime call failed; the handle should be destroyed */
    DFGKS_ENONPHYS = 4,    /* initial/state data with rho <= 0, p <= 0 or a non-finite value */
    DFGKS_ENONPOS = 5,     /* positivity (rho > 0, p > 0, finite) lost during a step */
    DFGKS_ENAN = 6,        /* reserved: non-finite value outside the positivity check */
    DFGKS_ETIMEOUT = 7,    /* reserved: a bounded device-side wait expired (no kernel here waits) */
    DFGKS_ENOTSUP = 8      /* the requested combination is not implemented */
} dfgks_status;

typedef enum { DFGKS_FLUX_GKS = 0, DFGKS_FLUX_LF = 1 } dfgks_flux;

/* Boundary conditions: periodic wrap; outflow = zero-gradient copy (the paper's "free" and
 * "non-reflecting" boundaries, Sect. 4.3); reflecting wall = mirror with negated normal momentum. */
typedef enum { DFGKS_BC_PERIODIC = 0, DFGKS_BC_OUTFLOW = 1, DFGKS_BC_REFLECT = 2 } dfgks_bc;

typedef enum { DFGKS_TIME_S2O4 = 0, DFGKS_TIME_SSPRK3 = 1 } dfgks_time_scheme;

typedef struct dfgks_config {
    int nx, ny;                    /* interior cells, each >= 1 (>= 3 along a direction with a periodic or
                                      reflecting boundary: the ghost layers copy 3 interior cells) */
    double x0, x1, y0, y1;         /* domain [x0,x1] x [y0,y1] */
    double gamma;                  /* specific heat ratio; K = (4 - 2 gamma)/(gamma - 1) (Sect. 2.2) */
    double cfl;                    /* dt = cfl * min over cells of the dt_rule bound */
    int bc_xlo, bc_xhi, bc_ylo, bc_yhi;   /* dfgks_bc */
    double alpha_thres;            /* DF threshold of Eq. 34 (paper: 0.5) */
    double dH, dL;                 /* WENO-AO linear-weight parameters (paper: 0.85, 0.85) */
    double eps;                    /* WENO-Z and time-limiter epsilon (paper: 1e-6) */
    double C1, C2;                 /* numerical collision time tau_n = C1 dt + C2 |dp/sum p| dt (0.01, 5) */
    int time_limiter;              /* 1: S2O4 with the non-linear time limiter (Sect. 2.2) */
    int tau_reading;               /* 0: physical tau = 0 outside the exponentials; 1: tau = tau_n */
    int gp_fallback;               /* 1: Gauss-point states with rho <= 0 or p <= 0 use the cell average */
    int time_scheme;               /* dfgks_time_scheme */
    int dt_rule;                   /* CFL bound per cell (Alg. 1 gives no formula): 0 min(dx/(|U|+c), dy/(|V|+c)),
                                      1 1/((|U|+c)/dx + (|V|+c)/dy) */
    int df_states;                 /* the left and right states of a Gauss point's DF factor (Sect. 3.2):
                                      0 the reconstructed Gauss-point states (the paper's interface
                                      reconstruction values; default), 1 the cell averages of the two
                                      cells beside the face (an alternative, not the paper's reading) */
    int alpha_source;              /* where alpha^{n+1} comes from (Alg. 1 "update DF factor", Sect. 3.2):
                                      0 the Gauss-point states of the step's last stage (default), 1 one
                                      more reconstruction after the stages, of W^{n+1} itself with alpha^n
                                      deciding its DF branches (an extra face-line and tangential sweep
                                      per step).  Single-problem stepping only: the batch and the block
                                      decomposition refuse 1 with DFGKS_EINVAL, the checkpointed forward
                                      and adjoint with DFGKS_ENOTSUP */
} dfgks_config;

typedef struct dfgks dfgks;        /* opaque; owns every device buffer it uses */

/* Counters accumulated since the last dfgks_set_ic / dfgks_set_state. */
typedef struct dfgks_counters {
    unsigned long long fallbacks;      /* Gauss-point side states replaced by the cell average */
    unsigned long long df_normal;      /* normal reconstructions (per face line side) on the DF branch */
    unsigned long long df_tangential;  /* tangential reconstructions (per face side) on the DF branch */
} dfgks_counters;

/* Human-readable name of a status code (static storage). */
DFGKS_API const char* dfgks_status_string(int status);

/* Fill *cfg with the paper's constants (Sect. 2.2, 3.1, 3.3) for an nx x ny mesh on [0,1]^2 with
 * outflow boundaries, gamma 1.4, CFL 0.5, S2O4 with the time limiter, tau reading 0, fallback on. */
DFGKS_API dfgks_status dfgks_config_default(dfgks_config* cfg, int nx, int ny);

/* Create a solver for cfg on the current CUDA device.  stream: a cudaStream_t to order all work
 * on (cudaStreamLegacy for the legacy default stream), or NULL to create a private non-blocking
 * stream, which is not ordered with work the caller puts on other streams.  Allocates every device buffer the step
 * needs (about 140 doubles per cell for the default path).  On success *out owns them. */
DFGKS_API dfgks_status dfgks_create(const dfgks_config* cfg, void* stream, dfgks** out);

/* Release every buffer and the private stream, if any.  Accepts NULL. */
DFGKS_API dfgks_status dfgks_destroy(dfgks* h);

/* Load the initial cell averages W [4][ny][nx] (host memory if on_device == 0, else device),
 * set t = 0, step = 0, reset the counters, and compute alpha^0 as the product of the Gauss-point
 * DF factors (Sect. 3.2) of a reconstruction of W with alpha = 1 (the paper leaves alpha^0 open).
 * Returns DFGKS_ENONPHYS (state unchanged) if any cell has rho <= 0, p <= 0 or a non-finite value. */
DFGKS_API dfgks_status dfgks_set_ic(dfgks* h, const double* W, int on_device);

/* Copy out the current state.  W [4][ny][nx] and alpha [ny][nx] may each be NULL; they are host
 * memory if on_device == 0, else device.  t and step may be NULL.  Synchronises the stream. */
DFGKS_API dfgks_status dfgks_get_state(dfgks* h, double* W, double* alpha, double* t, long* step, int on_device);

/* Replace the current state (checkpoint resume).  alpha may be NULL (then alpha^0 is recomputed
 * as in dfgks_set_ic).  Returns DFGKS_ENONPHYS on non-physical W, leaving the state unchanged. */
DFGKS_API dfgks_status dfgks_set_state(dfgks* h, const double* W, const double* alpha, double t, long step, int on_device);

/* Algorithm 1, repeated: advance up to n steps with flux solver `flux`.
 *   dt > 0: fixed step; dt <= 0: the CFL rule of dfgks_config.cfl, from W^n, every step.
 *   t_end > 0: the step that would pass t_end is clipped to end exactly there (a remainder below
 *   1e-12 |t_end| is absorbed) and no further steps are taken; t_end <= 0: no limit.
 * Each step: dt (device-resident), ghost fill, then per stage the fused reconstruction + flux
 * sweeps and the stage update (S2O4, Eq. 24 with the time limiter; or SSP-RK3, Sect. 2.3);
 * alpha^{n+1} is the product of the DF factors at the last stage's Gauss points.
 * dts_out (host, length n) receives each executed step's dt, may be NULL; *steps_done (may be
 * NULL) receives the number of steps executed.  Synchronises the stream once, at the end.
 * On a positivity failure returns DFGKS_ENONPOS with the state left at the last good step;
 * dfgks_last_error_detail gives the failing step and cell. */
DFGKS_API dfgks_status dfgks_step(dfgks* h, int n, double dt, int flux, double t_end, double* dts_out, int* steps_done);

/* Single-stage operator of Eq. 2 with two-point Gauss quadrature (Sect. 2.1, 2.2, 3): from device
 * W [4][ny][nx] and alpha [ny][nx], with ghosts filled by the handle's boundary conditions, write
 * to device memory L = L(W), dtL = dL/dt (Eq. 27 summed as in Eq. 2), dtLt = the time-limited
 * dL/dt (omega^t applied per face, Sect. 2.2), alpha_next = product of the Gauss-point DF factors.
 * Any output may be NULL.  The GKS flux depends on dt through tau_n and the time integrals
 * (Eqs. 25-27); L-F ignores dt.  Does not touch the handle's state. Asynchronous on the stream. */
DFGKS_API dfgks_status dfgks_residual(dfgks* h, const double* W, const double* alpha, double dt, int flux,
                            double* L, double* dtL, double* dtLt, double* alpha_next);

/* The stage operator of dfgks_residual for callers that cannot allocate device memory (code that
 * runs while a CUDA graph is being built, hosts whose device memory belongs to their own pool
 * allocator, latency-bound loops).  The paper has no counterpart; this is a deployment variant.
 * Takes a configuration instead of a handle; inputs and outputs as in dfgks_residual (device
 * memory, dense [4][ny][nx] / [ny][nx]; outputs may be NULL); work is ordered on `stream`
 * (a cudaStream_t, or NULL for the legacy default stream).  No cudaMalloc or cudaFree is called:
 * every intermediate lives in one file-scope 16 MiB device array that each GPU using the library
 * holds until exit.  A mesh with a side above 128 cells (nx > 128 or ny > 128) is rejected with
 * DFGKS_EINVAL, and so is every configuration dfgks_create refuses (for instance a periodic or
 * reflecting direction with fewer than 3 cells); both checks run before any device work.
 * The first call on a device looks up that array's device address (cudaGetSymbolAddress) with the
 * device current; make that first call before any stream capture.  All calls share the array and
 * it keeps the last call's contents: calls that overlap on the GPU (different streams, concurrent
 * graphs) race on it and must be serialised by the caller. */
DFGKS_API dfgks_status dfgks_residual_noalloc(const dfgks_config* cfg, void* stream,
                                              const double* W, const double* alpha, double dt, int flux,
                                              double* L, double* dtL, double* dtLt, double* alpha_next);

/* Vector-Jacobian product of dfgks_residual with respect to W, with alpha, dt and every branch
 * decision (DF switch, Gauss-point fallback, the sign of |.|, the arguments chosen by min/max)
 * held at the values of the forward pass:
 *   W_bar += (dL/dW)^T L_bar + (d dtL/dW)^T dtL_bar + (d dtLt/dW)^T dtLt_bar.
 * All pointers device, dense [4][ny][nx]; L_bar / dtL_bar / dtLt_bar may be NULL (zero).  Not part
 * of the paper: a hand-written reverse sweep of the operator of Eq. 2 (ghost fill, normal and
 * tangential reconstruction, GKS / L-F flux, time-limiter weight).  Asynchronous on the stream;
 * uses the handle's scratch (allocated on first use). */
DFGKS_API dfgks_status dfgks_adjoint_residual(dfgks* h, const double* W, const double* alpha, double dt, int flux,
                                              const double* L_bar, const double* dtL_bar, const double* dtLt_bar,
                                              double* W_bar);

/* Forward pass for a later gradient: sets the state to W0 (device, dense; alpha^0 computed from W0
 * as in dfgks_set_ic, t = 0) and advances n S2O4 steps of flux `flux`, with the step sizes dts_in[n]
 * (host) or, if dts_in is NULL, the CFL rule; dts_out[n] (host, may be NULL) receives them.  Keeps W
 * and alpha every ckpt_every steps, the step sizes, and the last segment's stage states and (if they
 * fit in half of the free device memory) its sweep records and tapes, in the handle (allocated on
 * demand, freed by dfgks_destroy) for dfgks_adjoint_checkpointed.  Not part of the paper.  S2O4 with
 * alpha_source 0 only (DFGKS_ENOTSUP otherwise, also through dfgks_adjoint_steps); DFGKS_ENONPOS if
 * the trajectory loses positivity.  Synchronises. */
DFGKS_API dfgks_status dfgks_forward_checkpointed(dfgks* h, const double* W0, int n, const double* dts_in, int flux,
                                                  int ckpt_every, double* dts_out);

/* Gradient through the steps of the last dfgks_forward_checkpointed (Eq. 24 with the time
 * limiter): W0_bar = (dW^n/dW0)^T WT_bar, both device, dense [4][ny][nx], with the alpha sequence,
 * step sizes and branch decisions of the forward trajectory held fixed.  Each segment of
 * ckpt_every steps is recomputed from its checkpoint (the last one only if the forward pass could not
 * keep it), keeping its stage states and (if they take at most half of the free device memory) every
 * stage's forward sweep records with the reconstructions' and GKS flux's intermediates, and then
 * reversed.
 * DFGKS_EINVAL if no forward pass was kept or the state changed since (set_ic, set_state, step).
 * Allocates its segment buffers for the call.  Leaves the handle at W^n.  Synchronises. */
DFGKS_API dfgks_status dfgks_adjoint_checkpointed(dfgks* h, const double* WT_bar, double* W0_bar);

/* dfgks_forward_checkpointed with the given step sizes dts[n] followed by
 * dfgks_adjoint_checkpointed: the gradient through n steps from W0 in one call. */
DFGKS_API dfgks_status dfgks_adjoint_steps(dfgks* h, const double* W0, int n, const double* dts, int flux,
                                           int ckpt_every, const double* WT_bar, double* W0_bar);

/* ---- Batched problems ----------------------------------------------------------------------
 * Many independent problems (each its own mesh size, boundary conditions, flux solver and CFL dt)
 * advanced together: every phase of a step is one launch over all problems, the sweep kernels on
 * 1-D blocks of an autotuned size over each problem's face lines, face sides and Gauss points, and
 * n steps are captured once in a CUDA graph that one launch replays.  Not part of the paper (a
 * throughput mode for many small problems on one GPU).  S2O4 only (time_scheme 0).  Each problem's
 * state, alpha, dt, time and step counter are its own; a problem that loses positivity stops at
 * its last good step while the others continue. */
typedef struct dfgks_batch dfgks_batch;

/* cfgs[np], flux[np] (dfgks_flux); stream NULL creates a private stream (graph capture needs a
 * non-default stream).  Allocates every problem's buffers. */
DFGKS_API dfgks_status dfgks_batch_create(const dfgks_config* cfgs, const int* flux, int np, void* stream,
                                          dfgks_batch** out);
DFGKS_API dfgks_status dfgks_batch_destroy(dfgks_batch* b);
/* Initial state of problem p (host if on_device == 0); alpha^0 as in dfgks_set_ic; ENONPHYS on bad data. */
DFGKS_API dfgks_status dfgks_batch_set_ic(dfgks_batch* b, int p, const double* W, int on_device);
/* Capture the CUDA graph that advances every problem n steps (1 <= n <= 100000); dfgks_batch_step
 * does this on first use of an n, so calling it ahead keeps the capture out of a timed region.
 * The graph is dropped when the block sizes change. */
DFGKS_API dfgks_status dfgks_batch_prepare(dfgks_batch* b, int n);
/* Advance every problem n steps; use_graph != 0: one launch of the n-step graph, otherwise the
 * same launches issued one by one.  Synchronises the batch's stream at the end.
 * Returns DFGKS_ENONPOS if any problem lost positivity (see dfgks_batch_status). */
DFGKS_API dfgks_status dfgks_batch_step(dfgks_batch* b, int n, int use_graph);
DFGKS_API dfgks_status dfgks_batch_get_state(dfgks_batch* b, int p, double* W, double* alpha, double* t, long* step,
                                             int on_device);
/* Step count, error flag (0 or DFGKS_ENONPOS) and normal DF-branch count of problem p. */
DFGKS_API dfgks_status dfgks_batch_status(dfgks_batch* b, int p, long* step, int* err, unsigned long long* df_normal);
/* Threads per block (64, 128 or 256) of the face-line, tangential and flux kernels. */
DFGKS_API dfgks_status dfgks_batch_set_blocks(dfgks_batch* b, const int* blocks3);
/* Pick those sizes by timing one batched step per candidate (64, 128, 256), kernel class by class;
 * states are saved and restored around the trials.  blocks3 (may be NULL) receives the choice,
 * best_ms (may be NULL) the last class's best step time. */
DFGKS_API dfgks_status dfgks_batch_autotune(dfgks_batch* b, int* blocks3, double* best_ms);

/* ---- One problem in blocks (domain decomposition) -------------------------------------------
 * The mesh split into px x py rectangular blocks (block b = by * px + bx covers cells
 * [i0, i1) x [j0, j1), i0 = floor(nx bx / px), likewise in y), each with its own ghosted buffers on
 * the current device.  Before every stage the ghost layers are filled in two passes over all
 * blocks: the ghost columns of the interior rows (a shared side by copying the neighbouring
 * block's G boundary columns), then the ghost rows including the ghost columns (a shared side by
 * copying the neighbour's G boundary rows, which carries the diagonal neighbour's cells into the
 * corners); sides on the mesh boundary keep their boundary condition, and a periodic side of a
 * split direction is shared with the block at the other end.  dt is the minimum over all blocks.
 * A decomposed run reproduces dfgks_step on the whole mesh bit for bit.  Not part of the paper
 * (one mesh per case there).  S2O4 only; a split direction needs at least 3 cells per block. */
typedef struct dfgks_decomp dfgks_decomp;
/* A block's place in the decomposition: its cells [i0, i1) x [j0, j1) of the whole mesh, per side
 * (x-low, x-high, y-low, y-high) the boundary condition (dfgks_bc, or 3 for a side filled by a halo
 * copy) and the neighbouring block the copy comes from (-1 for a boundary side).  Host only. */
typedef struct dfgks_block_plan { int i0, i1, j0, j1; int bc[4]; int neighbour[4]; } dfgks_block_plan;
DFGKS_API dfgks_status dfgks_decomp_plan(const dfgks_config* cfg, int px, int py, int block, dfgks_block_plan* out);
/* The halo copy that fills side `side` (0 x-low, 1 x-high, 2 y-low, 3 y-high) of block `block`:
 * the neighbouring block it comes from (-1: a boundary side, no copy), the window of this block's
 * ghosted field it fills (first cell (di, dj) in the block's cell indices, ghosts negative or
 * >= the block's size; w x h cells) and the first cell (si, sj) of the same-sized window in the
 * neighbour's field.  x sides are copied in the first pass of the ghost fill, y sides (whose
 * windows include the ghost columns) in the second.  Host only: a run with one block per device
 * sends and receives exactly these windows. */
typedef struct dfgks_halo_window { int neighbour, di, dj, si, sj, w, h; } dfgks_halo_window;
DFGKS_API dfgks_status dfgks_decomp_halo(const dfgks_config* cfg, int px, int py, int block, int side,
                                         dfgks_halo_window* out);
/* Allocate the blocks (stream NULL: a private stream).  EINVAL for configurations the whole-mesh
 * handle refuses, time_scheme != S2O4, or fewer than 3 cells per block along a split direction. */
DFGKS_API dfgks_status dfgks_decomp_create(const dfgks_config* cfg, int px, int py, void* stream, dfgks_decomp** out);
DFGKS_API dfgks_status dfgks_decomp_destroy(dfgks_decomp* d);
/* Initial state of the whole mesh, dense [4][ny][nx] (host if on_device == 0), scattered to the
 * blocks; alpha^0 as in dfgks_set_ic; ENONPHYS on a non-physical cell. */
DFGKS_API dfgks_status dfgks_decomp_set_ic(dfgks_decomp* d, const double* W, int on_device);
/* n S2O4 steps with the CFL dt, the last clipped to t_end > 0; synchronises once at the end.
 * ENONPOS on a positivity failure, the state left at the last good step. */
DFGKS_API dfgks_status dfgks_decomp_step(dfgks_decomp* d, int n, int flux, double t_end, int* steps_done);
/* The whole mesh's state gathered from the blocks: W [4][ny][nx], alpha [ny][nx] (either may be
 * NULL; host memory if on_device == 0), time and step count. */
DFGKS_API dfgks_status dfgks_decomp_get_state(dfgks_decomp* d, double* W, double* alpha, double* t, long* step,
                                              int on_device);
/* Error flag (0 or DFGKS_ENONPOS), the first failing cell (whole-mesh indices, -1 if none) and the
 * branch counters summed over the blocks.  Any pointer may be NULL. */
DFGKS_API dfgks_status dfgks_decomp_status(dfgks_decomp* d, int* err, int* fail_i, int* fail_j, dfgks_counters* counters);

/* Per-face intermediates of one stage, for diagnostics and kernel-by-kernel comparison.
 * dir 0: x-faces, [ny][nx+1] (face index fastest); dir 1: y-faces, [nx][ny+1].
 * Per face 59 doubles: F[4], dtF[4] (global frame, Gauss-averaged), omega^t, alpha_{p,1},
 * alpha_{p,2}, then for side (left, right) x Gauss point (1, 2): W[4], W_n[4], W_t[4] in the
 * face's local frame (Sect. 2.1).  W, alpha device; out is device memory of nfaces*59 doubles. */
DFGKS_API dfgks_status dfgks_face_records(dfgks* h, const double* W, const double* alpha, double dt, int flux,
                                int dir, double* out);

/* Counters since the last set_ic/set_state (synchronises the stream). */
DFGKS_API dfgks_status dfgks_get_counters(dfgks* h, dfgks_counters* out);

/* Step index and cell of the first positivity failure reported by dfgks_step (-1 if none). */
DFGKS_API dfgks_status dfgks_last_error_detail(dfgks* h, long* step, int* i, int* j);

/* Per-kernel-class timing for profiling.  Classes, in order: 0 face-line normal reconstruction,
 * 1 tangential reconstruction, 2 Gauss-point flux, 3 stage update, 4 other (ghost fill, dt,
 * bookkeeping).  When enabled, dfgks_step records a CUDA event pair on the handle's stream around
 * each launch of a class; kernels themselves are unchanged.  Synchronises the stream. */
DFGKS_API dfgks_status dfgks_set_timing(dfgks* h, int enable);

/* Accumulated event time (ms), number of timed launches and number of kernel launches issued by
 * dfgks_step, per class (arrays of 5; each may be NULL).  reset != 0 clears the accumulators.
 * Synchronises the stream. */
DFGKS_API dfgks_status dfgks_get_timing(dfgks* h, double* total_ms, long long* timed, long long* launches, int reset);

/* FP64 throughput probe on the current device: independent fused multiply-add chains (8 per
 * thread, `iters` iterations, 8 blocks of 256 threads per SM), timed with CUDA events.  Writes the
 * achieved GFLOP/s (2 per FMA) and the kernel time in ms (may be NULL).  Allocates 512 KiB. */
DFGKS_API dfgks_status dfgks_probe_fp64(int iters, double* gflops, double* ms);

/* Device bytes held by the handle. */
DFGKS_API dfgks_status dfgks_device_bytes(dfgks* h, unsigned long long* bytes);

#ifdef __cplusplus
}
#endif
#endif /* DFGKS_H */
