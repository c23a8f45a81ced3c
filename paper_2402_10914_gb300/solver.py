"""Python front end of the CUDA solver: a handle per problem, torch for device memory/streams.

``Solver`` marshals arguments to the C ABI (``_lib``); all arithmetic runs in the CUDA library.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from .inputs import Settings

FACE_RECORD = 59


def make_config(s: Settings) -> _lib.Config:
    c = _lib.Config()
    _lib.check(_lib.lib().dfgks_config_default(C.byref(c), int(s.nx), int(s.ny)), "dfgks_config_default")
    for f in ("nx", "ny", "x0", "x1", "y0", "y1", "gamma", "cfl", "alpha_thres", "dH", "dL", "eps", "C1", "C2",
              "time_limiter", "tau_reading", "gp_fallback", "time_scheme", "dt_rule", "df_states",
              "alpha_source"):
        setattr(c, f, getattr(s, f))
    c.bc_xlo, c.bc_xhi, c.bc_ylo, c.bc_yhi = (int(b) for b in s.bc)
    return c


CUDA_STREAM_LEGACY = 0x1        # cudaStreamLegacy


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        assert t.dtype == torch.float64 and t.is_contiguous()
        return C.c_void_p(t.data_ptr())
    assert isinstance(t, np.ndarray) and t.dtype == np.float64 and t.flags.c_contiguous
    return C.c_void_p(t.ctypes.data)


class Solver:
    """One 2-D Euler problem on the current CUDA device, ordered on a torch stream."""

    def __init__(self, settings: Settings, stream: torch.cuda.Stream | None = None):
        self.settings = settings
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._cfg = make_config(settings)
        h = C.c_void_p()
        # torch's default stream has the handle 0, the legacy default stream; the C ABI reads NULL as
        # "create a private stream", so the legacy stream goes in as cudaStreamLegacy
        handle = self.stream.cuda_stream or CUDA_STREAM_LEGACY
        _lib.check(_lib.lib().dfgks_create(C.byref(self._cfg), C.c_void_p(handle), C.byref(h)), "dfgks_create")
        self._h = h

    # -- lifecycle ---------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            _lib.lib().dfgks_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def shape(self):
        return (4, self.settings.ny, self.settings.nx)

    # -- state -------------------------------------------------------------------------
    def set_ic(self, W):
        on_dev = isinstance(W, torch.Tensor) and W.is_cuda
        W = W if on_dev else np.ascontiguousarray(np.asarray(W, dtype=np.float64))
        assert tuple(W.shape) == self.shape
        _lib.check(_lib.lib().dfgks_set_ic(self._h, _ptr(W), int(on_dev)), "dfgks_set_ic")

    def set_state(self, W, alpha=None, t=0.0, step=0):
        on_dev = isinstance(W, torch.Tensor) and W.is_cuda
        if not on_dev:
            W = np.ascontiguousarray(np.asarray(W, dtype=np.float64))
            alpha = None if alpha is None else np.ascontiguousarray(np.asarray(alpha, dtype=np.float64))
        _lib.check(_lib.lib().dfgks_set_state(self._h, _ptr(W), _ptr(alpha), float(t), int(step), int(on_dev)),
                   "dfgks_set_state")

    def get_state(self, device: bool = False, out=None):
        """(W, alpha, t, step).  out: optional (W, alpha) to fill instead of new arrays, both host
        arrays (numpy, ideally views of pinned memory: the copy then needs no staging) or both CUDA
        tensors, float64, C-contiguous, shaped (4, ny, nx) and (ny, nx)."""
        if out is not None:
            W, a = out
            device = isinstance(W, torch.Tensor) and W.is_cuda
            if tuple(W.shape) != self.shape or tuple(a.shape) != self.shape[1:] or \
                    device != (isinstance(a, torch.Tensor) and a.is_cuda):
                raise ValueError("get_state: out must be (W, alpha) of shapes %s and %s, both on the host or "
                                 "both on the device" % (self.shape, self.shape[1:]))
        elif device:
            W = torch.empty(self.shape, dtype=torch.float64, device="cuda")
            a = torch.empty(self.shape[1:], dtype=torch.float64, device="cuda")
        else:
            W = np.empty(self.shape)
            a = np.empty(self.shape[1:])
        t = C.c_double()
        st = C.c_long()
        _lib.check(_lib.lib().dfgks_get_state(self._h, _ptr(W), _ptr(a), C.byref(t), C.byref(st), int(device)),
                   "dfgks_get_state")
        return W, a, t.value, st.value

    # -- stepping ----------------------------------------------------------------------
    def step(self, n: int, dt: float = 0.0, flux: int | None = None, t_end: float = 0.0, record_dts: bool = False):
        """Advance up to n steps; returns (steps_done, dts or None).  Raises DfgksError on failure."""
        flux = self.settings.flux if flux is None else flux
        dts = np.zeros(max(n, 1)) if record_dts else None
        done = C.c_int()
        rc = _lib.lib().dfgks_step(self._h, int(n), float(dt or 0.0), int(flux), float(t_end or 0.0),
                                   None if dts is None else dts.ctypes.data_as(C.POINTER(C.c_double)), C.byref(done))
        _lib.check(rc, "dfgks_step")
        return done.value, (dts[:done.value] if dts is not None else None)

    def run(self, t_end: float | None = None, steps: int | None = None, dt: float = 0.0, chunk: int = 64,
            record_dts: bool = False):
        """Run to t_end (chunks of `chunk` steps) or for a fixed number of steps."""
        total, all_dts = 0, []
        if t_end is None:
            done, d = self.step(steps, dt=dt, record_dts=record_dts)
            return done, d
        while True:
            n = chunk if steps is None else min(chunk, steps - total)
            if n <= 0:
                break
            done, d = self.step(n, dt=dt, t_end=t_end, record_dts=record_dts)
            total += done
            if d is not None:
                all_dts.append(d)
            if done < n:
                break
        return total, (np.concatenate(all_dts) if all_dts else None)

    def last_error(self):
        s, i, j = C.c_long(), C.c_int(), C.c_int()
        _lib.check(_lib.lib().dfgks_last_error_detail(self._h, C.byref(s), C.byref(i), C.byref(j)),
                   "dfgks_last_error_detail")
        return s.value, i.value, j.value

    def counters(self):
        c = _lib.Counters()
        _lib.check(_lib.lib().dfgks_get_counters(self._h, C.byref(c)), "dfgks_get_counters")
        return {"fallbacks": c.fallbacks, "df_normal": c.df_normal, "df_tangential": c.df_tangential}

    KERNEL_CLASSES = ("lines", "faces", "flux", "update", "other")

    def set_timing(self, enable: bool) -> None:
        _lib.check(_lib.lib().dfgks_set_timing(self._h, int(enable)), "dfgks_set_timing")

    def timing(self, reset: bool = False) -> dict:
        ms = np.zeros(5)
        timed = np.zeros(5, dtype=np.int64)
        launches = np.zeros(5, dtype=np.int64)
        _lib.check(_lib.lib().dfgks_get_timing(self._h, C.c_void_p(ms.ctypes.data), C.c_void_p(timed.ctypes.data),
                                               C.c_void_p(launches.ctypes.data), int(reset)), "dfgks_get_timing")
        return {k: {"ms": float(ms[q]), "timed": int(timed[q]), "launches": int(launches[q])}
                for q, k in enumerate(self.KERNEL_CLASSES)}

    def device_bytes(self) -> int:
        b = C.c_ulonglong()
        _lib.check(_lib.lib().dfgks_device_bytes(self._h, C.byref(b)), "dfgks_device_bytes")
        return b.value

    # -- stage operator ------------------------------------------------------------------
    def residual(self, W: torch.Tensor, alpha: torch.Tensor, dt: float, flux: int | None = None):
        """(L, dL/dt, limited dL/dt, alpha_next) as new CUDA tensors."""
        flux = self.settings.flux if flux is None else flux
        L = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        dL, dLt = torch.empty_like(L), torch.empty_like(L)
        an = torch.empty(self.shape[1:], dtype=torch.float64, device="cuda")
        _lib.check(_lib.lib().dfgks_residual(self._h, _ptr(W), _ptr(alpha), float(dt), int(flux),
                                             _ptr(L), _ptr(dL), _ptr(dLt), _ptr(an)), "dfgks_residual")
        return L, dL, dLt, an

    def face_records(self, W: torch.Tensor, alpha: torch.Tensor, dt: float, direction: int, flux: int | None = None):
        flux = self.settings.flux if flux is None else flux
        s = self.settings
        nf, nt = (s.nx + 1, s.ny) if direction == 0 else (s.ny + 1, s.nx)
        out = torch.empty((nt, nf, FACE_RECORD), dtype=torch.float64, device="cuda")
        _lib.check(_lib.lib().dfgks_face_records(self._h, _ptr(W), _ptr(alpha), float(dt), int(flux),
                                                 int(direction), _ptr(out)), "dfgks_face_records")
        return out


class BatchSolver:
    """Many independent problems advanced together (dfgks_batch_*): one launch per phase over all
    problems, optionally replayed from a CUDA graph.  ``settings`` is a list of ``Settings``."""

    def __init__(self, settings: list, autotune_cache: str | None = None, stream=None):
        """``stream``: a non-default torch.cuda.Stream to order the batch's work on (events recorded
        on it time the batch); None lets the library create a private stream."""
        self.settings = list(settings)
        n = len(self.settings)
        cfgs = (_lib.Config * n)()
        for k, s in enumerate(self.settings):
            cfgs[k] = make_config(s)
        flux = (C.c_int * n)(*[int(s.flux) for s in self.settings])
        h = C.c_void_p()
        self.stream = stream
        handle = None if stream is None else C.c_void_p(stream.cuda_stream)
        _lib.check(_lib.lib().dfgks_batch_create(C.cast(cfgs, C.c_void_p), C.cast(flux, C.c_void_p), n, handle,
                                                 C.byref(h)), "dfgks_batch_create")
        self._h = h
        self.blocks = None
        self._cache = autotune_cache

    def close(self):
        if getattr(self, "_h", None):
            _lib.lib().dfgks_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_ic(self, p: int, W):
        W = np.ascontiguousarray(np.asarray(W, dtype=np.float64))
        _lib.check(_lib.lib().dfgks_batch_set_ic(self._h, int(p), C.c_void_p(W.ctypes.data), 0), "dfgks_batch_set_ic")

    def step(self, n: int, use_graph: bool = True) -> int:
        """Advance all problems n steps (with use_graph, one launch of the n-step CUDA graph); returns
        the status (0 or ENONPOS) instead of raising on positivity loss, since the other problems
        continue."""
        rc = _lib.lib().dfgks_batch_step(self._h, int(n), int(use_graph))
        if rc not in (_lib.OK, _lib.ENONPOS):
            _lib.check(rc, "dfgks_batch_step")
        return rc

    def get_state(self, p: int):
        s = self.settings[p]
        W = np.empty((4, s.ny, s.nx))
        a = np.empty((s.ny, s.nx))
        t, st = C.c_double(), C.c_long()
        _lib.check(_lib.lib().dfgks_batch_get_state(self._h, int(p), C.c_void_p(W.ctypes.data), C.c_void_p(a.ctypes.data),
                                                    C.byref(t), C.byref(st), 0), "dfgks_batch_get_state")
        return W, a, t.value, st.value

    def status(self, p: int):
        st, err, dfn = C.c_long(), C.c_int(), C.c_ulonglong()
        _lib.check(_lib.lib().dfgks_batch_status(self._h, int(p), C.byref(st), C.byref(err), C.byref(dfn)),
                   "dfgks_batch_status")
        return {"step": st.value, "err": err.value, "df_normal": dfn.value}

    def prepare(self, n: int):
        """Capture the CUDA graph that advances every problem n steps (dfgks_batch_prepare)."""
        _lib.check(_lib.lib().dfgks_batch_prepare(self._h, int(n)), "dfgks_batch_prepare")

    def set_blocks(self, blocks):
        arr = (C.c_int * 3)(*[int(v) for v in blocks])
        _lib.check(_lib.lib().dfgks_batch_set_blocks(self._h, C.cast(arr, C.c_void_p)), "dfgks_batch_set_blocks")
        self.blocks = [int(v) for v in blocks]

    def signature(self) -> str:
        return ";".join("%dx%d:%d" % (s.nx, s.ny, s.flux) for s in self.settings)

    def autotune(self):
        """Pick the sweep kernels' block sizes by timing (dfgks_batch_autotune); with a cache file,
        reuse an earlier choice for the same set of problems."""
        import json
        import os
        key = self.signature()
        if self._cache and os.path.exists(self._cache):
            try:
                cached = json.load(open(self._cache)).get(key)
            except Exception:
                cached = None
            if cached:
                self.set_blocks(cached)
                return self.blocks, None
        arr = (C.c_int * 3)()
        best = C.c_double()
        _lib.check(_lib.lib().dfgks_batch_autotune(self._h, C.cast(arr, C.c_void_p), C.byref(best)),
                   "dfgks_batch_autotune")
        self.blocks = [arr[0], arr[1], arr[2]]
        if self._cache:
            data = {}
            if os.path.exists(self._cache):
                try:
                    data = json.load(open(self._cache))
                except Exception:
                    data = {}
            data[key] = self.blocks
            with open(self._cache, "w") as f:
                json.dump(data, f)
        return self.blocks, best.value


def block_plan(settings: Settings, px: int, py: int, block: int) -> dict:
    """Where block `block` of a px x py decomposition sits (dfgks_decomp_plan; host only): its cells
    [i0, i1) x [j0, j1), per side (x-low, x-high, y-low, y-high) its boundary code (BC_EXTERNAL for
    a side a halo copy fills) and the neighbouring block that copy comes from (-1 for none)."""
    p = _lib.BlockPlan()
    cfg = make_config(settings)
    _lib.check(_lib.lib().dfgks_decomp_plan(C.byref(cfg), int(px), int(py), int(block), C.byref(p)),
               "dfgks_decomp_plan")
    return {"i0": p.i0, "i1": p.i1, "j0": p.j0, "j1": p.j1, "bc": list(p.bc), "neighbour": list(p.neighbour)}


def halo_window(settings: Settings, px: int, py: int, block: int, side: int) -> dict:
    """The halo copy filling one side of a block (dfgks_decomp_halo; host only): the neighbour it
    comes from (-1: none), the window (di, dj, w, h) of the block's ghosted field and its start
    (si, sj) in the neighbour's field, both in block cell indices (ghosts negative / >= size)."""
    hw = _lib.HaloWindow()
    cfg = make_config(settings)
    _lib.check(_lib.lib().dfgks_decomp_halo(C.byref(cfg), int(px), int(py), int(block), int(side), C.byref(hw)),
               "dfgks_decomp_halo")
    return {f: getattr(hw, f) for f, _ in _lib.HaloWindow._fields_}


class DecompSolver:
    """One problem split into px x py blocks with halo exchange (dfgks_decomp_*), on the current
    device; the state goes in and out as the whole mesh."""

    def __init__(self, settings: Settings, px: int, py: int, stream: torch.cuda.Stream | None = None):
        self.settings = settings
        self.px, self.py = int(px), int(py)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._cfg = make_config(settings)
        h = C.c_void_p()
        handle = self.stream.cuda_stream or CUDA_STREAM_LEGACY
        _lib.check(_lib.lib().dfgks_decomp_create(C.byref(self._cfg), self.px, self.py, C.c_void_p(handle), C.byref(h)),
                   "dfgks_decomp_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.lib().dfgks_decomp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_ic(self, W):
        W = np.ascontiguousarray(np.asarray(W, dtype=np.float64))
        assert W.shape == (4, self.settings.ny, self.settings.nx)
        _lib.check(_lib.lib().dfgks_decomp_set_ic(self._h, C.c_void_p(W.ctypes.data), 0), "dfgks_decomp_set_ic")

    def step(self, n: int, t_end: float = 0.0, flux: int | None = None) -> int:
        done = C.c_int(0)
        f = self.settings.flux if flux is None else flux
        _lib.check(_lib.lib().dfgks_decomp_step(self._h, int(n), int(f), float(t_end), C.byref(done)),
                   "dfgks_decomp_step")
        return done.value

    def get_state(self):
        s = self.settings
        W = np.empty((4, s.ny, s.nx))
        a = np.empty((s.ny, s.nx))
        t, st = C.c_double(), C.c_long()
        _lib.check(_lib.lib().dfgks_decomp_get_state(self._h, C.c_void_p(W.ctypes.data), C.c_void_p(a.ctypes.data),
                                                     C.byref(t), C.byref(st), 0), "dfgks_decomp_get_state")
        return W, a, t.value, st.value

    def status(self) -> dict:
        err, fi, fj = C.c_int(), C.c_int(), C.c_int()
        c = _lib.Counters()
        _lib.check(_lib.lib().dfgks_decomp_status(self._h, C.byref(err), C.byref(fi), C.byref(fj), C.byref(c)),
                   "dfgks_decomp_status")
        return {"err": err.value, "fail_i": fi.value, "fail_j": fj.value, "fallbacks": c.fallbacks,
                "df_normal": c.df_normal, "df_tangential": c.df_tangential}


def _dev(t):
    return t if (isinstance(t, torch.Tensor) and t.is_cuda) else torch.as_tensor(
        np.ascontiguousarray(t), dtype=torch.float64, device="cuda")


def adjoint_residual(sol: "Solver", W, alpha, dt, L_bar=None, dtL_bar=None, dtLt_bar=None, flux=None,
                     W_bar=None) -> torch.Tensor:
    """W_bar (+)= J^T (L_bar, dtL_bar, dtLt_bar) of the stage operator (dfgks_adjoint_residual)."""
    flux = sol.settings.flux if flux is None else flux
    W, alpha = _dev(W).contiguous(), _dev(alpha).contiguous()
    bars = [None if b is None else _dev(b).contiguous() for b in (L_bar, dtL_bar, dtLt_bar)]
    out = torch.zeros_like(W) if W_bar is None else W_bar
    _lib.check(_lib.lib().dfgks_adjoint_residual(sol._h, _ptr(W), _ptr(alpha), float(dt), int(flux),
                                                 *[_ptr(b) for b in bars], _ptr(out)), "dfgks_adjoint_residual")
    return out


def adjoint_steps(sol: "Solver", W0, dts, WT_bar, ckpt_every: int = 10, flux=None) -> torch.Tensor:
    """(dW^n/dW0)^T WT_bar through the recorded S2O4 steps (dfgks_adjoint_steps)."""
    flux = sol.settings.flux if flux is None else flux
    W0 = _dev(W0).contiguous()
    WTb = _dev(WT_bar).contiguous()
    dts = np.ascontiguousarray(np.asarray(dts, dtype=np.float64))
    out = torch.zeros_like(W0)
    _lib.check(_lib.lib().dfgks_adjoint_steps(sol._h, _ptr(W0), int(dts.size), dts.ctypes.data_as(C.POINTER(C.c_double)),
                                              int(flux), int(ckpt_every), _ptr(WTb), _ptr(out)), "dfgks_adjoint_steps")
    return out


def forward_checkpointed(sol: "Solver", W0, nsteps: int, ckpt_every: int = 10, dts=None, flux=None):
    """Set the state to W0 and advance nsteps S2O4 steps (CFL dt unless dts is given), keeping
    checkpoints for adjoint_checkpointed (dfgks_forward_checkpointed).  Returns the step sizes."""
    flux = sol.settings.flux if flux is None else flux
    W0 = _dev(W0).contiguous()
    out = np.zeros(int(nsteps))
    dp = None
    if dts is not None:
        dts = np.ascontiguousarray(np.asarray(dts, dtype=np.float64))
        assert dts.size == nsteps
        dp = dts.ctypes.data_as(C.POINTER(C.c_double))
    _lib.check(_lib.lib().dfgks_forward_checkpointed(sol._h, _ptr(W0), int(nsteps), dp, int(flux), int(ckpt_every),
                                                     out.ctypes.data_as(C.POINTER(C.c_double))),
               "dfgks_forward_checkpointed")
    return out


def adjoint_checkpointed(sol: "Solver", WT_bar) -> torch.Tensor:
    """(dW^n/dW0)^T WT_bar through the last forward_checkpointed (dfgks_adjoint_checkpointed)."""
    WTb = _dev(WT_bar).contiguous()
    out = torch.zeros_like(WTb)
    _lib.check(_lib.lib().dfgks_adjoint_checkpointed(sol._h, _ptr(WTb), _ptr(out)), "dfgks_adjoint_checkpointed")
    return out


class GKSRun(torch.autograd.Function):
    """W^n = n S2O4 steps of the CUDA solver from W0 (CFL step sizes); the forward pass keeps a
    checkpoint every ckpt_every steps and the backward pass is the hand-written adjoint with
    checkpointed recompute (dfgks_forward_checkpointed / dfgks_adjoint_checkpointed).  alpha^0 comes
    from W0 and the alpha sequence, step sizes and branch decisions of the forward trajectory are
    held fixed.  The solver handle must not be stepped or reset between forward and backward."""

    @staticmethod
    def forward(ctx, W0, sol, nsteps, ckpt_every=10):
        ctx.dts = forward_checkpointed(sol, W0.detach(), int(nsteps), int(ckpt_every))
        ctx.sol = sol
        W, _, _, _ = sol.get_state(device=True)
        return W

    @staticmethod
    def backward(ctx, WT_bar):
        return adjoint_checkpointed(ctx.sol, WT_bar), None, None, None
