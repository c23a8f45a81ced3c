"""The block decomposition's halo bookkeeping with one block per rank, on the CPU: two gloo ranks on
127.0.0.1, as torchrun would start them.

Each rank holds one block of a seeded field as a ghosted array and fills its ghost layers the way
the decomposed solver does on one device, in two passes (ghost columns of the interior rows, then
ghost rows including the ghost columns), with the windows the library's plan gives
(dfgks_decomp_plan / dfgks_decomp_halo): sides on the mesh boundary by their boundary condition,
shared sides by receiving the neighbouring rank's window, sent point to point.  The result must
equal the whole mesh's ghost fill computed by the oracle, window by window."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
G = 3


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def boundary_fill(U, nx, ny, side, bc):
    """One side's ghost layers of a ghosted block U [5][ny+2G][nx+2G] (W and alpha) by a boundary
    condition: 0 periodic within the block, 1 zero gradient, 2 mirror with the normal momentum
    negated.  x sides fill the interior rows, y sides all columns."""
    for g in range(G):
        if side == 0:
            d, s = G - 1 - g, {0: G + nx - 1 - g, 1: G, 2: G + g}[bc]
            U[:, G:G + ny, d] = U[:, G:G + ny, s]
            if bc == 2:
                U[1, G:G + ny, d] *= -1.0
        elif side == 1:
            d, s = G + nx + g, {0: G + g, 1: G + nx - 1, 2: G + nx - 1 - g}[bc]
            U[:, G:G + ny, d] = U[:, G:G + ny, s]
            if bc == 2:
                U[1, G:G + ny, d] *= -1.0
        elif side == 2:
            d, s = G - 1 - g, {0: G + ny - 1 - g, 1: G, 2: G + g}[bc]
            U[:, d, :] = U[:, s, :]
            if bc == 2:
                U[2, d, :] *= -1.0
        else:
            d, s = G + ny + g, {0: G + g, 1: G + ny - 1, 2: G + ny - 1 - g}[bc]
            U[:, d, :] = U[:, s, :]
            if bc == 2:
                U[2, d, :] *= -1.0


def rank_main(rank, ws, port, case, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    from paper_2402_10914_gb300 import inputs as I
    from paper_2402_10914_gb300.solver import block_plan, halo_window
    nx, ny, px, py, bc = case
    s = I.Settings(nx=nx, ny=ny, bc=bc)
    rng = np.random.default_rng(11)
    W = rng.uniform(0.5, 2.0, (4, ny, nx))
    alpha = rng.uniform(0.0, 1.0, (ny, nx))
    plans = [block_plan(s, px, py, b) for b in range(ws)]
    wins = [[halo_window(s, px, py, b, side) for side in range(4)] for b in range(ws)]
    p = plans[rank]
    bnx, bny = p["i1"] - p["i0"], p["j1"] - p["j0"]
    U = np.full((5, bny + 2 * G, bnx + 2 * G), np.nan)
    U[:4, G:G + bny, G:G + bnx] = W[:, p["j0"]:p["j1"], p["i0"]:p["i1"]]
    U[4, G:G + bny, G:G + bnx] = alpha[p["j0"]:p["j1"], p["i0"]:p["i1"]]
    for ps in range(2):
        sides = (0, 1) if ps == 0 else (2, 3)
        for side in sides:
            if p["neighbour"][side] < 0:
                boundary_fill(U, bnx, bny, side, p["bc"][side])
        # send every window another block needs from this one, receive this block's windows
        reqs, recv, keep = [], [], []
        for b in range(ws):
            for side in sides:
                hw = wins[b][side]
                if hw["neighbour"] == rank and b != rank:
                    src = U[:, G + hw["sj"]:G + hw["sj"] + hw["h"], G + hw["si"]:G + hw["si"] + hw["w"]]
                    keep.append(torch.from_numpy(np.ascontiguousarray(src)))
                    reqs.append(dist.isend(keep[-1], dst=b, tag=10 * b + side))
        for side in sides:
            hw = wins[rank][side]
            if hw["neighbour"] < 0:
                continue
            buf = torch.empty((5, hw["h"], hw["w"]), dtype=torch.float64)
            if hw["neighbour"] == rank:
                buf = torch.from_numpy(U[:, G + hw["sj"]:G + hw["sj"] + hw["h"], G + hw["si"]:G + hw["si"] + hw["w"]].copy())
            else:
                dist.recv(buf, src=hw["neighbour"], tag=10 * rank + side)
            recv.append((hw, buf.numpy()))
        for r in reqs:
            r.wait()
        for hw, a in recv:
            U[:, G + hw["dj"]:G + hw["dj"] + hw["h"], G + hw["di"]:G + hw["di"] + hw["w"]] = a
    out[rank] = (p, U)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("case", [
    (10, 7, 2, 1, (0, 0, 2, 1)),      # split in x, periodic in x (both neighbours are the other rank), walls / outflow in y
    (9, 12, 1, 2, (2, 1, 0, 0)),      # split in y, periodic in y, wall / outflow in x
    (11, 8, 2, 1, (1, 1, 1, 1)),      # split in x, outflow all round
    (8, 13, 1, 2, (2, 2, 2, 2)),      # split in y, walls all round
])
def test_two_ranks_fill_ghosts_like_the_whole_mesh(case):
    import oracle
    sys.path.insert(0, ROOT)
    from paper_2402_10914_gb300 import inputs as I
    ws = 2
    out = mp.Manager().dict()
    mp.spawn(rank_main, args=(ws, free_port(), case, out), nprocs=ws, join=True)
    nx, ny, px, py, bc = case
    s = I.Settings(nx=nx, ny=ny, bc=bc)
    rng = np.random.default_rng(11)
    W = rng.uniform(0.5, 2.0, (4, ny, nx))
    alpha = rng.uniform(0.0, 1.0, (ny, nx))
    Wg, ag = oracle.fill_ghosts(s, W, alpha)
    ref = np.concatenate([Wg, ag[None]])
    for rank in range(ws):
        p, U = out[rank]
        win = ref[:, p["j0"]:p["j1"] + 2 * G, p["i0"]:p["i1"] + 2 * G]
        assert not np.isnan(U).any(), rank
        assert np.array_equal(U, win), (rank, np.argwhere(U != win)[:5])


def test_plan_refuses_blocks_below_the_stencil_width():
    sys.path.insert(0, ROOT)
    from paper_2402_10914_gb300 import _lib, inputs as I
    from paper_2402_10914_gb300.solver import block_plan
    with pytest.raises(_lib.DfgksError):
        block_plan(I.Settings(nx=5, ny=8), 2, 1, 0)           # 2 cells in a split direction
    with pytest.raises(_lib.DfgksError):
        block_plan(I.Settings(nx=8, ny=8, time_scheme=I.SSPRK3), 2, 1, 0)
    p = block_plan(I.Settings(nx=7, ny=8), 2, 1, 1)
    assert (p["i0"], p["i1"], p["j0"], p["j1"]) == (3, 7, 0, 8)
