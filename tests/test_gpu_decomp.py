"""One problem split into blocks with halo exchange (dfgks_decomp_*) against the undivided mesh.

Every ghost cell of a block holds what the whole mesh's ghost fill puts there (halo copies in two
passes, boundary conditions on the mesh's sides) and each cell's arithmetic is the same, so the
decomposed run must reproduce the undivided CUDA run bit for bit, and through it the oracle."""
import numpy as np
import pytest

import oracle
from paper_2402_10914_gb300 import inputs as I
from tests.parity_util import comp_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def whole(w, nsteps, t_end=0.0):
    from paper_2402_10914_gb300.solver import Solver
    with Solver(w.settings) as s:
        s.set_ic(w.W0)
        done, _ = s.step(nsteps, t_end=t_end)
        W, a, t, step = s.get_state()
        cnt = s.counters()
    return done, W, a, t, step, cnt


def split(w, px, py, nsteps, t_end=0.0):
    from paper_2402_10914_gb300.solver import DecompSolver
    with DecompSolver(w.settings, px, py) as d:
        d.set_ic(w.W0)
        done = d.step(nsteps, t_end=t_end)
        W, a, t, step = d.get_state()
        st = d.status()
    return done, W, a, t, step, st


CASES = {
    "quadrants_outflow": lambda: I.quadrants(64, seed=3),
    "rough_periodic_lf": lambda: I.random_rough(30, 24, seed=5, bc=(I.PERIODIC,) * 4, flux=I.LF, time_limiter=0),
    "rough_periodic_gks": lambda: I.random_rough(30, 24, seed=6, bc=(I.PERIODIC,) * 4, flux=I.GKS),
    "blast_walls": lambda: I.blast(48),
    "mixed_bc": lambda: I.random_smooth(27, 33, seed=7, bc=(I.PERIODIC, I.PERIODIC, I.REFLECT, I.OUTFLOW)),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("px,py", [(2, 1), (1, 2), (2, 2), (3, 2)])
def test_decomposed_run_equals_the_whole_mesh_bitwise(name, px, py):
    w = CASES[name]()
    ref = whole(w, 6)
    got = split(w, px, py, 6)
    assert got[0] == ref[0] == 6
    assert np.array_equal(got[1], ref[1]), (name, px, py, comp_rel_err(got[1], ref[1]))
    assert np.array_equal(got[2], ref[2])
    assert got[3] == ref[3] and got[4] == ref[4]
    st, cnt = got[5], ref[5]
    assert st["err"] == 0
    # the counters count reconstructions performed; blocks recompute the face lines and faces on
    # their shared boundaries (and the padding lines of the tangential stencil), so never fewer
    for k in ("df_normal", "df_tangential", "fallbacks"):
        assert st[k] >= cnt[k], (k, st[k], cnt[k])


def test_decomposed_one_step_against_the_oracle():
    w = I.quadrants(96, seed=3)
    done, W, a, t, step, _ = split(w, 3, 2, 1)
    rc, Wo, ao, to, _, _ = oracle.run(w.settings, w.W0, oracle.alpha0(w.settings, w.W0), 1)
    assert rc == 0 and done == 1 and abs(t - to) <= 1e-15 * to
    assert comp_rel_err(W, Wo) <= 1e-12
    assert comp_rel_err(a[None], ao[None], floor_frac=1e-12) <= 1e-11


def test_decomposed_run_to_end_time():
    w = I.quadrants(48, seed=4, t_end=0.05)
    ref = whole(w, 1000, t_end=w.t_end)
    got = split(w, 2, 3, 1000, t_end=w.t_end)
    assert got[3] == ref[3] == w.t_end and got[4] == ref[4]
    assert np.array_equal(got[1], ref[1])


def test_decomposed_positivity_failure_reports_the_whole_mesh_cell():
    # seed 2 loses positivity at step 12 (near-vacuum rarefaction): the decomposed run stops at
    # the same step with the same last good state and names the same cell of the whole mesh
    from paper_2402_10914_gb300 import _lib
    from paper_2402_10914_gb300.solver import DecompSolver, Solver
    w = I.quadrants(64, seed=2, t_end=0.25)
    with Solver(w.settings) as s:
        s.set_ic(w.W0)
        with pytest.raises(_lib.DfgksError):
            s.step(40, t_end=w.t_end)
        Wr, ar, tr, sr = s.get_state()
        fstep, fi, fj = s.last_error()
    with DecompSolver(w.settings, 2, 2) as d:
        d.set_ic(w.W0)
        with pytest.raises(_lib.DfgksError) as e:
            d.step(40, t_end=w.t_end)
        assert e.value.status == _lib.ENONPOS
        W, a, t, step = d.get_state()
        st = d.status()
    assert step == sr and np.array_equal(W, Wr)
    assert (st["fail_i"], st["fail_j"]) == (fi, fj)
