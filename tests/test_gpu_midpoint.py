"""Self-consistent midpoint spin update on the GPU against the FP64 oracle.

Both sides implement the reading stated in include/spinlat.h (Section 5.1.3): lattice
midpoint r_mid = (r_n + r_{n+1})/2, midpoint spins M_m = (S_n + X_m)/|S_n + X_m|, field at
(r_mid, M_m), G_m = Rot(S_n, omega(M_m, H_m + eta) dt), stop at max |G - X| < tol or the
cap, optional regularised Anderson mixing; forces and fields then at the end state."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_14073_gb300 import nep_params, spinlat as S, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def params():
    return nep_params.load()


@pytest.fixture(scope="module")
def model(params):
    return O.Model(params)


def _pair(params, wl, **mid):
    s = S.system_from_workload(wl, params, steps_per_graph=mid.pop("steps_per_graph", 10), **mid)
    st = s.get_state()
    o = O.State(st["positions"], st["velocities"], st["spins"], wl.species, wl.box, wl.periodic)
    o.F, o.H, o.have_fh = st["forces"].copy(), st["fields"].copy(), True
    return s, o


def _close(g, o, wl, tol):
    d = g["positions"] - o.pos
    d -= wl.box * np.rint(d / wl.box)
    assert np.abs(d).max() < tol
    assert np.abs(g["spins"] - o.spin).max() < tol
    assert np.abs(g["velocities"] - o.vel).max() < tol
    assert np.abs(np.linalg.norm(g["spins"], axis=1) - 1).max() < 1e-14


def test_fixed_iteration_count_matches_oracle(params, model):
    """Cap 3, tolerance 0 (every step runs the cap): 20 Langevin steps at 300 K in a field."""
    wl = W.fege_small()
    B = (0.0, 0.0, 0.5)
    s, o = _pair(params, wl, midpoint_iters=3, midpoint_tol=0.0)
    for chunk in (1, 4, 15):
        s.step(chunk, 1.0, 300.0, B)
        O.run(model, o, chunk, 1.0, 300.0, B, seed=wl.seed, midpoint_iters=3, midpoint_tol=0.0)
        _close(s.get_state(), o, wl, 1e-9)
    assert s.midpoint_evaluations() == 3 * 20
    s.destroy()


def test_tolerance_stop_matches_oracle(params, model):
    wl = W.fege_small()
    B = (0.0, 0.0, 0.2)
    s, o = _pair(params, wl, midpoint_iters=30, midpoint_tol=1e-10)
    s.step(12, 1.0, 300.0, B)
    O.run(model, o, 12, 1.0, 300.0, B, seed=wl.seed, midpoint_iters=30, midpoint_tol=1e-10)
    _close(s.get_state(), o, wl, 1e-9)
    ev = s.midpoint_evaluations()
    assert ev == o.last_iterations and 12 < ev < 12 * 30, (ev, o.last_iterations)
    s.destroy()


def test_anderson_matches_oracle_and_saves_evaluations(params, model):
    wl = W.fege_small()
    B = (0.0, 0.0, 0.0)
    kw = dict(midpoint_iters=40, midpoint_tol=1e-11)
    s, o = _pair(params, wl, anderson_depth=3, anderson_reg=1e-10, **kw)
    p, _ = _pair(params, wl, **kw)
    s.step(5, 3.0, 0.0, B)
    p.step(5, 3.0, 0.0, B)
    O.run(model, o, 5, 3.0, 0.0, B, seed=wl.seed, anderson_depth=3, anderson_reg=1e-10, **kw)
    g = s.get_state()
    _close(g, o, wl, 1e-8)
    # the accelerated and the plain iteration stop at the same fixed point
    assert np.abs(g["spins"] - p.get_state()["spins"]).max() < 1e-9
    assert s.midpoint_evaluations() < p.midpoint_evaluations()
    s.destroy()
    p.destroy()


def test_loose_tolerance_stops_after_one_evaluation(params):
    wl = W.fege_small()
    s = S.system_from_workload(wl, params, midpoint_iters=8, midpoint_tol=1.0)
    s.step(7, 1.0, 300.0, (0, 0, 0))
    assert s.midpoint_evaluations() == 7
    s.destroy()


@pytest.mark.parametrize("prec", [S.SL_PREC_FP64, S.SL_PREC_MIXED])
def test_graphs_match_direct_launches(params, prec):
    wl = W.fege_small()
    kw = dict(precision=prec, midpoint_iters=6, midpoint_tol=1e-9, anderson_depth=2)
    a = S.system_from_workload(wl, params, steps_per_graph=5, **kw)
    b = S.system_from_workload(wl, params, steps_per_graph=0, **kw)
    a.step(15, 1.0, 300.0, (0, 0, 0.3))
    b.step(15, 1.0, 300.0, (0, 0, 0.3))
    ga, gb = a.get_state(), b.get_state()
    for k in ("positions", "velocities", "spins", "forces", "fields"):
        assert np.array_equal(ga[k], gb[k]), k
    assert a.midpoint_evaluations() == b.midpoint_evaluations()
    a.destroy()
    b.destroy()


def test_mixed_midpoint_stays_close_to_fp64(params):
    wl = W.fege_small()
    kw = dict(midpoint_iters=10, midpoint_tol=1e-7)
    m = S.system_from_workload(wl, params, precision=S.SL_PREC_MIXED, **kw)
    d = S.system_from_workload(wl, params, precision=S.SL_PREC_FP64, **kw)
    m.step(20, 1.0, 300.0, (0, 0, 0))
    d.step(20, 1.0, 300.0, (0, 0, 0))
    gm, gd = m.get_state(), d.get_state()
    assert np.abs(gm["spins"] - gd["spins"]).max() < 1e-3
    assert np.abs(np.linalg.norm(gm["spins"], axis=1) - 1).max() < 1e-14
    m.destroy()
    d.destroy()


def test_midpoint_replicas_in_a_batch_match_alone(params):
    wls = [W.fege_cube(c, seed=120 + c, replica=c) for c in (4, 5)]
    kw = dict(midpoint_iters=5, midpoint_tol=1e-8, anderson_depth=2)
    alone = []
    for w in wls:
        s = S.system_from_workload(w, params, replica=w.seed - W.LANGEVIN_SEED0, **kw)
        s.step(12, 1.0, 200.0, (0, 0, 0.2))
        alone.append((s.get_state(), s.midpoint_evaluations()))
        s.destroy()
    syss = [S.system_from_workload(w, params, replica=w.seed - W.LANGEVIN_SEED0, **kw) for w in wls]
    b = S.Batch(syss)
    b.step(12, 1.0, 200.0, (0, 0, 0.2))
    assert b.graph_launches() == 1
    for s, (ref, ev) in zip(syss, alone):
        g = s.get_state()
        for key in ("positions", "velocities", "spins", "forces", "fields"):
            assert np.array_equal(g[key], ref[key]), key
        assert s.midpoint_evaluations() == ev
    b.destroy()
    for s in syss:
        s.destroy()
