"""Longitudinal moment mode on the GPU against the FP64 oracle (variable |S_i|, Landau
onsite energy, Langevin form with longitudinal damping; the reading is stated in
include/spinlat.h at sl_set_longitudinal)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_14073_gb300 import nep_params, spinlat as S, workloads as W

pytestmark = pytest.mark.gpu

LANDAU = [[-0.2, 0.08], [-0.15, 0.06]]


@pytest.fixture(scope="module")
def params():
    return nep_params.load()


@pytest.fixture(scope="module")
def model(params):
    return O.Model(params, landau=LANDAU)


def _scaled(wl, seed=11):
    return wl.spins * np.random.default_rng(seed).uniform(0.7, 1.4, size=(wl.n, 1))


def _long_system(params, wl, alpha, spins=None, **kw):
    s = S.system_from_workload(wl, params, **kw)
    s.set_longitudinal(True, alpha, LANDAU)
    if spins is not None:
        st = s.get_state()
        s.set_state(st["positions"], st["velocities"], spins)
    return s


def _close(g, o, wl, tol):
    d = g["positions"] - o.pos
    d -= wl.box * np.rint(d / wl.box)
    assert np.abs(d).max() < tol
    assert np.abs(g["spins"] - o.spin).max() < tol
    assert np.abs(g["velocities"] - o.vel).max() < tol


def test_energy_forces_fields_at_unequal_lengths(params, model):
    wl = W.fege_small()
    Sx = _scaled(wl)
    s = _long_system(params, wl, 0.2, spins=Sx)
    g = s.get_state()
    assert np.array_equal(g["spins"], Sx)   # lengths are state in this mode
    r = s.energy_forces_fields(want_virial=False)
    ref = O.evaluate(model, wl.positions, Sx, wl.species, wl.box, wl.periodic)
    assert abs(r["E"] - ref["E"]) <= 1e-10 * abs(ref["E"])
    assert np.abs(r["F"] - ref["F"]).max() <= 1e-10 * np.abs(ref["F"]).max()
    assert np.abs(r["H"] - ref["H"]).max() <= 1e-10 * np.abs(ref["H"]).max()
    s.destroy()


def test_trajectory_matches_oracle(params, model):
    wl = W.fege_small()
    B = (0.0, 0.0, 0.5)
    s = _long_system(params, wl, 0.2, steps_per_graph=10)
    st = s.get_state()
    o = O.State(st["positions"], st["velocities"], st["spins"], wl.species, wl.box, wl.periodic)
    # the carried forces and fields (evaluated before the first step's field was given)
    o.F, o.H, o.have_fh = st["forces"].copy(), st["fields"].copy(), True
    for chunk in (1, 4, 15):
        s.step(chunk, 1.0, 300.0, B)
        O.run(model, o, chunk, 1.0, 300.0, B, seed=wl.seed, longitudinal=True, alpha_long=0.2)
        _close(s.get_state(), o, wl, 1e-9)
    lengths = np.linalg.norm(s.get_state()["spins"], axis=1)
    assert np.abs(lengths - 1).max() > 1e-2   # the lengths do move
    s.destroy()


def test_mixed_stays_close_to_fp64(params):
    wl = W.fege_small()
    m = _long_system(params, wl, 0.1, precision=S.SL_PREC_MIXED)
    d = _long_system(params, wl, 0.1, precision=S.SL_PREC_FP64)
    m.step(20, 1.0, 300.0, (0, 0, 0.2))
    d.step(20, 1.0, 300.0, (0, 0, 0.2))
    assert np.abs(m.get_state()["spins"] - d.get_state()["spins"]).max() < 1e-3
    m.destroy()
    d.destroy()


@pytest.mark.parametrize("prec", [S.SL_PREC_FP64, S.SL_PREC_MIXED])
def test_graphs_and_resume_are_bit_identical(params, prec):
    wl = W.fege_small()
    a = _long_system(params, wl, 0.15, precision=prec, steps_per_graph=5)
    b = _long_system(params, wl, 0.15, precision=prec, steps_per_graph=0)
    a.step(15, 1.0, 300.0, (0, 0, 0.3))
    b.step(7, 1.0, 300.0, (0, 0, 0.3))
    # checkpoint b and resume it in a fresh system
    ck = b.get_state()
    c = _long_system(params, wl, 0.15, precision=prec, steps_per_graph=0)
    c.set_state(ck["positions"], ck["velocities"], ck["spins"], forces=ck["forces"], fields=ck["fields"],
                step=ck["step"], ref_positions=ck["ref_positions"])
    c.step(8, 1.0, 300.0, (0, 0, 0.3))
    ga, gc = a.get_state(), c.get_state()
    for k in ("positions", "velocities", "spins", "forces", "fields"):
        assert np.array_equal(ga[k], gc[k]), k
    for x in (a, b, c):
        x.destroy()


def test_replica_in_batch_matches_alone(params):
    wls = [W.fege_cube(c, seed=130 + c, replica=c) for c in (4, 5)]
    alone = []
    for w in wls:
        s = _long_system(params, w, 0.1, replica=w.seed - W.LANGEVIN_SEED0)
        s.step(12, 1.0, 200.0, (0, 0, 0.2))
        alone.append(s.get_state())
        s.destroy()
    syss = [_long_system(params, w, 0.1, replica=w.seed - W.LANGEVIN_SEED0) for w in wls]
    b = S.Batch(syss)
    b.step(12, 1.0, 200.0, (0, 0, 0.2))
    for s, ref in zip(syss, alone):
        g = s.get_state()
        for key in ("positions", "velocities", "spins", "forces", "fields"):
            assert np.array_equal(g[key], ref[key]), key
    b.destroy()
    for s in syss:
        s.destroy()


def test_leaving_the_mode_normalises_and_unit_mode_resumes(params):
    wl = W.fege_small()
    s = _long_system(params, wl, 0.3)
    s.step(10, 1.0, 300.0, (0, 0, 0))
    s.set_longitudinal(False)
    g = s.get_state()
    assert np.abs(np.linalg.norm(g["spins"], axis=1) - 1).max() < 1e-14
    s.step(5, 1.0, 300.0, (0, 0, 0))
    assert np.abs(np.linalg.norm(s.get_state()["spins"], axis=1) - 1).max() < 1e-14
    s.destroy()


def test_refused_with_midpoint_and_bad_alpha(params):
    wl = W.fege_small()
    s = S.system_from_workload(wl, params, midpoint_iters=3)
    with pytest.raises(S.SpinlatError) as e:
        s.set_longitudinal(True, 0.1, LANDAU)
    assert e.value.code == S.SL_EINVAL
    s.destroy()
    s = S.system_from_workload(wl, params)
    with pytest.raises(S.SpinlatError):
        s.set_longitudinal(True, -0.5, LANDAU)
    s.destroy()
