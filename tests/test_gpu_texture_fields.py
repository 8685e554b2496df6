"""Per-atom external fields and on-device texture diagnostics against the oracle."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from oracle import texture as T
from paper_2606_14073_gb300 import nep_params, spinlat as S, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def params():
    return nep_params.load()


@pytest.fixture(scope="module")
def model(params):
    return O.Model(params)


def _stripe_field(pos, box, values=(0.0, 0.05, 0.1, 0.15)):
    """B_z stepping along x through len(values) equal segments."""
    seg = np.clip((pos[:, 0] / box[0] * len(values)).astype(int), 0, len(values) - 1)
    b = np.zeros((len(pos), 3))
    b[:, 2] = np.asarray(values)[seg]
    return b


def test_per_atom_field_evaluation_and_trajectory(params, model):
    wl = W.fege_small()
    rng = np.random.default_rng(5)
    Ba = rng.normal(0, 0.4, (wl.n, 3))
    B = (0.0, 0.0, 0.1)
    s = S.system_from_workload(wl, params)
    s.set_atom_fields(Ba)
    s.step(0, 1.0, 0.0, B)
    r = s.energy_forces_fields()
    st = s.get_state()
    ref = O.evaluate(model, st["positions"], st["spins"], wl.species, wl.box, wl.periodic, B, B_atoms=Ba)
    assert abs(r["E"] - ref["E"]) <= 1e-10 * abs(ref["E"])
    assert np.abs(r["H"] - ref["H"]).max() <= 1e-10 * np.abs(ref["H"]).max()
    o = O.State(st["positions"], st["velocities"], st["spins"], wl.species, wl.box, wl.periodic)
    o.F, o.H, o.have_fh = st["forces"].copy(), st["fields"].copy(), True
    s.step(20, 1.0, 300.0, B)
    O.run(model, o, 20, 1.0, 300.0, B, seed=wl.seed, B_atoms=Ba)
    g = s.get_state()
    d = g["positions"] - o.pos
    d -= wl.box * np.rint(d / wl.box)
    assert np.abs(d).max() < 1e-9 and np.abs(g["spins"] - o.spin).max() < 1e-9
    s.destroy()


def test_setting_the_field_after_graph_capture_takes_effect(params):
    wl = W.fege_small()
    Ba = _stripe_field(wl.positions, wl.box, values=(0.0, 2.0, 4.0, 6.0))
    runs = []
    for spg in (5, 0):
        s = S.system_from_workload(wl, params, steps_per_graph=spg)
        s.step(10, 1.0, 100.0, (0, 0, 0))
        s.set_atom_fields(Ba)
        s.step(10, 1.0, 100.0, (0, 0, 0))
        s.set_atom_fields(None)
        s.step(5, 1.0, 100.0, (0, 0, 0))
        runs.append(s.get_state())
        s.destroy()
    for k in ("positions", "velocities", "spins"):
        assert np.array_equal(runs[0][k], runs[1][k]), k


@pytest.mark.parametrize("normal,cell", [(2, 4.7), (2, 3.1), (0, 4.0)])
def test_texture_matches_oracle(params, normal, cell):
    wl = W.fege_slab_helix(10, 8, 3, seed=11)
    rng = np.random.default_rng(17)
    spins = W.random_unit_vectors(rng, wl.n)
    s = S.System(wl.positions, spins, wl.box, wl.periodic, wl.species, params, wl.velocities)
    s.step(3, 1.0, 160.0, (0, 0, 0))
    m, q = s.texture(normal, cell)
    st = s.get_state()
    mo, qo = T.texture(st["positions"], st["spins"], wl.box, wl.periodic, normal, cell)
    assert m.shape == mo.shape
    assert np.abs(m - mo).max() < 1e-10
    assert abs(q - qo) < 1e-8
    s.destroy()


def test_film_skyrmion_has_unit_charge(params):
    wl = W.fege_slab_helix(24, 24, 2, seed=12)
    c = wl.box[:2] / 2
    d = wl.positions[:, :2] - c
    r = np.hypot(d[:, 0], d[:, 1])
    R = 9 * 4.70
    th = np.where(r < R, math.pi * r / R, math.pi)
    ph = np.arctan2(d[:, 1], d[:, 0])
    spins = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    s = S.System(wl.positions, spins, wl.box, wl.periodic, wl.species, params)
    m, q = s.texture(2, 4.70)
    assert q == pytest.approx(1.0, abs=1e-9)
    assert np.allclose(np.linalg.norm(m, axis=2), 1.0)
    s.destroy()
