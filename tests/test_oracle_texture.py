"""Pins of the texture oracle (coarse-grained magnetisation, lattice topological charge)
and of the per-atom external field in the oracle's Zeeman term.

The charge is pinned by closed forms: the continuum charge of a compact skyrmion
profile (+1 for a core-up, far-down texture of vorticity +1; -1 for the antiskyrmion
or the reversed texture; additive for two textures), which the Berg-Luescher lattice
charge reproduces exactly (to rounding) on a periodic grid with a uniform far field;
zero for uniform and helical states.  The coarse-graining is pinned against brute
force; the per-atom field against the energy it defines (finite differences)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from oracle import texture as T
from paper_2606_14073_gb300 import workloads as W


def _grid_atoms(na, nb, cell=4.7):
    """One atom at the centre of every in-plane cell of a one-layer film (normal z)."""
    ia, ib = np.meshgrid(np.arange(na), np.arange(nb))
    pos = np.stack([(ia.ravel() + 0.5) * cell, (ib.ravel() + 0.5) * cell, np.full(ia.size, 5.0)], 1)
    box = np.array([na * cell, nb * cell, 10.0])
    return pos, box


def _skyrmion(pos, centre, R, vort=1, core=1.0):
    """Compact profile: polar angle theta = pi r / R inside R, pi outside; azimuth vort*phi."""
    d = pos[:, :2] - centre
    r = np.hypot(d[:, 0], d[:, 1])
    th = np.where(r < R, math.pi * r / R, math.pi)
    ph = vort * np.arctan2(d[:, 1], d[:, 0])
    s = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    return core * s


PER = np.array([1, 1, 0], np.int32)


def test_uniform_and_helix_have_zero_charge():
    pos, box = _grid_atoms(40, 30)
    m, q = T.texture(pos, np.tile([0.3, 0.4, math.sqrt(0.75)], (len(pos), 1)), box, PER)
    assert q == pytest.approx(0.0, abs=1e-12)
    ph = 2 * math.pi * pos[:, 0] / box[0] * 2
    helix = np.stack([np.zeros_like(ph), np.cos(ph), np.sin(ph)], 1)
    assert T.texture(pos, helix, box, PER)[1] == pytest.approx(0.0, abs=1e-12)


@pytest.mark.parametrize("vort,core,expected", [(1, 1.0, 1.0), (-1, 1.0, -1.0), (1, -1.0, -1.0), (2, 1.0, 2.0)])
def test_compact_skyrmion_charge_is_the_continuum_value(vort, core, expected):
    pos, box = _grid_atoms(64, 64)
    spin = _skyrmion(pos, box[:2] / 2, R=18 * 4.7, vort=vort, core=core)
    q = T.texture(pos, spin, box, PER)[1]
    assert q == pytest.approx(expected, abs=1e-9)


def test_charge_is_additive_and_survives_open_edges():
    pos, box = _grid_atoms(96, 48)
    s1 = _skyrmion(pos, np.array([24 * 4.7, 24 * 4.7]), R=15 * 4.7)
    s2 = _skyrmion(pos, np.array([72 * 4.7, 24 * 4.7]), R=15 * 4.7)
    inside1 = np.hypot(*(pos[:, :2] - [24 * 4.7, 24 * 4.7]).T) < 15 * 4.7
    spin = np.where(inside1[:, None], s1, s2)
    assert T.texture(pos, spin, box, PER)[1] == pytest.approx(2.0, abs=1e-9)
    # a non-periodic grid with the textures inside: the boundary is uniform, nothing is lost
    assert T.texture(pos, spin, box, np.array([0, 0, 0], np.int32))[1] == pytest.approx(2.0, abs=1e-9)


def test_solid_angle_of_an_octant_is_pi_over_2():
    ex, ey, ez = np.eye(3)
    assert T.solid_angle(ex, ey, ez) == pytest.approx(math.pi / 2, abs=1e-14)
    assert T.solid_angle(ex, ez, ey) == pytest.approx(-math.pi / 2, abs=1e-14)


def test_coarse_graining_against_brute_force():
    rng = np.random.default_rng(3)
    box = np.array([20.0, 15.0, 8.0])
    pos = rng.uniform(0, 1, (300, 3)) * box
    spin = W.random_unit_vectors(rng, 300)
    m = T.magnetisation_map(pos, spin, box, PER, normal=2, cell=4.0)
    nb, na = m.shape[:2]
    assert (na, nb) == (5, 3)
    for j in range(nb):
        for i in range(na):
            sel = (np.floor(pos[:, 0] / (box[0] / na)) == i) & (np.floor(pos[:, 1] / (box[1] / nb)) == j)
            v = spin[sel].sum(0)
            assert np.allclose(m[j, i], v / np.linalg.norm(v), atol=1e-14)


def test_per_atom_field_enters_energy_and_field(model):
    wl = W.fege_small()
    rng = np.random.default_rng(9)
    Ba = rng.normal(0, 0.3, (wl.n, 3))
    B = np.array([0.0, 0.1, 0.2])
    r0 = O.evaluate(model, wl.positions, wl.spins, wl.species, wl.box, wl.periodic, B)
    r1 = O.evaluate(model, wl.positions, wl.spins, wl.species, wl.box, wl.periodic, B, B_atoms=Ba)
    mu = np.asarray(model.moment)[wl.species] * O.MUB
    assert r1["E"] - r0["E"] == pytest.approx(-(mu[:, None] * Ba * wl.spins).sum(), rel=1e-12, abs=1e-12)
    assert np.allclose(r1["H"] - r0["H"], mu[:, None] * Ba, rtol=0, atol=1e-13)
    assert np.array_equal(r1["F"], r0["F"])
    # the field is minus the spin gradient of the energy, per-atom part included
    h = 1e-6
    for i in (3, 200):
        for c in range(3):
            sp, sm = wl.spins.copy(), wl.spins.copy()
            sp[i, c] += h
            sm[i, c] -= h
            ep = O.evaluate(model, wl.positions, sp, wl.species, wl.box, wl.periodic, B, B_atoms=Ba)["E"]
            em = O.evaluate(model, wl.positions, sm, wl.species, wl.box, wl.periodic, B, B_atoms=Ba)["E"]
            assert -(ep - em) / (2 * h) == pytest.approx(r1["H"][i, c], rel=1e-6, abs=1e-9)
    sub = O.evaluate_subset(model, wl.positions, wl.spins, wl.species, wl.box, wl.periodic, [3, 200], B, B_atoms=Ba)
    assert np.allclose(sub["H"], r1["H"][[3, 200]], rtol=0, atol=1e-12)
