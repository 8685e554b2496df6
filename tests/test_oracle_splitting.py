"""Pins of the oracle's coloured Suzuki-Trotter spin sweep.

The colouring is checked against a brute-force greedy colouring written here from its
definition, and against what it is for: the field on a spin does not change when a spin of
its own colour changes.  The sweep is checked against exact Larmor precession of free spins,
against the dissipation sign and unit length under damping, and for convergence of the
energy error with the time step."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_14073_gb300 import workloads as W

from conftest import variant

RC = 6.0


def _min_image_d2(pos, box, periodic, i):
    d = pos - pos[i]
    for a in range(3):
        if periodic[a]:
            d[:, a] -= box[a] * np.rint(d[:, a] / box[a])
    return (d ** 2).sum(1)


def test_colouring_matches_brute_force_greedy_and_separates_classes():
    wl = W.fege_cube(4)
    col, nc = O.colour(wl.positions, wl.box, wl.periodic, RC)
    ref = np.full(wl.n, -1)
    for i in range(wl.n):
        d2 = _min_image_d2(wl.positions, wl.box, wl.periodic, i)
        nb = np.where((d2 < (2 * RC) ** 2) & (np.arange(wl.n) < i))[0]
        used = set(ref[nb].tolist())
        c = 0
        while c in used:
            c += 1
        ref[i] = c
    assert np.array_equal(col, ref) and nc == ref.max() + 1
    for i in range(0, wl.n, 37):   # no two atoms of one colour closer than 2 rc
        d2 = _min_image_d2(wl.positions, wl.box, wl.periodic, i)
        same = (col == col[i]) & (np.arange(wl.n) != i)
        assert (d2[same] >= (2 * RC) ** 2).all()


def test_field_on_a_spin_ignores_spins_of_its_colour(model):
    wl = W.fege_cube(6)
    col, _ = O.colour(wl.positions, wl.box, wl.periodic, RC)
    i = 100
    same = np.where((col == col[i]) & (np.arange(wl.n) != i))[0]
    d2 = _min_image_d2(wl.positions, wl.box, wl.periodic, i)
    j = same[np.argmin(d2[same])]          # the nearest spin of the same colour
    near = np.where((col != col[i]) & (d2 < 5.0 ** 2) & (np.arange(wl.n) != i))[0][0]
    h0 = O.evaluate(model, wl.positions, wl.spins, wl.species, wl.box, wl.periodic)["H"]
    S = wl.spins.copy()
    S[j] = [0.0, 0.6, 0.8]
    h1 = O.evaluate(model, wl.positions, S, wl.species, wl.box, wl.periodic)["H"]
    assert np.array_equal(h0[i], h1[i])
    # whereas a neighbouring spin (another colour) does reach it
    S = wl.spins.copy()
    S[near] = [0.0, 0.6, 0.8]
    h2 = O.evaluate(model, wl.positions, S, wl.species, wl.box, wl.periodic)["H"]
    assert not np.array_equal(h0[i], h2[i])


def _free_spins(params, n=3, spacing=20.0):
    m = O.Model(variant(params, net=0.0))
    pos = np.stack([np.arange(n) * spacing + 5.0, np.full(n, 5.0), np.full(n, 5.0)], 1)
    box = np.array([n * spacing + 10.0, 10.0, 10.0])
    return m, pos, box, np.array([0, 0, 0], np.int32)


def test_free_spins_precess_exactly(params):
    m, pos, box, per = _free_spins(params)
    S0 = np.array([[0.6, 0.0, 0.8], [0.0, 1.0, 0.0], [0.8, 0.0, -0.6]])
    B = np.array([0.0, 0.0, 50.0])
    st = O.State(pos, np.zeros((3, 3)), S0, np.zeros(3, np.int32), box, per)
    w = 5.7883818060e-5 * 50.0 / 0.6582119569
    O.run(m, st, 40, 0.5, 0.0, B, gamma=0.0, lam=0.0, st_sweep=True)
    t = 20.0
    Rz = np.array([[math.cos(w * t), -math.sin(w * t), 0], [math.sin(w * t), math.cos(w * t), 0], [0, 0, 1]])
    assert np.allclose(st.spin, S0 @ Rz.T, atol=1e-12)


def test_damping_lowers_the_energy_and_keeps_unit_length(model):
    wl = W.fege_cube(4, seed=50)
    st = O.State(wl.positions, wl.velocities * 0.0, wl.spins, wl.species, wl.box, wl.periodic)
    B = (0.0, 0.0, 2.0)
    e = []
    for _ in range(3):
        O.run(model, st, 1, 0.5, 0.0, B, gamma=0.0, lam=0.5, st_sweep=True)
        # lattice frozen in place: zero velocities and forces small over one half step; compare
        # the spin part of the energy at (nearly) fixed positions
        e.append(O.evaluate(model, st.pos, st.spin, st.species, st.box, st.periodic, B)["E"]
                 + O.kinetic_energy(st.vel, st.species, model.mass))
        assert np.abs(np.linalg.norm(st.spin, axis=1) - 1).max() < 1e-14
    assert e[1] < e[0] and e[2] < e[1], e


@pytest.mark.slow
def test_energy_error_converges_with_the_step(model):
    wl = W.fege_cube(4, seed=51, T=50.0)
    err = []
    for dt in (1.0, 0.5):
        st = O.State(wl.positions, wl.velocities, wl.spins, wl.species, wl.box, wl.periodic)
        e0 = O.evaluate(model, st.pos, st.spin, st.species, st.box, st.periodic)["E"] + \
            O.kinetic_energy(st.vel, st.species, model.mass)
        O.run(model, st, int(round(2.0 / dt)), dt, 0.0, (0, 0, 0), gamma=0.0, lam=0.0, st_sweep=True)
        e1 = O.evaluate(model, st.pos, st.spin, st.species, st.box, st.periodic)["E"] + \
            O.kinetic_energy(st.vel, st.species, model.mass)
        err.append(abs(e1 - e0))
    assert err[1] < err[0] / 1.7, err


def test_sweep_options_are_checked(model):
    wl = W.fege_cube(2, seed=52)
    st = O.State(wl.positions, wl.velocities, wl.spins, wl.species, wl.box, wl.periodic)
    with pytest.raises(RuntimeError):
        O.run(model, st, 1, 1.0, 0.0, st_sweep=True, midpoint_iters=2)
    with pytest.raises(RuntimeError):
        O.run(model, st, 1, 1.0, 0.0, st_sweep=True, longitudinal=True, alpha_long=0.1)
