"""Pins of the oracle's self-consistent midpoint spin update (Section 5.1.3).

The reading: the lattice part of the step is unchanged; r_mid = (r_n + r_{n+1})/2 (minimum
image) is the lattice midpoint.  From X_0 = Rot(S_n, omega(S_n, H_n + eta) dt), iterate
M_m = (S_n + X_m)/|S_n + X_m|, H_m = H(r_mid, M_m), G_m = Rot(S_n, omega(M_m, H_m + eta) dt)
until max_i |G_m - X_m| < tol or the cap; S_{n+1} = G_m; forces and fields carried from
(r_{n+1}, S_{n+1}).  Evaluating at the midpoint of both the lattice and the spins keeps the
coupled step time-symmetric (second order); the field at the end-of-step lattice alone
gives a first-order energy error.  The pins check the oracle against things fixed independently of
its code: the exact Larmor precession, the analytic damped precession angle, the
fixed-point equation itself re-evaluated from outside (rotations by scipy), the
geometric convergence of the plain iteration, the accelerated variant reaching the
same fixed point, and second-order energy behaviour."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as O
from paper_2606_14073_gb300 import workloads as W
from tests.conftest import variant


def _free_spins(params, n=1, spacing=20.0):
    p = variant(params, net=0.0)
    m = O.Model(p)
    pos = np.stack([np.arange(n) * spacing + 5.0, np.full(n, 5.0), np.full(n, 5.0)], 1)
    box = np.array([n * spacing + 10.0, 10.0, 10.0])
    return m, pos, box, np.array([0, 0, 0], np.int32)


def _omega(S, Hp, lam):
    """Damped precession vector (H' + lam S x H') / ((1 + lam^2) hbar), row by row."""
    return (Hp + lam * np.cross(S, Hp)) / ((1.0 + lam * lam) * O.HBAR)


def _rot(S, w, dt):
    return Rotation.from_rotvec(w * dt).apply(S)


def test_larmor_precession_exact_with_one_evaluation(params):
    m, pos, box, per = _free_spins(params)
    B = np.array([0.0, 0.0, 50.0])
    st = O.State(pos, np.zeros((1, 3)), [[0.6, 0.0, 0.8]], np.array([0], np.int32), box, per)
    w = O.MUB * 50.0 / O.HBAR
    t = 0.0
    for _ in range(4):
        O.run(m, st, 40, 0.5, 0.0, B, gamma=0.0, lam=0.0, midpoint_iters=6, midpoint_tol=1e-14)
        # omega does not depend on S without damping: the first image is the fixed point
        assert st.last_iterations == 40
        t += 20.0
        ref = np.array([0.6 * math.cos(w * t), 0.6 * math.sin(w * t), 0.8])
        assert np.allclose(st.spin[0], ref, atol=1e-12)


def test_damped_precession_second_order(params):
    m, pos, box, per = _free_spins(params)
    B = np.array([0.0, 0.0, 400.0])
    lam, th0, T_end = 0.2, 2.5, 200.0
    w = O.MUB * 400.0 / O.HBAR
    errs = []
    for dt in (1.0, 0.5, 0.25):
        st = O.State(pos, np.zeros((1, 3)), [[math.sin(th0), 0, math.cos(th0)]], np.array([0], np.int32), box, per)
        O.run(m, st, int(round(T_end / dt)), dt, 0.0, B, gamma=0.0, lam=lam, midpoint_iters=50,
              midpoint_tol=1e-15)
        th = 2 * math.atan(math.tan(th0 / 2) * math.exp(-lam * w * T_end / (1 + lam * lam)))
        errs.append(abs(math.acos(st.spin[0, 2]) - th))
        assert abs(np.linalg.norm(st.spin[0]) - 1) < 1e-14
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.25) and errs[1] / errs[2] == pytest.approx(4.0, rel=0.25)


def _step_from(model, wl, dt, T, B, seed, **mid):
    st = O.State(wl.positions, wl.velocities, wl.spins, wl.species, wl.box, wl.periodic)
    O.run(model, st, 0, dt, T, B, seed=seed)                 # forces and fields of the start state
    start = dict(pos=st.pos.copy(), vel=st.vel.copy(), spin=st.spin.copy(), F=st.F.copy(), H=st.H.copy(),
                 step=st.step)
    O.run(model, st, 1, dt, T, B, seed=seed, **mid)
    return start, st


def test_converged_step_satisfies_the_midpoint_equation(model):
    wl = W.fege_small()
    dt, T, B, seed, lam = 1.0, 300.0, (0.0, 0.0, 0.5), 1234, 0.1
    start, st = _step_from(model, wl, dt, T, B, seed, midpoint_iters=60, midpoint_tol=1e-13)
    assert 1 < st.last_iterations < 60
    # lattice part is that of the predictor-corrector step
    pc = O.State(wl.positions, wl.velocities, wl.spins, wl.species, wl.box, wl.periodic)
    O.run(model, pc, 0, dt, T, B, seed=seed)
    O.run(model, pc, 1, dt, T, B, seed=seed)
    assert np.array_equal(st.pos, pc.pos)
    # the fixed point, evaluated from outside the oracle's integrator
    sig = math.sqrt(2 * lam * O.KB * T * O.HBAR / dt)
    eta = sig * np.array([O.gauss4(start["step"], i, 2, seed, 0)[:3] for i in range(wl.n)])
    S0, S1 = start["spin"], st.spin
    Mid = (S0 + S1) / np.linalg.norm(S0 + S1, axis=1)[:, None]
    d = st.pos - start["pos"]
    d -= wl.box * np.rint(d / wl.box) * wl.periodic
    rmid = start["pos"] + 0.5 * d
    rmid = np.where(wl.periodic.astype(bool), rmid - wl.box * np.floor(rmid / wl.box), rmid)
    Hm = O.evaluate(model, rmid, Mid, wl.species, wl.box, wl.periodic, B)["H"]
    G = _rot(S0, _omega(Mid, Hm + eta, lam), dt)
    assert np.abs(G - S1).max() < 1e-11
    # carried forces and fields are those of the end state
    r = O.evaluate(model, st.pos, st.spin, wl.species, wl.box, wl.periodic, B)
    assert np.allclose(st.F, r["F"], rtol=0, atol=1e-12) and np.allclose(st.H, r["H"], rtol=0, atol=1e-12)
    mass = np.asarray(model.mass)[wl.species][:, None]
    assert np.allclose(st.vel - pc.vel, 0.5 * dt * (st.F - pc.F) / mass * O.ACC, rtol=0, atol=1e-13)


def test_plain_iteration_contracts_geometrically(model):
    wl = W.fege_small()
    args = dict(dt=2.0, T=0.0, B=(0.0, 0.0, 0.0), seed=5)
    _, ref = _step_from(model, wl, args["dt"], args["T"], args["B"], args["seed"], midpoint_iters=80,
                        midpoint_tol=1e-15)
    errs = []
    for cap in (1, 2, 3, 4, 5):
        _, st = _step_from(model, wl, args["dt"], args["T"], args["B"], args["seed"], midpoint_iters=cap)
        assert st.last_iterations == cap
        errs.append(np.abs(st.spin - ref.spin).max())
    rates = [b / a for a, b in zip(errs, errs[1:])]
    assert all(r < 0.5 for r in rates), errs


def test_anderson_reaches_the_same_fixed_point_in_fewer_iterations(model):
    wl = W.fege_small()
    dt, T, B, seed = 4.0, 0.0, (0.0, 0.0, 0.0), 6
    _, plain = _step_from(model, wl, dt, T, B, seed, midpoint_iters=200, midpoint_tol=1e-12)
    _, acc = _step_from(model, wl, dt, T, B, seed, midpoint_iters=200, midpoint_tol=1e-12, anderson_depth=3,
                        anderson_reg=1e-10)
    assert np.abs(acc.spin - plain.spin).max() < 1e-10
    assert acc.last_iterations < plain.last_iterations, (acc.last_iterations, plain.last_iterations)


def test_cap_zero_is_the_predictor_corrector(model):
    wl = W.fege_small()
    a = O.State(wl.positions, wl.velocities, wl.spins, wl.species, wl.box, wl.periodic)
    b = O.State(wl.positions, wl.velocities, wl.spins, wl.species, wl.box, wl.periodic)
    O.run(model, a, 3, 1.0, 300.0, (0, 0, 0.2))
    O.run(model, b, 3, 1.0, 300.0, (0, 0, 0.2), midpoint_iters=0, midpoint_tol=1e-3, anderson_depth=2)
    assert np.array_equal(a.spin, b.spin) and np.array_equal(a.vel, b.vel) and b.last_iterations == 0


@pytest.mark.slow
def test_midpoint_nve_energy_second_order(model):
    wl = W.fege_cube(3, seed=40, T=100.0)
    drift = []
    for dt in (1.0, 0.5, 0.25):
        st = O.State(wl.positions, wl.velocities, wl.spins, wl.species, wl.box, wl.periodic)
        e0 = O.evaluate(model, st.pos, st.spin, st.species, st.box, st.periodic)["E"] + \
            O.kinetic_energy(st.vel, st.species, model.mass)
        worst = 0.0
        for _ in range(8):
            O.run(model, st, int(round(5.0 / dt)), dt, 0.0, (0, 0, 0), gamma=0.0, lam=0.0, midpoint_iters=40,
                  midpoint_tol=1e-13)
            e = O.evaluate(model, st.pos, st.spin, st.species, st.box, st.periodic)["E"] + \
                O.kinetic_energy(st.vel, st.species, model.mass)
            worst = max(worst, abs(e - e0))
        drift.append(worst / wl.n)
    # time-symmetric second-order step: the error at fixed time falls four-fold per halving
    for a, b in zip(drift, drift[1:]):
        assert 3.6 < a / b < 4.4, drift
