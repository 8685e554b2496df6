"""Pins of the oracle's longitudinal mode (variable moment lengths, paper Section 3).

The spin equation is the Langevin form with longitudinal fluctuations (Ma and Dudarev,
Phys. Rev. B 86, 054416, 2012): dS/dt = (H/hbar) x S + (alpha/hbar) H + xi with a Landau
onsite energy a|S|^2 + b|S|^4.  Each test checks the oracle against mathematics fixed
independently of it: a finite difference of the energy, the closed-form logistic relaxation
of |S|^2, exact Larmor precession, the Boltzmann density over R^3 by quadrature, the sign of
the dissipation, second-order convergence in dt, and the reduction to the unit-length mode
at alpha = 0."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_2606_14073_gb300 import workloads as W

from conftest import variant

MUB, HBAR, KB = 5.7883818060e-5, 0.6582119569, 8.617333262e-5


def _free_spins(params, n=1, spacing=20.0, landau=None):
    m = O.Model(variant(params, net=0.0), landau=landau)
    pos = np.stack([np.arange(n) * spacing + 5.0, np.full(n, 5.0), np.full(n, 5.0)], 1)
    box = np.array([n * spacing + 10.0, 10.0, 10.0])
    return m, pos, box, np.array([0, 0, 0], np.int32)


def _scaled_spins(wl, seed=3):
    rng = np.random.default_rng(seed)
    return wl.spins * rng.uniform(0.6, 1.5, size=(wl.n, 1))


def test_landau_energy_closed_form_on_free_spins(params):
    lan = [[-0.3, 0.1], [-0.2, 0.05]]
    m, pos, box, per = _free_spins(params, n=2, landau=lan)
    S = np.array([[0.3, -1.1, 0.4], [0.0, 0.7, -0.2]])
    sp = np.array([0, 1], np.int32)
    B = np.array([0.0, 0.5, 2.0])
    r = O.evaluate(m, pos, S, sp, box, per, B)
    m0 = O.evaluate(O.Model(variant(params, net=0.0)), pos, S, sp, box, per, B)
    e = 0.0
    for i, t in enumerate(sp):
        a, b = lan[t]
        q = S[i] @ S[i]
        e += a * q + b * q * q
        assert np.allclose(r["H"][i] - m0["H"][i], -(2 * a + 4 * b * q) * S[i], atol=1e-15)
    assert r["E"] - m0["E"] == pytest.approx(e, abs=1e-14)


def test_landau_fields_finite_difference_at_unequal_lengths(params):
    wl = W.fege_small()
    m = O.Model(params, landau=[[-0.25, 0.1], [-0.1, 0.04]])
    S = _scaled_spins(wl)
    B = (0.1, -0.2, 0.7)
    r = O.evaluate(m, wl.positions, S, wl.species, wl.box, wl.periodic, B)
    h = 1e-5
    for i in (0, 7, 100, 301):
        for c in range(3):
            Sp, Sm = S.copy(), S.copy()
            Sp[i, c] += h
            Sm[i, c] -= h
            ep = O.evaluate(m, wl.positions, Sp, wl.species, wl.box, wl.periodic, B)["E"]
            em = O.evaluate(m, wl.positions, Sm, wl.species, wl.box, wl.periodic, B)["E"]
            fd = -(ep - em) / (2 * h)
            assert r["H"][i, c] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_logistic_relaxation_second_order(params):
    """T = 0, no field, no network: d|S|^2/dt = (4 alpha/hbar)(|a| - 2b|S|^2)|S|^2, a logistic
    curve u(t) = K / (1 + (K/u0 - 1) exp(-r t)), r = 4 alpha |a|/hbar, K = |a|/(2b); the
    direction of S does not change."""
    a, b, alpha = -0.1, 0.05, 0.2
    m, pos, box, per = _free_spins(params, landau=[[a, b], [a, b]])
    d0 = np.array([0.48, -0.6, 0.64])
    T_end = 20.0
    r, K, u0 = 4 * alpha * abs(a) / HBAR, abs(a) / (2 * b), 0.25
    ref = K / (1 + (K / u0 - 1) * math.exp(-r * T_end))
    errs = []
    for dt in (1.0, 0.5, 0.25):
        st = O.State(pos, np.zeros((1, 3)), [0.5 * d0], np.array([0], np.int32), box, per)
        O.run(m, st, int(round(T_end / dt)), dt, 0.0, (0, 0, 0), gamma=0.0, longitudinal=True, alpha_long=alpha)
        u = float(st.spin[0] @ st.spin[0])
        errs.append(abs(u - ref))
        assert np.allclose(st.spin[0] / math.sqrt(u), d0, atol=1e-14)
    assert errs[2] < 1e-4 * ref
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.25) and errs[1] / errs[2] == pytest.approx(4.0, rel=0.25)


def test_larmor_precession_keeps_length(params):
    m, pos, box, per = _free_spins(params)
    S0 = 1.7 * np.array([0.6, 0.0, 0.8])
    B = np.array([0.0, 0.0, 50.0])
    st = O.State(pos, np.zeros((1, 3)), [S0], np.array([0], np.int32), box, per)
    w = MUB * 50.0 / HBAR
    t = 0.0
    for _ in range(5):
        O.run(m, st, 40, 0.5, 0.0, B, gamma=0.0, longitudinal=True, alpha_long=0.0)
        t += 20.0
        ref = 1.7 * np.array([0.6 * math.cos(w * t), 0.6 * math.sin(w * t), 0.8])
        assert np.allclose(st.spin[0], ref, atol=1e-12)
    # with a Landau term and no damping the length is still kept exactly (rotations only)
    m2, _, _, _ = _free_spins(params, landau=[[-0.2, 0.05], [-0.2, 0.05]])
    st = O.State(pos, np.zeros((1, 3)), [S0], np.array([0], np.int32), box, per)
    O.run(m2, st, 100, 0.5, 0.0, B, gamma=0.0, longitudinal=True, alpha_long=0.0)
    assert abs(np.linalg.norm(st.spin[0]) - 1.7) < 1e-13


def _boltzmann_moments(a, b, h, kT):
    """<|S|^2> and <S.B^> under exp(-(a m^2 + b m^4 - h m cos th)/kT) d^3S, the angle done
    in closed form: int e^{x c} dc = 2 sinh(x)/x, int c e^{x c} dc = 2 (cosh x / x - sinh x / x^2)."""
    def w(mm):
        return math.exp(-(a * mm * mm + b * mm ** 4) / kT) * mm * mm

    def ang0(x):
        return 2.0 if x < 1e-8 else 2 * math.sinh(x) / x

    def ang1(x):
        return 2 * x / 3 if x < 1e-4 else 2 * (math.cosh(x) / x - math.sinh(x) / (x * x))

    top = 6.0
    Z = integrate.quad(lambda mm: w(mm) * ang0(h * mm / kT), 0, top, epsabs=0, epsrel=1e-12)[0]
    M2 = integrate.quad(lambda mm: w(mm) * mm * mm * ang0(h * mm / kT), 0, top, epsabs=0, epsrel=1e-12)[0]
    Mz = integrate.quad(lambda mm: w(mm) * mm * ang1(h * mm / kT), 0, top, epsabs=0, epsrel=1e-12)[0]
    return M2 / Z, Mz / Z


@pytest.mark.slow
def test_thermal_lengths_and_magnetisation_follow_boltzmann(params):
    n = 800
    a, b = -0.02, 0.01
    T, Bz, alpha = 100.0, 100.0, 0.5
    m, pos, box, per = _free_spins(params, n=n, landau=[[a, b], [a, b]])
    st = O.State(pos, np.zeros((n, 3)), W.random_unit_vectors(np.random.default_rng(5), n),
                 np.zeros(n, np.int32), box, per)
    kw = dict(gamma=0.0, longitudinal=True, alpha_long=alpha, seed=91)
    O.run(m, st, 1500, 1.0, T, (0, 0, Bz), **kw)
    m2s, mzs = [], []
    for _ in range(60):
        O.run(m, st, 50, 1.0, T, (0, 0, Bz), **kw)
        m2s.append((st.spin ** 2).sum(1).mean())
        mzs.append(st.spin[:, 2].mean())
    ref2, refz = _boltzmann_moments(a, b, MUB * Bz, KB * T)
    for vals, ref in ((m2s, ref2), (mzs, refz)):
        sem = np.std(vals) / math.sqrt(len(vals))
        assert abs(np.mean(vals) - ref) < max(4 * sem, 0.01 * abs(ref)), (np.mean(vals), ref)


def _total_energy(m, st, B):
    r = O.evaluate(m, st.pos, st.spin, st.species, st.box, st.periodic, B)
    return r["E"] + O.kinetic_energy(st.vel, st.species, m.mass)


def test_damping_dissipates_energy(params):
    """T = 0, no lattice friction: the longitudinal-mode damping term can only lower the
    total energy (dE/dt = -(alpha/hbar)|H|^2 for the spin part); moments grow toward the
    Landau minimum |S|^2 = -a/(2b) = 1.44."""
    wl = W.fege_small()
    m = O.Model(params, landau=[[-0.144, 0.05], [-0.144, 0.05]])
    st = O.State(wl.positions, wl.velocities * 0.1, wl.spins, wl.species, wl.box, wl.periodic)
    B = (0.0, 0.0, 0.5)
    e = [_total_energy(m, st, B)]
    for _ in range(10):
        O.run(m, st, 4, 0.25, 0.0, B, gamma=0.0, longitudinal=True, alpha_long=0.1)
        e.append(_total_energy(m, st, B))
    d = np.diff(e)
    assert (d < 0).all(), d
    lengths = np.linalg.norm(st.spin, axis=1)
    assert lengths.mean() > 1.02


def test_alpha_zero_reduces_to_unit_length_mode(model):
    """At alpha = 0 the longitudinal step is the predictor-corrector rotation of the unit
    mode at lambda = 0 without the renormalisation (rotations keep |S| = 1 to roundoff)."""
    wl = W.fege_cube(3, seed=44)
    a = O.State(wl.positions, wl.velocities, wl.spins, wl.species, wl.box, wl.periodic)
    b = O.State(wl.positions, wl.velocities, wl.spins, wl.species, wl.box, wl.periodic)
    O.run(model, a, 20, 1.0, 300.0, (0, 0, 0.4), lam=0.0, longitudinal=True, alpha_long=0.0)
    O.run(model, b, 20, 1.0, 300.0, (0, 0, 0.4), lam=0.0)
    assert np.abs(a.spin - b.spin).max() < 1e-12
    assert np.abs(a.pos - b.pos).max() < 1e-12
    assert np.abs(np.linalg.norm(a.spin, axis=1) - 1).max() < 1e-13


def test_second_order_convergence_with_network(params):
    """T = 0, network on, Landau term, damping: the state at a fixed time converges as dt^2."""
    wl = W.fege_cube(2, seed=45, T=50.0)
    m = O.Model(params, landau=[[-0.2, 0.08], [-0.2, 0.08]])
    S0 = _scaled_spins(wl, seed=9)
    T_end = 4.0

    def run(dt):
        st = O.State(wl.positions, wl.velocities, S0, wl.species, wl.box, wl.periodic)
        O.run(m, st, int(round(T_end / dt)), dt, 0.0, (0, 0, 0.3), gamma=0.0, longitudinal=True, alpha_long=0.3)
        return st.spin.copy()

    ref = run(0.0625)
    errs = [np.abs(run(dt) - ref).max() for dt in (0.5, 0.25, 0.125)]
    assert errs[0] / errs[1] > 3.2 and errs[1] / errs[2] > 3.2, errs


def test_longitudinal_options_are_checked(model):
    wl = W.fege_cube(2, seed=46)
    st = O.State(wl.positions, wl.velocities, wl.spins, wl.species, wl.box, wl.periodic)
    with pytest.raises(RuntimeError):
        O.run(model, st, 1, 1.0, 0.0, longitudinal=True, alpha_long=-1.0)
    with pytest.raises(RuntimeError):
        O.run(model, st, 1, 1.0, 0.0, longitudinal=True, alpha_long=0.1, midpoint_iters=3)
