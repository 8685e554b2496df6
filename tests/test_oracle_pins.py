"""Pins of the FP64 CPU oracle against what mathematics and the paper fix.

None of these compare the oracle with itself: each checks a closed form, a library
routine, an invariance, a conservation law or a finite difference, chosen so that
a dropped term, a flipped sign, a wrong index or a transposed operand fails one.
The paper prints no worked example, so there are no printed values to pin to.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb
from scipy import special, stats

from oracle import oracle as O
from paper_2606_14073_gb300 import workloads as W

from conftest import variant

NCH, K = 5, 9
D = 66
iO = NCH + 4 * NCH


def iA(n, l):
    return NCH + n * 4 + (l - 1)


def iX(g, n):  # g: 0 EX, 1 DMI, 2 ANI, 3 SIA
    return iO + 1 + g * NCH + n


def iSA(n, l):
    return iO + 1 + 4 * NCH + n * 4 + (l - 1)


def onehot_params(params):
    """Coefficients c^G_{n k} = delta_{nk} for every group and species pair, so
    g^G_n(r) = f_n(r) and the descriptor reduces to the carrier itself."""
    p = variant(params)
    c = np.zeros_like(p["coeffs"])
    for n in range(NCH):
        c[:, :, :, n, n] = 1.0
    p["coeffs"] = c
    return p


def cheb_closed(x, k):
    return math.cos(k * math.acos(x))


def carrier_closed(r, rc, k):
    if r >= rc:
        return 0.0
    fc = 0.5 * (1.0 + math.cos(math.pi * r / rc))
    x = 2.0 * (r / rc - 1.0) ** 2 - 1.0
    return 0.5 * (cheb_closed(x, k) + 1.0) * fc


# ---------------------------------------------------------------- Philox / noise
def test_philox_matches_numpy_library():
    rng = np.random.default_rng(3)
    for _ in range(20):
        ctr = rng.integers(1, 2 ** 63, size=4, dtype=np.uint64)
        key = rng.integers(0, 2 ** 63, size=2, dtype=np.uint64)
        ours = O.philox4x64_10(ctr, key)
        # numpy advances its 256-bit counter before each block
        c = int(ctr[0]) | (int(ctr[1]) << 64) | (int(ctr[2]) << 128) | (int(ctr[3]) << 192)
        ref = np.random.Philox(counter=c - 1, key=int(key[0]) | (int(key[1]) << 64)).random_raw(4)
        assert np.array_equal(ours, ref)


def test_gaussians_are_standard_normal():
    z = np.array([O.gauss4(s, a, 1, 1234, 0) for s in range(50) for a in range(200)]).ravel()
    assert abs(z.mean()) < 4.0 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 4.0 * math.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # different streams / keys are uncorrelated
    a = np.array([O.gauss4(s, 7, 1, 1234, 0)[0] for s in range(4000)])
    b = np.array([O.gauss4(s, 7, 2, 1234, 0)[0] for s in range(4000)])
    c = np.array([O.gauss4(s, 7, 1, 1234, 1)[0] for s in range(4000)])
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.06 and abs(np.corrcoef(a, c)[0, 1]) < 0.06


# ---------------------------------------------------------------- carrier
def test_chebyshev_closed_form_and_derivative():
    for x in np.linspace(-1.0, 1.0, 41):
        T, dT = O.chebyshev(x, K)
        for k in range(K):
            assert T[k] == pytest.approx(cheb_closed(x, k), abs=1e-13)
            ref = npcheb.chebval(x, npcheb.chebder(np.eye(K)[k]))
            assert dT[k] == pytest.approx(ref, abs=1e-11 * max(1, k * k))


def test_carrier_closed_form_cutoff_and_derivative():
    rc = 6.0
    for r in np.linspace(0.5, 6.5, 61):
        f, df = O.carrier(r, rc, K)
        for k in range(K):
            assert f[k] == pytest.approx(carrier_closed(r, rc, k), abs=1e-14)
        h = 1e-6
        fp, _ = O.carrier(r + h, rc, K)
        fm, _ = O.carrier(r - h, rc, K)
        if abs(r - rc) > 2 * h:
            assert np.allclose(df, (fp - fm) / (2 * h), atol=1e-8)
    # smooth at the cutoff: value and slope vanish
    f, df = O.carrier(rc * (1 - 1e-9), rc, K)
    assert np.abs(f).max() < 1e-15 and np.abs(df).max() < 1e-8
    f, df = O.carrier(rc, rc, K)
    assert not f.any() and not df.any()


# ---------------------------------------------------------------- closed forms
def _isolated(pos, spins, species):
    return (np.asarray(pos, float), np.asarray(spins, float), np.asarray(species, np.int32),
            np.array([60.0, 60.0, 60.0]), np.array([0, 0, 0], np.int32))


def test_dimer_closed_forms(params):
    p = onehot_params(params)
    m = O.Model(p)
    rng = np.random.default_rng(1)
    S1, S2 = W.random_unit_vectors(rng, 2)
    for r in (2.1, 3.3, 3.9, 5.0):
        pos = np.array([[10.0, 10.0, 10.0], [10.0, 10.0, 10.0]])
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        pos[1] += r * d
        q = O.descriptors(m, *_isolated(pos, [S1, S2], [0, 1]))
        u = d
        for n in range(NCH):
            fR, fA = carrier_closed(r, 6.0, n), carrier_closed(r, 4.0, n)
            assert q[0, n] == pytest.approx(fR, abs=1e-13)
            for l in range(1, 5):  # P_l(1) = 1 for the j = k term
                assert q[0, iA(n, l)] == pytest.approx(fA * fA, abs=1e-13)
                assert q[0, iSA(n, l)] == pytest.approx((fA * (S1 @ S2)) ** 2, abs=1e-13)
            assert q[0, iX(0, n)] == pytest.approx(fR * (S1 @ S2), abs=1e-13)
            assert q[0, iX(1, n)] == pytest.approx(fR * (np.cross(S1, S2) @ u), abs=1e-13)
            assert q[0, iX(2, n)] == pytest.approx(fR * (S1 @ u) * (S2 @ u), abs=1e-13)
            assert q[0, iX(3, n)] == pytest.approx(fR * (S1 @ u) ** 2, abs=1e-13)
            # the second atom sees -u
            assert q[1, iX(1, n)] == pytest.approx(fR * (np.cross(S2, S1) @ -u), abs=1e-13)
        assert q[0, iO] == pytest.approx(1.0, abs=1e-15)


def test_trimer_legendre_closed_form(params):
    p = onehot_params(params)
    m = O.Model(p)
    rng = np.random.default_rng(2)
    S = W.random_unit_vectors(rng, 3)
    for theta in (0.3, 1.1, 2.0, 3.0):
        r1, r2 = 2.4, 3.1
        pos = np.array([[10.0, 10.0, 10.0],
                        [10.0 + r1, 10.0, 10.0],
                        [10.0 + r2 * math.cos(theta), 10.0 + r2 * math.sin(theta), 10.0]])
        q = O.descriptors(m, *_isolated(pos, S, [0, 0, 1]))
        s1, s2 = S[0] @ S[1], S[0] @ S[2]
        for n in range(NCH):
            g1, g2 = carrier_closed(r1, 4.0, n), carrier_closed(r2, 4.0, n)
            for l in range(1, 5):
                Pl = special.eval_legendre(l, math.cos(theta))
                assert q[0, iA(n, l)] == pytest.approx(g1 ** 2 + g2 ** 2 + 2 * g1 * g2 * Pl, abs=1e-12)
                w1, w2 = g1 * s1, g2 * s2
                assert q[0, iSA(n, l)] == pytest.approx(w1 ** 2 + w2 ** 2 + 2 * w1 * w2 * Pl, abs=1e-12)


def test_species_pair_indexing(params):
    """Coefficients are indexed [centre species][neighbour species]: a dimer Fe-Ge
    with only the (Fe, Ge) block nonzero gives q^R on the Fe atom only."""
    p = variant(params)
    c = np.zeros_like(p["coeffs"])
    c[0, 1, 0, 2, 4] = 1.0   # centre Fe, neighbour Ge, group R, n = 2, k = 4
    p["coeffs"] = c
    m = O.Model(p)
    pos = np.array([[10.0, 10.0, 10.0], [13.0, 10.0, 10.0]])
    S = np.array([[0, 0, 1.0], [0, 0, 1.0]])
    q = O.descriptors(m, *_isolated(pos, S, [0, 1]))
    assert q[0, 2] == pytest.approx(carrier_closed(3.0, 6.0, 4), abs=1e-14)
    assert q[1, 2] == 0.0 and not np.delete(q[0], [2, iO]).any()


# ---------------------------------------------------------------- derivatives
def _fd_check(m, pos, spins, species, box, per, B, atoms, h=1e-5):
    r = O.evaluate(m, pos, spins, species, box, per, B)
    scale_F = np.abs(r["F"]).max()
    scale_H = np.abs(r["H"]).max()
    for i in atoms:
        for c in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, c] += h
            pm[i, c] -= h
            fd = -(O.evaluate(m, pp, spins, species, box, per, B)["E"]
                   - O.evaluate(m, pm, spins, species, box, per, B)["E"]) / (2 * h)
            assert abs(r["F"][i, c] - fd) <= 1e-7 * scale_F, (i, c, r["F"][i, c], fd)
            sp, sm = spins.copy(), spins.copy()
            sp[i, c] += h
            sm[i, c] -= h
            fd = -(O.evaluate(m, pos, sp, species, box, per, B)["E"]
                   - O.evaluate(m, pos, sm, species, box, per, B)["E"]) / (2 * h)
            assert abs(r["H"][i, c] - fd) <= 1e-7 * scale_H, (i, c, r["H"][i, c], fd)
    return r


def test_forces_fields_finite_difference_periodic(model):
    wl = W.fege_cube(3, seed=11)
    B = np.array([0.7, -0.4, 1.1])
    rng = np.random.default_rng(5)
    _fd_check(model, wl.positions, wl.spins, wl.species, wl.box, wl.periodic, B,
              rng.choice(wl.n, 5, replace=False))


@pytest.mark.parametrize("group", ["R", "A", "EX", "DMI", "ANI", "SIA"])
def test_forces_fields_finite_difference_single_group(params, group):
    """Each group alone, so a term that cancels against another cannot hide."""
    scale = {g: 0.0 for g in ("R", "A", "EX", "DMI", "ANI", "SIA") if g != group}
    m = O.Model(variant(params, **scale))
    pos, spins, species, box, per = W.isolated_cluster(2, seed=3)
    _fd_check(m, pos, spins, species, box, per, np.zeros(3), [0, 5, 11])


def test_virial_matches_strain_derivative(model):
    # periodic: diagonal strain of box and positions
    wl = W.fege_cube(3, seed=12)
    r = O.evaluate(model, wl.positions, wl.spins, wl.species, wl.box, wl.periodic)
    h = 1e-6
    for a in range(3):
        s = np.ones(3)
        s[a] = 1 + h
        Ep = O.evaluate(model, wl.positions * s, wl.spins, wl.species, wl.box * s, wl.periodic)["E"]
        s[a] = 1 - h
        Em = O.evaluate(model, wl.positions * s, wl.spins, wl.species, wl.box * s, wl.periodic)["E"]
        assert r["W"][a, a] == pytest.approx(-(Ep - Em) / (2 * h), rel=1e-6, abs=1e-7)
    # isolated cluster: full 3x3 deformation r -> (I + eps) r
    pos, spins, species, box, per = W.isolated_cluster(2, seed=4)
    r = O.evaluate(model, pos, spins, species, box, per)
    for a in range(3):
        for b in range(3):
            e = np.zeros((3, 3))
            e[a, b] = h
            Ep = O.evaluate(model, pos @ (np.eye(3) + e).T, spins, species, box, per)["E"]
            Em = O.evaluate(model, pos @ (np.eye(3) - e).T, spins, species, box, per)["E"]
            # dE/d eps_ab = sum_pairs D_b... -> W_ba = -dE/deps_ab
            assert r["W"][b, a] == pytest.approx(-(Ep - Em) / (2 * h), rel=1e-6, abs=1e-7)


# ---------------------------------------------------------------- invariances
def random_rotation(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


def test_translation_and_permutation_invariance(model):
    wl = W.fege_cube(3, seed=13)
    r0 = O.evaluate(model, wl.positions, wl.spins, wl.species, wl.box, wl.periodic)
    shifted = W.wrap(wl.positions + np.array([1.3, -2.7, 0.45]), wl.box, wl.periodic)
    r1 = O.evaluate(model, shifted, wl.spins, wl.species, wl.box, wl.periodic)
    assert r1["E"] == pytest.approx(r0["E"], rel=1e-12, abs=1e-12)
    assert np.allclose(r1["F"], r0["F"], atol=1e-11) and np.allclose(r1["H"], r0["H"], atol=1e-11)
    perm = np.random.default_rng(0).permutation(wl.n)
    r2 = O.evaluate(model, wl.positions[perm], wl.spins[perm], wl.species[perm], wl.box, wl.periodic)
    assert r2["E"] == pytest.approx(r0["E"], rel=1e-12, abs=1e-12)
    assert np.allclose(r2["F"], r0["F"][perm], atol=1e-12) and np.allclose(r2["H"], r0["H"][perm], atol=1e-12)


def test_joint_rotation_covariance(model):
    pos, spins, species, box, per = W.isolated_cluster(2, seed=6)
    rng = np.random.default_rng(6)
    Q = random_rotation(rng)
    c = pos.mean(0)
    r0 = O.evaluate(model, pos, spins, species, box, per)
    r1 = O.evaluate(model, (pos - c) @ Q.T + c, spins @ Q.T, species, box, per)
    assert r1["E"] == pytest.approx(r0["E"], rel=1e-11, abs=1e-12)
    assert np.allclose(r1["F"], r0["F"] @ Q.T, atol=1e-11)
    assert np.allclose(r1["H"], r0["H"] @ Q.T, atol=1e-11)


def test_time_reversal(model):
    wl = W.fege_cube(3, seed=14)
    r0 = O.evaluate(model, wl.positions, wl.spins, wl.species, wl.box, wl.periodic)
    r1 = O.evaluate(model, wl.positions, -wl.spins, wl.species, wl.box, wl.periodic)
    assert r1["E"] == pytest.approx(r0["E"], rel=1e-12, abs=1e-12)
    assert np.allclose(r1["F"], r0["F"], atol=1e-12) and np.allclose(r1["H"], -r0["H"], atol=1e-12)


def test_chirality_only_from_dmi(params):
    pos, spins, species, box, per = W.isolated_cluster(2, seed=7)
    c = pos.mean(0)
    inv = 2 * c - pos          # spatial inversion; spins are axial and stay
    full = O.Model(params)
    e0 = O.evaluate(full, pos, spins, species, box, per)["E"]
    e1 = O.evaluate(full, inv, spins, species, box, per)["E"]
    assert abs(e1 - e0) > 1e-6
    nodmi = O.Model(variant(params, DMI=0.0))
    e0 = O.evaluate(nodmi, pos, spins, species, box, per)["E"]
    e1 = O.evaluate(nodmi, inv, spins, species, box, per)["E"]
    assert e1 == pytest.approx(e0, rel=1e-12, abs=1e-13)


def test_spin_only_rotation(params):
    pos, spins, species, box, per = W.isolated_cluster(2, seed=8)
    Q = random_rotation(np.random.default_rng(8))
    iso = O.Model(variant(params, DMI=0.0, ANI=0.0, SIA=0.0))
    assert O.evaluate(iso, pos, spins @ Q.T, species, box, per)["E"] == pytest.approx(
        O.evaluate(iso, pos, spins, species, box, per)["E"], rel=1e-12, abs=1e-13)
    ani = O.Model(variant(params, DMI=0.0, SIA=0.0))
    assert abs(O.evaluate(ani, pos, spins @ Q.T, species, box, per)["E"]
               - O.evaluate(ani, pos, spins, species, box, per)["E"]) > 1e-7


def test_momentum_and_angular_momentum_identities(model):
    wl = W.fege_cube(3, seed=15)
    r = O.evaluate(model, wl.positions, wl.spins, wl.species, wl.box, wl.periodic)
    assert np.abs(r["F"].sum(0)).max() < 1e-11
    pos, spins, species, box, per = W.isolated_cluster(2, seed=9)
    r = O.evaluate(model, pos, spins, species, box, per)
    assert np.abs(r["F"].sum(0)).max() < 1e-12
    torque = np.cross(pos, r["F"]).sum(0) + np.cross(spins, r["H"]).sum(0)
    assert np.abs(torque).max() < 1e-11


def test_zeeman_term(model):
    wl = W.fege_cube(3, seed=16)
    B = np.array([0.2, 0.5, -1.3])
    r0 = O.evaluate(model, wl.positions, wl.spins, wl.species, wl.box, wl.periodic)
    r1 = O.evaluate(model, wl.positions, wl.spins, wl.species, wl.box, wl.periodic, B)
    mu = np.asarray(W.MOMENT_MUB)[wl.species] * 5.7883818060e-5
    assert r1["E"] - r0["E"] == pytest.approx(-(mu * (wl.spins @ B)).sum(), rel=1e-12)
    assert np.allclose(r1["H"] - r0["H"], mu[:, None] * B[None, :], atol=1e-14)


def test_subset_evaluation_matches_full(model):
    wl = W.fege_cube(4, seed=17)
    full = O.evaluate(model, wl.positions, wl.spins, wl.species, wl.box, wl.periodic)
    sample = np.array([0, 17, 255, 300, 511])
    sub = O.evaluate_subset(model, wl.positions, wl.spins, wl.species, wl.box, wl.periodic, sample)
    assert np.allclose(sub["F"], full["F"][sample], atol=1e-13)
    assert np.allclose(sub["H"], full["H"][sample], atol=1e-13)
    assert np.allclose(sub["Ei"], full["Ei"][sample], atol=1e-14)


# ---------------------------------------------------------------- neighbours
@pytest.mark.parametrize("cells,per", [(4, (1, 1, 1)), (3, (1, 1, 1)), (5, (1, 1, 0)), (6, (1, 0, 0))])
def test_cell_list_equals_brute_force(cells, per):
    wl = W.fege_cube(cells, seed=20 + cells)
    per = np.array(per, np.int32)
    pos = wl.positions.copy()
    if not per.all():
        pos[:, ~per.astype(bool)] += np.random.default_rng(0).normal(0, 3.0, size=(wl.n, int((~per.astype(bool)).sum())))
    for cut in (5.0, 7.0):
        a = O.neighbors(pos, wl.box, per, cut, method=0)
        b = O.neighbors(pos, wl.box, per, cut, method=1)
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
        # symmetric relation
        for i in range(0, wl.n, 37):
            for j in a[i]:
                assert i in set(a[j].tolist())


def test_neighbor_count_matches_density():
    wl = W.fege_cube(6, seed=31)
    nb = O.neighbors(wl.positions, wl.box, wl.periodic, 7.0, method=1)
    rho = 8 / 4.70 ** 3
    assert np.mean([len(x) for x in nb]) == pytest.approx(4 / 3 * math.pi * 7.0 ** 3 * rho, rel=0.03)


# ---------------------------------------------------------------- integrator
def _free_spins(params, n=1, spacing=20.0):
    p = variant(params, net=0.0)
    m = O.Model(p)
    pos = np.stack([np.arange(n) * spacing + 5.0, np.full(n, 5.0), np.full(n, 5.0)], 1)
    box = np.array([n * spacing + 10.0, 10.0, 10.0])
    return m, pos, box, np.array([0, 0, 0], np.int32)


def test_larmor_precession_exact(params):
    m, pos, box, per = _free_spins(params)
    S0 = np.array([[0.6, 0.0, 0.8]])
    B = np.array([0.0, 0.0, 50.0])
    st = O.State(pos, np.zeros((1, 3)), S0, np.array([0], np.int32), box, per)
    w = 1.0 * 5.7883818060e-5 * 50.0 / 0.6582119569   # rad/fs
    t = 0
    for _ in range(5):
        O.run(m, st, 40, 0.5, 0.0, B, gamma=0.0, lam=0.0)
        t += 20.0
        ref = np.array([0.6 * math.cos(w * t), 0.6 * math.sin(w * t), 0.8])  # dS/dt = (muB B/hbar) x S
        assert np.allclose(st.spin[0], ref, atol=1e-12)


def test_damped_precession_second_order(params):
    m, pos, box, per = _free_spins(params)
    B = np.array([0.0, 0.0, 400.0])
    lam = 0.2
    th0 = 2.5
    w = 5.7883818060e-5 * 400.0 / 0.6582119569
    T_end = 200.0
    errs = []
    for dt in (1.0, 0.5, 0.25):
        st = O.State(pos, np.zeros((1, 3)), [[math.sin(th0), 0, math.cos(th0)]], np.array([0], np.int32), box, per)
        O.run(m, st, int(round(T_end / dt)), dt, 0.0, B, gamma=0.0, lam=lam)
        th = 2 * math.atan(math.tan(th0 / 2) * math.exp(-lam * w * T_end / (1 + lam * lam)))
        errs.append(abs(math.acos(st.spin[0, 2]) - th))
        assert abs(np.linalg.norm(st.spin[0]) - 1) < 1e-14
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.2) and errs[1] / errs[2] == pytest.approx(4.0, rel=0.2)


def test_unit_spin_norm_every_step(model):
    wl = W.fege_small()
    st = O.State(wl.positions, wl.velocities, wl.spins, wl.species, wl.box, wl.periodic)
    for _ in range(5):
        O.run(model, st, 2, 1.0, 300.0, (0, 0, 1.0))
        assert np.abs(np.linalg.norm(st.spin, axis=1) - 1).max() < 1e-14


@pytest.mark.slow
def test_thermal_spin_langevin_function(params):
    n = 600
    m, pos, box, per = _free_spins(params, n=n)
    T, Bz, lam = 100.0, 100.0, 1.0
    x = 5.7883818060e-5 * Bz / (8.617333262e-5 * T)
    st = O.State(pos, np.zeros((n, 3)), W.random_unit_vectors(np.random.default_rng(1), n),
                 np.zeros(n, np.int32), box, per)
    O.run(m, st, 1500, 1.0, T, (0, 0, Bz), gamma=0.0, lam=lam, seed=77)
    samples = []
    for _ in range(60):
        O.run(m, st, 50, 1.0, T, (0, 0, Bz), gamma=0.0, lam=lam, seed=77)
        samples.append(st.spin[:, 2].mean())
    ref = 1.0 / math.tanh(x) - 1.0 / x
    sem = np.std(samples) / math.sqrt(len(samples)) * 3 + 0.2 / math.sqrt(n * 10)
    assert abs(np.mean(samples) - ref) < max(3 * sem, 0.02), (np.mean(samples), ref)


@pytest.mark.slow
def test_thermal_lattice_equipartition(params):
    n = 800
    m, pos, box, per = _free_spins(params, n=n)
    T = 300.0
    species = (np.arange(n) % 2).astype(np.int32)
    st = O.State(pos, np.zeros((n, 3)), np.tile([0, 0, 1.0], (n, 1)), species, box, per)
    st.periodic = np.array([1, 1, 1], np.int32)
    O.run(m, st, 500, 1.0, T, (0, 0, 0), gamma=0.05, lam=0.0, seed=78)
    vals = []
    for _ in range(40):
        O.run(m, st, 25, 1.0, T, (0, 0, 0), gamma=0.05, lam=0.0, seed=78)
        mass = np.asarray(W.MASS_AMU)[species]
        vals.append((mass[:, None] * st.vel ** 2).sum(1).mean() / 9.6485332e-3)
    ref = 3 * 8.617333262e-5 * T
    assert np.mean(vals) == pytest.approx(ref, rel=0.03)


@pytest.mark.slow
def test_nve_energy_drift_second_order(model):
    wl = W.fege_cube(3, seed=40, T=100.0)
    drift = []
    for dt in (1.0, 0.5, 0.25):
        st = O.State(wl.positions, wl.velocities, wl.spins, wl.species, wl.box, wl.periodic)
        r = O.evaluate(model, st.pos, st.spin, st.species, st.box, st.periodic)
        e0 = r["E"] + O.kinetic_energy(st.vel, st.species, model.mass)
        worst = 0.0
        for _ in range(8):
            O.run(model, st, int(round(5.0 / dt)), dt, 0.0, (0, 0, 0), gamma=0.0, lam=0.0)
            e = O.evaluate(model, st.pos, st.spin, st.species, st.box, st.periodic)["E"] + \
                O.kinetic_energy(st.vel, st.species, model.mass)
            worst = max(worst, abs(e - e0))
        drift.append(worst / wl.n)
    # second-order integrator: the energy error at fixed time shrinks at least as
    # dt^2 (ratio >= 4 per halving; this scheme shows ~8); a first-order slip gives ~2
    for a, b in zip(drift, drift[1:]):
        assert 3.4 < a / b < 10.5, drift


def test_run_is_deterministic_and_resumable(model):
    wl = W.fege_cube(3, seed=41)
    a = O.State(wl.positions, wl.velocities, wl.spins, wl.species, wl.box, wl.periodic)
    O.run(model, a, 6, 1.0, 300.0, (0, 0, 0.5))
    b = O.State(wl.positions, wl.velocities, wl.spins, wl.species, wl.box, wl.periodic)
    O.run(model, b, 2, 1.0, 300.0, (0, 0, 0.5))
    O.run(model, b, 4, 1.0, 300.0, (0, 0, 0.5))
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.spin, b.spin) and np.array_equal(a.vel, b.vel)


def test_network_special_cases(params):
    """E_i = sum_h w1_h tanh(sum_v W0_hv s_v q_v - b0_h) - b1, pinned by cases whose
    value is fixed without the network: W0 = 0 makes E_i a constant; a single
    W0 entry (h, v) selects exactly one scaled descriptor entry."""
    wl = W.fege_cube(3, seed=50)
    p = variant(params)
    p["w0"] = np.zeros_like(p["w0"])
    p["b1"] = 0.37
    r = O.evaluate(O.Model(p), wl.positions, wl.spins, wl.species, wl.box, wl.periodic)
    const = float(np.sum(p["w1"] * np.tanh(-p["b0"]))) - 0.37
    assert np.allclose(r["Ei"], const, atol=1e-14)
    assert np.abs(r["F"]).max() == 0.0
    h, v = 3, 7
    p["w0"][h, v] = 1.0
    p["b0"] = np.zeros_like(p["b0"])
    p["w1"] = np.zeros_like(p["w1"])
    p["w1"][h] = 1.0
    p["b1"] = 0.0
    m = O.Model(p)
    q = O.descriptors(m, wl.positions, wl.spins, wl.species, wl.box, wl.periodic)
    r = O.evaluate(m, wl.positions, wl.spins, wl.species, wl.box, wl.periodic)
    assert np.allclose(r["Ei"], np.tanh(p["q_scaler"][v] * q[:, v]), atol=1e-14)
