"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances:
  FP64 mode   |gpu - oracle| <= 1e-10 * max|oracle| per output array (E, F, H, W, q);
              trajectories: 1e-9 after 100 steps (chaotic growth of the 1e-16
              rounding differences over 100 fs stays far below that).
  mixed mode  RMSE(F) <= 1e-3 eV/A and RMSE(H) <= 1e-3 eV against the oracle, every atom's
              |dF_i| <= 2e-3 eV/A and |dH_i| <= 2e-3 eV, virial within 1e-4 of max |W|.
  neighbours  bit-exact sets.
Sizes span several thread blocks and end in ragged tails (512, 1728, 1725, slab).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_14073_gb300 import nep_params, spinlat as S, workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
# mixed precision (FP32 descriptors and backward, FP16 hi/lo network): besides the RMSE bars,
# every atom's force and field error vector is bounded (eV/A and eV), and the virial relative
# to its largest entry
MIXED_ATOM_TOL = 2e-3
MIXED_VIRIAL_TOL = 1e-4


@pytest.fixture(scope="module")
def params():
    return nep_params.load()


@pytest.fixture(scope="module")
def model(params):
    return O.Model(params)


def ragged_cube(cells=6, drop=3, seed=71):
    wl = W.fege_cube(cells, seed=seed)
    keep = np.ones(wl.n, bool)
    keep[np.random.default_rng(seed).choice(wl.n, drop, replace=False)] = False
    wl.positions, wl.spins, wl.species, wl.velocities = (wl.positions[keep], wl.spins[keep], wl.species[keep],
                                                         wl.velocities[keep])
    return wl


def small_slab():
    return W.fege_slab_helix(8, 8, 3, vacuum=6.0, period_target=37.6, B_z=0.2, seed=72)


WORKLOADS = {
    "b20_512": lambda: W.fege_small(),
    "b20_1728": lambda: W.fege_cube(6, seed=70),
    "b20_1725_ragged": lambda: ragged_cube(),
    "slab_1536_free_z": small_slab,
}


def gpu_state(sys_):
    st = sys_.get_state()
    return st["positions"], st["spins"]


def maxrel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_neighbor_lists_bit_exact(params, name):
    wl = WORKLOADS[name]()
    s = S.system_from_workload(wl, params)
    pos, _ = gpu_state(s)
    rad, ang = s.get_neighbors()
    ref_r = O.neighbors(pos, wl.box, wl.periodic, 7.0, method=0 if wl.n <= 2000 else 1)
    ref_a = O.neighbors(pos, wl.box, wl.periodic, 5.0, method=0 if wl.n <= 2000 else 1)
    assert all(np.array_equal(a, b) for a, b in zip(rad, ref_r))
    assert all(np.array_equal(a, b) for a, b in zip(ang, ref_a))
    s.destroy()


def test_neighbor_lists_bit_exact_with_atoms_far_outside_a_free_axis(params):
    """The highest and the lowest atom of the slab, each with the atoms within 4 A of it,
    moved 25 A further out along the free axis: they sit more than a cell width beyond the edge
    cells that hold them, so every pair of theirs is decided by the exact FP64 test (their FP32
    cell-relative positions are not kept); the pairs inside each group keep their distances."""
    wl = small_slab()

    def group(k):
        d = wl.positions - wl.positions[k]
        d -= wl.box * wl.periodic * np.rint(d / wl.box)
        return np.flatnonzero(np.linalg.norm(d, axis=1) < 4.0)

    up, down = group(int(np.argmax(wl.positions[:, 2]))), group(int(np.argmin(wl.positions[:, 2])))
    assert len(up) > 1 and len(down) > 1 and not set(up) & set(down)
    wl.positions[up, 2] += 25.0
    wl.positions[down, 2] -= 25.0
    s = S.system_from_workload(wl, params)
    pos, _ = gpu_state(s)
    assert pos[:, 2].max() > wl.box[2] + 15.0 and pos[:, 2].min() < -15.0
    rad, ang = s.get_neighbors()
    ref_r = O.neighbors(pos, wl.box, wl.periodic, 7.0, method=0)
    ref_a = O.neighbors(pos, wl.box, wl.periodic, 5.0, method=0)
    assert all(np.array_equal(a, b) for a, b in zip(rad, ref_r))
    assert all(np.array_equal(a, b) for a, b in zip(ang, ref_a))
    assert all(len(rad[i]) > 0 for i in np.concatenate([up, down]))
    s.destroy()


def mixed_cells_box(seed=73):
    """3 x 6 x 6 B20 cells, periodic: 14.1 A along x holds 2 binning cells (the list build's
    whole-axis walk with the minimum image), 28.2 A along y and z hold 4 (placed images)."""
    pos, species, box = W.b20_lattice(3, 6, 6)
    rng = np.random.default_rng(seed)
    pos = W.wrap(pos + rng.normal(0.0, 0.05, pos.shape), box, np.ones(3, np.int32))
    return pos, W.random_unit_vectors(rng, len(pos)), species, box, np.ones(3, np.int32)


def free_cluster():
    """A 3 x 3 x 3-cell B20 fragment with free boundaries in a 100 A binning box."""
    return W.isolated_cluster(3, seed=74)


@pytest.mark.parametrize("make", [mixed_cells_box, free_cluster], ids=["mixed_cells_3x6x6", "free_cluster_3"])
def test_lists_and_fp64_forces_on_odd_grids(params, model, make):
    pos, spin, species, box, per = make()
    s = S.System(pos, spin, box, per, species, params)
    st = s.get_state()
    rad, ang = s.get_neighbors()
    ref_r = O.neighbors(st["positions"], box, per, 7.0, method=0)
    ref_a = O.neighbors(st["positions"], box, per, 5.0, method=0)
    assert all(np.array_equal(a, b) for a, b in zip(rad, ref_r))
    assert all(np.array_equal(a, b) for a, b in zip(ang, ref_a))
    r = s.energy_forces_fields()
    ref = O.evaluate(model, st["positions"], st["spins"], species, box, per)
    assert maxrel(r["F"], ref["F"]) <= FP64_TOL and maxrel(r["H"], ref["H"]) <= FP64_TOL
    assert maxrel(r["W"], ref["W"]) <= FP64_TOL
    s.destroy()


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_descriptors_fp64(params, model, name):
    wl = WORKLOADS[name]()
    s = S.system_from_workload(wl, params)
    pos, spin = gpu_state(s)
    q, e = s.get_descriptors()
    qr = O.descriptors(model, pos, spin, wl.species, wl.box, wl.periodic)
    scale = np.maximum(np.abs(qr).max(0), 1e-12)
    assert (np.abs(q - qr) / scale).max() <= FP64_TOL
    ref = O.evaluate(model, pos, spin, wl.species, wl.box, wl.periodic)
    assert maxrel(e, ref["Ei"]) <= FP64_TOL
    s.destroy()


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_energy_forces_fields_virial_fp64(params, model, name):
    wl = WORKLOADS[name]()
    B = (0.3, -0.7, 1.1)
    s = S.system_from_workload(wl, params)
    s.step(0, 1.0, 0.0, B)   # sets the field used by the evaluation
    pos, spin = gpu_state(s)
    r = s.energy_forces_fields()
    ref = O.evaluate(model, pos, spin, wl.species, wl.box, wl.periodic, B)
    assert abs(r["E"] - ref["E"]) <= FP64_TOL * max(abs(ref["E"]), np.abs(ref["Ei"]).sum())
    assert maxrel(r["F"], ref["F"]) <= FP64_TOL
    assert maxrel(r["H"], ref["H"]) <= FP64_TOL
    assert maxrel(r["W"], ref["W"]) <= FP64_TOL
    s.destroy()


def test_fp64_trajectory_100_steps(params, model):
    """512-atom FeGe, 100 Langevin steps of 1 fs at 300 K: GPU vs oracle integrator."""
    wl = W.fege_small()
    B = (0.0, 0.0, 0.0)
    s = S.system_from_workload(wl, params, steps_per_graph=10)
    st = s.get_state()
    o = O.State(st["positions"], st["velocities"], st["spins"], wl.species, wl.box, wl.periodic)
    o.F, o.H, o.have_fh = st["forces"].copy(), st["fields"].copy(), True
    assert maxrel(st["forces"], O.evaluate(model, o.pos, o.spin, wl.species, wl.box, wl.periodic)["F"]) <= FP64_TOL
    for chunk in (1, 9, 40, 50):
        s.step(chunk, wl.dt, wl.T, B)
        O.run(model, o, chunk, wl.dt, wl.T, B, gamma=0.01, lam=0.1, seed=wl.seed, replica=0)
        g = s.get_state()
        d = g["positions"] - o.pos
        d -= wl.box * np.rint(d / wl.box)
        assert np.abs(d).max() < 1e-9, (chunk, np.abs(d).max())
        assert np.abs(g["spins"] - o.spin).max() < 1e-9
        assert maxrel(g["velocities"], o.vel) < 1e-9
        assert np.abs(np.linalg.norm(g["spins"], axis=1) - 1).max() < 1e-14
    assert g["step"] == 100
    s.destroy()


@pytest.mark.parametrize("name", ["b20_512", "b20_1728", "slab_1536_free_z"])
def test_mixed_precision_force_field_error(params, model, name):
    wl = WORKLOADS[name]()
    B = (0.0, 0.0, 0.5)
    s = S.system_from_workload(wl, params, precision=S.SL_PREC_MIXED)
    s.step(0, 1.0, 0.0, B)
    pos, spin = gpu_state(s)
    r = s.energy_forces_fields()
    ref = O.evaluate(model, pos, spin, wl.species, wl.box, wl.periodic, B)
    rmse_f = np.sqrt(((r["F"] - ref["F"]) ** 2).mean())
    rmse_h = np.sqrt(((r["H"] - ref["H"]) ** 2).mean())
    assert rmse_f <= 1e-3 and rmse_h <= 1e-3, (rmse_f, rmse_h)
    # no single atom far off: per-atom error vectors within MIXED_ATOM_TOL
    err_f = np.linalg.norm(r["F"] - ref["F"], axis=1).max()
    err_h = np.linalg.norm(r["H"] - ref["H"], axis=1).max()
    assert err_f <= MIXED_ATOM_TOL and err_h <= MIXED_ATOM_TOL, (err_f, err_h)
    assert abs(r["E"] - ref["E"]) / wl.n <= 1e-4
    # virial (eV) within MIXED_VIRIAL_TOL of the largest oracle entry
    assert np.abs(r["W"] - ref["W"]).max() <= MIXED_VIRIAL_TOL * np.abs(ref["W"]).max(), (r["W"], ref["W"])
    s.destroy()


def test_mixed_trajectory_stays_close(params, model):
    wl = W.fege_small()
    s = S.system_from_workload(wl, params, precision=S.SL_PREC_MIXED)
    st = s.get_state()
    o = O.State(st["positions"], st["velocities"], st["spins"], wl.species, wl.box, wl.periodic)
    o.F, o.H, o.have_fh = st["forces"].copy(), st["fields"].copy(), True
    s.step(20, 1.0, 300.0, (0, 0, 0))
    O.run(model, o, 20, 1.0, 300.0, (0, 0, 0), seed=wl.seed)
    g = s.get_state()
    d = g["positions"] - o.pos
    d -= wl.box * np.rint(d / wl.box)
    assert np.abs(d).max() < 1e-3
    assert np.abs(g["spins"] - o.spin).max() < 1e-3
    assert np.abs(np.linalg.norm(g["spins"], axis=1) - 1).max() < 1e-14


@pytest.mark.parametrize("prec", [S.SL_PREC_FP64, S.SL_PREC_MIXED])
def test_determinism_and_bit_identical_resume(params, prec):
    wl = W.fege_small()
    a = S.system_from_workload(wl, params, precision=prec)
    a.step(30, 1.0, 300.0, (0, 0, 0.2))
    ga = a.get_state()
    b = S.system_from_workload(wl, params, precision=prec)
    b.step(12, 1.0, 300.0, (0, 0, 0.2))
    ck = b.get_state()
    # resume in a fresh system created from the checkpoint positions (its internal
    # atom order differs) with the checkpoint's carried forces, fields and list reference
    c = S.System(ck["positions"], ck["spins"], wl.box, wl.periodic, wl.species, params, ck["velocities"],
                 precision=prec, seed=wl.seed)
    c.set_state(ck["positions"], ck["velocities"], ck["spins"], ck["forces"], ck["fields"], ck["step"],
                ref_positions=ck["ref_positions"])
    c.step(18, 1.0, 300.0, (0, 0, 0.2))
    gc = c.get_state()
    b.step(18, 1.0, 300.0, (0, 0, 0.2))
    gb = b.get_state()
    for k in ("positions", "velocities", "spins", "forces", "fields"):
        assert np.array_equal(ga[k], gb[k]), k
        assert np.array_equal(ga[k], gc[k]), k
    # without the list reference positions the resumed run is the same trajectory up to
    # summation order (neighbour segments differ), i.e. equal to rounding
    d = S.system_from_workload(wl, params, precision=prec)
    d.set_state(ck["positions"], ck["velocities"], ck["spins"], ck["forces"], ck["fields"], ck["step"])
    d.step(18, 1.0, 300.0, (0, 0, 0.2))
    gd = d.get_state()
    dd = gd["positions"] - ga["positions"]
    dd -= wl.box * np.rint(dd / wl.box)
    assert np.abs(dd).max() < (1e-9 if prec == S.SL_PREC_FP64 else 1e-3)
    for x in (a, b, c, d):
        x.destroy()


def test_graphs_match_direct_launches(params):
    wl = W.fege_small()
    a = S.system_from_workload(wl, params, steps_per_graph=0)
    b = S.system_from_workload(wl, params, steps_per_graph=7)
    a.step(23, 1.0, 300.0, (0, 0, 0))
    b.step(23, 1.0, 300.0, (0, 0, 0))
    ga, gb = a.get_state(), b.get_state()
    for k in ("positions", "velocities", "spins"):
        assert np.array_equal(ga[k], gb[k])


def test_batch_equals_alone(params):
    """Uneven replicas in one batch (fused launches over every replica, each replica taking
    part until its own steps are done) match each replica run alone."""
    wls = [W.fege_cube(c, seed=80 + i, replica=i) for i, c in enumerate((4, 5, 4))]
    calls = [([15, 15, 15], (200.0, 250.0, 300.0)), ([25, 12, 31], (100.0, 50.0, 0.0))]
    alone = []
    for k, w in enumerate(wls):
        s = S.system_from_workload(w, params, replica=w.seed - W.LANGEVIN_SEED0)
        for n_steps, Ts in calls:
            s.step(n_steps[k], 1.0, Ts[k], (0, 0, 0.3))
        alone.append(s.get_state())
        s.destroy()
    syss = [S.system_from_workload(w, params, replica=w.seed - W.LANGEVIN_SEED0) for w in wls]
    b = S.Batch(syss)
    for n_steps, Ts in calls:
        b.step(n_steps, 1.0, list(Ts), (0, 0, 0.3))
    st = b.stats()
    # fused: 15 steps = one 10-step graph + 5 one-step graphs; 31 steps = 3 + 1
    assert st["fused_calls"] == 2 and st["replica_calls"] == 0 and st["fused_captures"] == 1
    assert st["fused_steps"] == 15 + 31 and b.graph_launches() == 6 + 4
    for s, ref in zip(syss, alone):
        g = s.get_state()
        assert g["step"] == ref["step"]
        for key in ("positions", "velocities", "spins", "forces", "fields"):
            assert np.array_equal(g[key], ref[key]), key
    b.destroy()
    for s in syss:
        s.destroy()


def test_empty_and_tiny_systems(params, model):
    box = np.array([30.0, 30.0, 30.0])
    s = S.System(np.zeros((0, 3)), np.zeros((0, 3)), box, [0, 0, 0], np.zeros(0, np.int32), params)
    s.step(3, 1.0, 300.0, (0, 0, 1.0))
    r = s.energy_forces_fields()
    assert r["E"] == 0.0 and r["F"].shape == (0, 3)
    s.destroy()
    pos = np.array([[10.0, 10.0, 10.0], [12.5, 10.3, 9.6]])
    spin = np.array([[0, 0, 1.0], [0.6, 0.0, 0.8]])
    s = S.System(pos, spin, box, [0, 0, 0], np.array([0, 1], np.int32), params)
    r = s.energy_forces_fields()
    ref = O.evaluate(model, pos, spin, np.array([0, 1], np.int32), box, np.array([0, 0, 0], np.int32))
    assert maxrel(r["F"], ref["F"]) <= FP64_TOL and maxrel(r["H"], ref["H"]) <= FP64_TOL
    s.destroy()


def test_neighbor_overflow_is_reported_and_state_restored(params):
    wl = W.fege_small()
    c = wl.box / 2
    d = wl.positions - c
    vel = -0.02 * d                     # inward flow: the centre densifies within a few dozen fs
    s = S.System(wl.positions, wl.spins, wl.box, wl.periodic, wl.species, params, vel, cap_rad=128, cap_ang=48,
                 gamma=0.0, steps_per_graph=0)
    before = None
    with pytest.raises(S.SpinlatError) as e:
        for _ in range(60):
            before = s.get_state()
            s.step(5, 1.0, 0.0, (0, 0, 0))
    assert e.value.code == S.SL_ENBR_OVERFLOW
    after = s.get_state()
    for k in ("positions", "velocities", "spins", "forces", "fields"):
        assert np.array_equal(after[k], before[k]), k
    assert after["step"] == before["step"]


def test_batch_overflow_restores_only_the_failing_replica(params):
    """In one batched call, a replica that overflows its lists goes back to its state at
    the start of the call; the other replica's steps are kept."""
    wl = W.fege_small()
    c = wl.box / 2
    vel = -0.02 * (wl.positions - c)
    bad = S.System(wl.positions, wl.spins, wl.box, wl.periodic, wl.species, params, vel, cap_rad=128, cap_ang=48,
                   gamma=0.0, steps_per_graph=0, replica=1)
    good = S.System(wl.positions, wl.spins, wl.box, wl.periodic, wl.species, params, wl.velocities, replica=2,
                    steps_per_graph=0)
    b = S.Batch([good, bad])
    code = None
    for _ in range(60):
        g0, b0 = good.get_state(), bad.get_state()
        try:
            b.step(5, 1.0, [0.0, 0.0], [(0, 0, 0), (0, 0, 0)])
        except S.SpinlatError as e:
            code = e.code
            break
    assert code == S.SL_ENBR_OVERFLOW
    b1, g1 = bad.get_state(), good.get_state()
    for k in ("positions", "velocities", "spins", "forces", "fields"):
        assert np.array_equal(b1[k], b0[k]), k
    assert b1["step"] == b0["step"]
    assert g1["step"] == g0["step"] + 5
    assert not np.array_equal(g1["positions"], g0["positions"])
    b.destroy()
    good.destroy()
    bad.destroy()


@pytest.mark.parametrize("prec", [S.SL_PREC_FP64, S.SL_PREC_MIXED])
def test_autotune_leaves_state_and_results_unchanged(params, prec):
    wl = W.fege_cube(5, seed=90)
    a = S.system_from_workload(wl, params, precision=prec)
    b = S.system_from_workload(wl, params, precision=prec)
    st0 = a.get_state()
    info = a.autotune(repeats=3)
    q = 64 if prec == S.SL_PREC_FP64 else 128
    assert info["crad_block"] in (64, 128) and info["ang_block"] in (q // 2, q) and info["bwd_block"] in (q // 2, q)
    assert info["mlp_ctas_per_sm"] in (1, 2) and info["eval_ms_after"] <= info["eval_ms_before"] * 1.5
    # the search covered block sizes and (mixed precision) register budgets; the library
    # checked that every candidate left forces and fields unchanged bit for bit
    cfg = a.launch_config()
    assert len(cfg["landscape_ms"]) == (2 if prec == S.SL_PREC_FP64 else 4)
    assert cfg["crad_minb"] in (0, 3) and cfg["ang_minb"] in (0, 1) and cfg["bwd_minb"] in (0, 3)
    if prec == S.SL_PREC_FP64:
        assert cfg["crad_minb"] == cfg["ang_minb"] == cfg["bwd_minb"] == 0
    st1 = a.get_state()
    for k in ("positions", "velocities", "spins", "forces", "fields"):
        assert np.array_equal(st0[k], st1[k]), k
    a.step(25, 1.0, 300.0, (0, 0, 0.1))
    b.step(25, 1.0, 300.0, (0, 0, 0.1))
    ga, gb = a.get_state(), b.get_state()
    for k in ("positions", "velocities", "spins", "forces", "fields"):
        assert np.array_equal(ga[k], gb[k]), k
    a.destroy()
    b.destroy()


@pytest.mark.parametrize("only", [0, 1])
def test_single_species_systems_match_oracle(params, model, only):
    """All-Fe and all-Ge systems (one species block, empty second block) in both precisions."""
    wl = W.fege_cube(4, seed=95)
    species = np.full(wl.n, only, np.int32)
    B = (0.0, 0.1, 0.2)
    for prec in (S.SL_PREC_FP64, S.SL_PREC_MIXED):
        s = S.System(wl.positions, wl.spins, wl.box, wl.periodic, species, params, wl.velocities, precision=prec)
        s.step(0, 1.0, 0.0, B)
        r = s.energy_forces_fields()
        pos, spin = gpu_state(s)
        ref = O.evaluate(model, pos, spin, species, wl.box, wl.periodic, B)
        if prec == S.SL_PREC_FP64:
            assert maxrel(r["F"], ref["F"]) <= FP64_TOL and maxrel(r["H"], ref["H"]) <= FP64_TOL
            assert abs(r["E"] - ref["E"]) <= FP64_TOL * abs(ref["E"])
        else:
            assert np.sqrt(((r["F"] - ref["F"]) ** 2).mean()) <= 1e-3
            assert np.sqrt(((r["H"] - ref["H"]) ** 2).mean()) <= 1e-3
        s.step(12, 1.0, 300.0, B)
        assert np.isfinite(s.get_state()["positions"]).all()
        s.destroy()


def test_fp32_carrier_matches_fp64_carrier():
    """The FP32 carrier's cutoff factor comes from Taylor polynomials of sin and cos (truncation
    below 6e-8 on its range); against the FP64 carrier (library sincospi) the basis and its
    slope stay at the FP32 rounding level of the Chebyshev recurrence (about 4e-6 of the largest
    value, the same with library cosines), at both cutoffs and in the tails near rc."""
    for rc in (6.0, 4.0):
        ef, edf = S.sl_selftest_carrier(200000, rc)
        assert ef < 1e-5 and edf < 1e-5, (rc, ef, edf)


def test_bounded_wait_gives_up_and_the_context_stays_usable(params, model):
    """A device wait on a barrier nothing arrives at stops after its poll limit and reports
    SL_ETIMEOUT through the status word; evaluations on the same context are unaffected."""
    assert S.lib().sl_selftest_bounded_wait(1000) == S.SL_ETIMEOUT
    wl = W.fege_small()
    s = S.system_from_workload(wl, params, precision=S.SL_PREC_MIXED)   # the tensor-core network path
    st = s.get_state()
    r = s.energy_forces_fields(want_virial=False)
    ref = O.evaluate(model, st["positions"], st["spins"], wl.species, wl.box, wl.periodic)
    assert np.sqrt(((r["F"] - ref["F"]) ** 2).mean()) <= 1e-3
    s.destroy()
