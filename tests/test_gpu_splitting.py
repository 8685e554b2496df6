"""Coloured Suzuki-Trotter spin sweep on the GPU against the FP64 oracle: the colouring
(integer work, bit-exact) and the trajectory (1e-9 in FP64)."""
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


def test_fp64_sweep_matches_oracle_and_colouring_is_exact(params, model):
    wl = W.fege_small()
    B = (0.0, 0.0, 0.5)
    s = S.system_from_workload(wl, params, precision=S.SL_PREC_FP64)
    s.set_spin_sweep(True)
    st = s.get_state()
    o = O.State(st["positions"], st["velocities"], st["spins"], wl.species, wl.box, wl.periodic)
    o.F, o.H, o.have_fh = st["forces"].copy(), st["fields"].copy(), True
    expected_evals = 0
    for chunk in (1, 1):
        s.step(chunk, 1.0, 300.0, B)
        O.run(model, o, chunk, 1.0, 300.0, B, seed=wl.seed, st_sweep=True)
        g = s.get_state()
        d = g["positions"] - o.pos
        d -= wl.box * np.rint(d / wl.box)
        assert np.abs(d).max() < 1e-9
        assert np.abs(g["spins"] - o.spin).max() < 1e-9
        assert np.abs(g["velocities"] - o.vel).max() < 1e-9
        col, nc, ev = s.sweep_colours()
        ref, nref = O.colour(g["positions"], wl.box, wl.periodic, params["rc_rad"])
        assert nc == nref and np.array_equal(col, ref)
        expected_evals += 2 * nc + 1
        assert ev == expected_evals
    assert np.abs(np.linalg.norm(s.get_state()["spins"], axis=1) - 1).max() < 1e-14
    s.destroy()


def test_mixed_sweep_close_to_fp64(params):
    wl = W.fege_small()
    m = S.system_from_workload(wl, params, precision=S.SL_PREC_MIXED)
    d = S.system_from_workload(wl, params, precision=S.SL_PREC_FP64)
    for x in (m, d):
        x.set_spin_sweep(True)
        x.step(2, 1.0, 300.0, (0, 0, 0.2))
    assert np.abs(m.get_state()["spins"] - d.get_state()["spins"]).max() < 1e-3
    m.destroy()
    d.destroy()


def test_sweep_is_refused_where_it_does_not_apply_and_can_be_left(params):
    wl = W.fege_small()
    s = S.system_from_workload(wl, params, midpoint_iters=2)
    with pytest.raises(S.SpinlatError):
        s.set_spin_sweep(True)
    s.destroy()
    a = S.system_from_workload(wl, params)
    a.set_spin_sweep(True)
    with pytest.raises(S.SpinlatError):
        a.set_longitudinal(True, 0.1)
    with pytest.raises(S.SpinlatError):
        a.step_profiled(1, 1.0, 300.0, (0, 0, 0))
    b = S.Batch([a])
    with pytest.raises(S.SpinlatError):
        b.step(1, 1.0, 300.0, (0, 0, 0))
    b.destroy()
    # back to the predictor-corrector: identical to a system that never used the sweep
    a.set_spin_sweep(False)
    ref = S.system_from_workload(wl, params)
    a.step(10, 1.0, 300.0, (0, 0, 0.3))
    ref.step(10, 1.0, 300.0, (0, 0, 0.3))
    ga, gr = a.get_state(), ref.get_state()
    for k in ("positions", "velocities", "spins"):
        assert np.array_equal(ga[k], gr[k]), k
    a.destroy()
    ref.destroy()
