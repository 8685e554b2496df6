"""The fused batch step: one launch of each kernel of the step covers every replica of a batch
(include/spinlat.h, batches).  A replica's trajectory is bit-identical alone and in a batch, in
both precision modes, with replicas of uneven size and uneven step counts, while replicas are
admitted into and retired from slots between calls without a new graph capture; batches that
cannot be fused (different models) run the replicas on their own streams."""
import numpy as np
import pytest

from paper_2606_14073_gb300 import nep_params
from paper_2606_14073_gb300 import spinlat as S
from paper_2606_14073_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("positions", "velocities", "spins", "forces", "fields")


@pytest.fixture(scope="module")
def params():
    return nep_params.load()


def _system(params, w, prec, **kw):
    return S.system_from_workload(w, params, precision=prec, replica=w.seed - W.LANGEVIN_SEED0, **kw)


def _alone(params, w, prec, calls, **kw):
    """State of w after stepping alone through calls [(n_steps, T, Bz)]."""
    s = _system(params, w, prec, **kw)
    for n, T, bz in calls:
        if n:
            s.step(n, 1.0, T, (0, 0, bz))
    st = s.get_state()
    s.destroy()
    return st


def _same(a, b):
    assert a["step"] == b["step"]
    for k in KEYS:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("prec", [S.SL_PREC_FP64, S.SL_PREC_MIXED])
def test_fused_batch_equals_alone(params, prec):
    wls = [W.fege_cube(c, seed=300 + i, replica=i) for i, c in enumerate((4, 6, 5, 4))]
    calls = [([13, 13, 3, 0], [150.0, 200.0, 250.0, 300.0], 0.2), ([7, 22, 11, 10], [50.0, 0.0, 100.0, 300.0], 0.0)]
    alone = [_alone(params, w, prec, [(c[0][k], c[1][k], c[2]) for c in calls]) for k, w in enumerate(wls)]
    syss = [_system(params, w, prec) for w in wls]
    b = S.Batch(syss)
    for n, Ts, bz in calls:
        b.step(n, 1.0, Ts, (0, 0, bz))
    st = b.stats()
    assert st["fused_calls"] == 2 and st["replica_calls"] == 0 and st["fused_captures"] == 1
    assert st["fused_steps"] == 13 + 22
    for s, ref in zip(syss, alone):
        _same(s.get_state(), ref)
    b.destroy()
    for s in syss:
        s.destroy()


def test_slots_admit_and_retire_without_new_capture(params):
    """Replicas join and leave the batch's slots between calls; the fused graphs are captured
    once, and every replica matches its run alone."""
    prec = S.SL_PREC_MIXED
    wls = [W.fege_cube(c, seed=320 + i, replica=20 + i) for i, c in enumerate((4, 5, 4, 6))]
    a, b_, c, d = (_system(params, w, prec) for w in wls)
    batch = S.Batch([a, None, b_, None])
    batch.step([12, 0, 9, 0], 1.0, [100.0, 0.0, 200.0, 0.0], (0, 0, 0.1))
    batch.set(1, c)                     # admit c
    batch.step([5, 14, 5, 0], 1.0, [100.0, 300.0, 200.0, 0.0], (0, 0, 0.1))
    ref_a = _alone(params, wls[0], prec, [(12, 100.0, 0.1), (5, 100.0, 0.1)])
    _same(a.get_state(), ref_a)
    batch.set(0, None)                  # retire a
    a.destroy()
    batch.set(3, d)                     # admit d into another slot
    batch.set(0, None)
    batch.step([0, 3, 10, 21], 1.0, [0.0, 300.0, 200.0, 250.0], (0, 0, 0.1))
    st = batch.stats()
    assert st["fused_captures"] == 1 and st["fused_calls"] == 3 and st["replica_calls"] == 0
    _same(b_.get_state(), _alone(params, wls[1], prec, [(9, 200.0, 0.1), (5, 200.0, 0.1), (10, 200.0, 0.1)]))
    _same(c.get_state(), _alone(params, wls[2], prec, [(14, 300.0, 0.1), (3, 300.0, 0.1)]))
    _same(d.get_state(), _alone(params, wls[3], prec, [(21, 250.0, 0.1)]))
    batch.destroy()
    for s in (b_, c, d):
        s.destroy()


@pytest.mark.parametrize("prec", [S.SL_PREC_FP64, S.SL_PREC_MIXED])
def test_launch_grids_follow_the_occupied_slots(params, prec):
    """The one-item-per-block kernels launch only the occupied slots' blocks: in a batch
    reserved for far more atoms than it holds, whose slots fill and empty between calls (the
    captured graphs' grids grow and shrink without a new capture), every replica follows its
    trajectory alone."""
    wls = [W.fege_cube(c, seed=380 + i, replica=50 + i) for i, c in enumerate((4, 8, 5))]
    a, b_, c = (_system(params, w, prec) for w in wls)
    batch = S.Batch([a, None, None])
    batch.reserve(1 << 20)
    batch.step([6, 0, 0], 1.0, [200.0, 0.0, 0.0], (0, 0, 0.1))
    batch.set(1, b_)                    # eight times a's atoms: the grids grow
    batch.step([5, 7, 0], 1.0, [200.0, 250.0, 0.0], (0, 0, 0.1))
    batch.set(0, None)                  # a leaves, c joins: they shrink
    batch.set(2, c)
    batch.step([0, 4, 9], 1.0, [0.0, 250.0, 150.0], (0, 0, 0.1))
    st = batch.stats()
    assert st["fused_captures"] == 1 and st["fused_calls"] == 3 and st["atom_capacity"] == 1 << 20
    _same(a.get_state(), _alone(params, wls[0], prec, [(6, 200.0, 0.1), (5, 200.0, 0.1)]))
    _same(b_.get_state(), _alone(params, wls[1], prec, [(7, 250.0, 0.1), (4, 250.0, 0.1)]))
    _same(c.get_state(), _alone(params, wls[2], prec, [(9, 150.0, 0.1)]))
    batch.destroy()
    for s in (a, b_, c):
        s.destroy()


def test_slot_reused_by_a_system_created_after_a_destroy(params):
    """A replica retired and destroyed, then a new one admitted into the same slot: the new
    system (which may sit at the destroyed one's address) gets its own table entries."""
    prec = S.SL_PREC_MIXED
    batch = S.Batch([None, None])
    for k in range(3):
        w = W.fege_cube(4 + k % 2, seed=360 + k, replica=40 + k)
        s = _system(params, w, prec)
        batch.set(0, s)
        batch.step([9 + k, 0], 1.0, [150.0 + 50 * k, 0.0], (0, 0, 0.1))
        _same(s.get_state(), _alone(params, w, prec, [(9 + k, 150.0 + 50 * k, 0.1)]))
        batch.set(0, None)
        s.destroy()
    assert batch.stats()["fused_captures"] == 1
    batch.destroy()


def test_batch_of_different_models_runs_replicas_alone(params):
    """Replicas with different model parameters cannot share fused launches: they run on their
    own streams, with the same results as alone."""
    p2 = {k: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v) for k, v in params.items()}
    p2["w1"] = p2["w1"] * 1.01
    wls = [W.fege_cube(4, seed=340, replica=30), W.fege_cube(4, seed=341, replica=31)]
    syss = [_system(params, wls[0], S.SL_PREC_FP64), _system(p2, wls[1], S.SL_PREC_FP64)]
    b = S.Batch(syss)
    b.step([6, 6], 1.0, [200.0, 200.0], (0, 0, 0))
    st = b.stats()
    assert st["fused_calls"] == 0 and st["replica_calls"] == 1
    _same(syss[0].get_state(), _alone(params, wls[0], S.SL_PREC_FP64, [(6, 200.0, 0.0)]))
    s2 = S.system_from_workload(wls[1], p2, precision=S.SL_PREC_FP64, replica=31)
    s2.step(6, 1.0, 200.0, (0, 0, 0))
    _same(syss[1].get_state(), s2.get_state())
    s2.destroy()
    b.destroy()
    for s in syss:
        s.destroy()


def test_slot_errors(params):
    wl = W.fege_cube(4, seed=350)
    m = _system(params, wl, S.SL_PREC_MIXED)
    f = _system(params, wl, S.SL_PREC_FP64)
    b = S.Batch([m, None])
    for slot, sys in ((2, f), (-1, m), (1, f), (1, m)):   # outside, outside, other precision, second slot
        with pytest.raises(S.SpinlatError) as e:
            b.set(slot, sys)
        assert e.value.code == S.SL_EINVAL
    ns = np.array([1, 1], np.int64)        # steps for the empty slot
    d, t, bb = np.ones(2), np.zeros(2), np.zeros((2, 3))
    rc = S.lib().sl_batch_step(b.handle, S._ptr(ns), S._ptr(d), S._ptr(t), S._ptr(bb))
    assert rc == S.SL_EINVAL
    b.destroy()
    m.destroy()
    f.destroy()


def test_submit_and_wait(params):
    """A submitted call runs while the host fills an empty slot; the slots taking part are locked
    until the wait, and a second submit before it is refused; results match the runs alone."""
    prec = S.SL_PREC_MIXED
    wa, wb = W.fege_cube(5, seed=370, replica=50), W.fege_cube(4, seed=371, replica=51)
    a = _system(params, wa, prec)
    batch = S.Batch([a, None])
    batch.submit([11, 0], 1.0, [200.0, 0.0], (0, 0, 0.2))
    b = _system(params, wb, prec)          # created while the call runs
    batch.set(1, b)                        # an empty slot may be filled
    with pytest.raises(S.SpinlatError) as e:
        batch.set(0, None)                 # a slot taking part may not
    assert e.value.code == S.SL_EINVAL
    with pytest.raises(S.SpinlatError) as e:
        batch.submit([1, 1], 1.0, [200.0, 200.0], (0, 0, 0.2))
    assert e.value.code == S.SL_EINVAL
    batch.wait()
    batch.wait()                           # nothing in flight
    batch.step([4, 9], 1.0, [200.0, 100.0], (0, 0, 0.2))
    _same(a.get_state(), _alone(params, wa, prec, [(11, 200.0, 0.2), (4, 200.0, 0.2)]))
    _same(b.get_state(), _alone(params, wb, prec, [(9, 100.0, 0.2)]))
    batch.destroy()
    a.destroy()
    b.destroy()
