"""The no-allocation entry point against the FP64 oracle and the regular entry point.

sl_descriptors_energies_noalloc serves callers that cannot allocate device memory:
plugins of simulation engines that give every device byte to their own pool, and
real-time loops that cannot take the synchronisation cudaMalloc/cudaFree may imply.
Its scratch is one fixed array in the library, shared by every call.  The first test
calls it twice in a row -- the second call on a smaller system, so the array still
holds the first call's contents -- and checks both results against the oracle's
descriptors and energies and against sl_get_descriptors of a regular system, at the
FP64 tolerance of the other parity tests (1e-10 of the largest value).  The others
check that a species value outside [0, 2) and a neighbourhood beyond the scratch's
160 slots are reported, not computed.  This file is named so that pytest collects
it last.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_14073_gb300 import nep_params, spinlat as S, workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _device_inputs(torch, pos, spins, species):
    n = pos.shape[0]
    p4 = np.zeros((n, 4))
    p4[:, :3] = pos
    s4 = np.zeros((n, 4))
    s4[:, :3] = spins
    dev = torch.device("cuda")
    return (torch.from_numpy(p4).to(dev), torch.from_numpy(s4).to(dev),
            torch.from_numpy(np.ascontiguousarray(species, dtype=np.int32)).to(dev))


def _ragged(cells, drop, seed):
    wl = W.fege_cube(cells, seed=seed)
    keep = np.ones(wl.n, bool)
    keep[np.random.default_rng(seed).choice(wl.n, drop, replace=False)] = False
    return wl.positions[keep], wl.spins[keep], wl.species[keep], wl.box, wl.periodic


def _call(torch, params, pos, spins, species, box, per):
    n = pos.shape[0]
    p4, s4, sp = _device_inputs(torch, pos, spins, species)
    q = torch.empty((n, 66), dtype=torch.float64, device="cuda")
    e = torch.empty((n,), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    S.sl_descriptors_energies_noalloc(p4.data_ptr(), s4.data_ptr(), sp.data_ptr(), n, box, per, params,
                                      q.data_ptr(), e.data_ptr(), stream.cuda_stream)
    return q.cpu().numpy(), e.cpu().numpy()


def test_noalloc_matches_oracle_and_regular_entry_point_on_two_calls():
    torch = pytest.importorskip("torch")
    params = nep_params.load()
    model = O.Model(params)
    cases = [_ragged(6, 5, 91), _ragged(4, 3, 92)]   # 1723 atoms, then 509 atoms
    for pos, spins, species, box, per in cases:
        # the library wraps positions into the box; both sides use its wrapped copy
        reg = S.System(pos, spins, box, per, species, params)
        st = reg.get_state()
        q_reg, e_reg = reg.get_descriptors()
        reg.destroy()
        qg, eg = _call(torch, params, st["positions"], st["spins"], species, box, per)
        q_or = O.descriptors(model, st["positions"], st["spins"], species, box, per)
        e_or = O.evaluate(model, st["positions"], st["spins"], species, box, per)["Ei"]
        scale = np.maximum(np.abs(q_or).max(0), 1e-12)
        assert (np.abs(qg - q_or) / scale).max() <= TOL
        assert np.abs(eg - e_or).max() <= TOL * np.abs(e_or).max()
        assert np.abs(qg - q_reg).max() <= TOL * np.abs(q_reg).max()
        assert np.abs(eg - e_reg).max() <= TOL * np.abs(e_reg).max()


def test_noalloc_rejects_species_outside_the_model():
    torch = pytest.importorskip("torch")
    params = nep_params.load()
    pos, spins, species, box, per = _ragged(4, 0, 93)
    bad = species.copy()
    bad[17] = 2
    with pytest.raises(S.SpinlatError) as ex:
        _call(torch, params, pos, spins, bad, box, per)
    assert ex.value.code == S.SL_EINVAL
    bad[17] = -1
    with pytest.raises(S.SpinlatError) as ex:
        _call(torch, params, pos, spins, bad, box, per)
    assert ex.value.code == S.SL_EINVAL
    # the next valid call is unaffected by the reported one (the status word is cleared per call)
    q, e = _call(torch, params, pos, spins, species, box, per)
    e_or = O.evaluate(O.Model(params), np.mod(pos, box), spins, species, box, per)["Ei"]
    assert np.abs(e - e_or).max() <= TOL * np.abs(e_or).max()


def test_noalloc_reports_neighbourhoods_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    params = nep_params.load()
    wl = W.fege_small()
    # the crystal compressed to 0.7 of its lattice constant: about 200 atoms inside 6 A
    # of each atom, more than the 160 slots per atom of the scratch (box 13.2 A >= 2 rc_rad)
    box = wl.box * 0.7
    pos = np.mod(wl.positions, wl.box) * 0.7
    with pytest.raises(S.SpinlatError) as ex:
        _call(torch, params, pos, wl.spins, wl.species, box, wl.periodic)
    assert ex.value.code == S.SL_ENBR_OVERFLOW


def test_noalloc_rejects_sizes_beyond_its_scratch():
    params = nep_params.load()
    with pytest.raises(S.SpinlatError) as ex:
        S.sl_descriptors_energies_noalloc(0, 0, 0, 4096, [30.0, 30.0, 30.0], [1, 1, 1], params, None, 0, None)
    assert ex.value.code == S.SL_EINVAL
