"""The no-allocation entry point against the regular one.

sl_descriptors_energies_noalloc serves callers that may not allocate device
memory (code inside a host framework's CUDA-graph capture, plugins whose engine
owns every device byte, real-time loops).  Its scratch is one fixed array in the
library shared by all calls.  This test calls it twice in a row -- the second
call on a smaller system, so the array still holds the first call's contents --
and checks both results against sl_get_descriptors of a regular system at the
FP64 tolerance of the other parity tests (1e-10 of the largest value).  This file
is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2606_14073_gb300 import nep_params, spinlat as S, workloads as W

pytestmark = pytest.mark.gpu


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


def test_noalloc_matches_regular_entry_point_on_two_calls():
    torch = pytest.importorskip("torch")
    params = nep_params.load()
    cases = [_ragged(6, 5, 91), _ragged(4, 3, 92)]   # 1723 atoms, then 509 atoms
    for pos, spins, species, box, per in cases:
        reg = S.System(pos, spins, box, per, species, params)
        st = reg.get_state()
        q_ref, e_ref = reg.get_descriptors()
        reg.destroy()
        n = pos.shape[0]
        p4, s4, sp = _device_inputs(torch, st["positions"], st["spins"], species)
        q = torch.empty((n, 66), dtype=torch.float64, device="cuda")
        e = torch.empty((n,), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream()
        S.sl_descriptors_energies_noalloc(p4.data_ptr(), s4.data_ptr(), sp.data_ptr(), n, box, per, params,
                                          q.data_ptr(), e.data_ptr(), stream.cuda_stream)
        qg, eg = q.cpu().numpy(), e.cpu().numpy()
        assert np.abs(qg - q_ref).max() <= 1e-10 * np.abs(q_ref).max()
        assert np.abs(eg - e_ref).max() <= 1e-10 * np.abs(e_ref).max()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    params = nep_params.load()
    with pytest.raises(S.SpinlatError) as ex:
        S.sl_descriptors_energies_noalloc(0, 0, 0, 4096, [30.0, 30.0, 30.0], [1, 1, 1], params, None, 0, None)
    assert ex.value.code == S.SL_EINVAL
