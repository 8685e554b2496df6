"""Host-side checks of the CUDA library (no GPU needed): it builds, loads, exports
every symbol the header declares, validates arguments before touching a device,
and its compile-time harmonic table satisfies the addition theorem."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2606_14073_gb300 import nep_params, spinlat as S, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "spinlat.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(sl_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = S.lib()
    decl = declared_functions()
    assert len(decl) >= 15
    for name in decl:
        assert hasattr(L, name), name
    assert set(decl) == set(S.EXPORTS)


def test_harmonic_table_addition_theorem_and_gradients():
    add_err, grad_err = S.sl_selftest_harmonics(5000)
    assert add_err < 1e-13
    assert grad_err < 1e-6


def test_default_options():
    o = S.sl_default_options()
    assert o.precision == S.SL_PREC_FP64 and o.skin == 1.0 and o.nbr_cap_rad == 160 and o.nbr_cap_ang == 64


def _create(**kw):
    p = nep_params.load()
    wl = W.fege_small()
    args = dict(positions=wl.positions, spins=wl.spins, box=wl.box, periodic=wl.periodic, species=wl.species,
                params=p)
    args.update(kw)
    return S.System(args.pop("positions"), args.pop("spins"), args.pop("box"), args.pop("periodic"),
                    args.pop("species"), args.pop("params"), **args)


@pytest.mark.parametrize("bad", [
    dict(box=np.array([10.0, 18.8, 18.8])),                       # periodic length below 2 (rc + skin)
    dict(species=np.full(512, 2, np.int32)),                      # species out of range
    dict(precision=7),
    dict(skin=0.0),
    dict(cap_rad=300),
    dict(cap_ang=200, cap_rad=160),
    dict(midpoint_iters=-1),
    dict(midpoint_iters=65),                                      # above the iteration cap limit
    dict(midpoint_iters=4, anderson_depth=9),
    dict(midpoint_iters=4, midpoint_tol=-1e-3),
    dict(midpoint_iters=4, anderson_reg=float("nan")),
])
def test_invalid_arguments_rejected_before_device_use(bad):
    with pytest.raises(S.SpinlatError) as e:
        _create(**bad)
    assert e.value.code == S.SL_EINVAL


def test_wrong_model_shape_rejected():
    p = dict(nep_params.load())
    p["n_hidden"] = 31
    with pytest.raises(S.SpinlatError) as e:
        _create(params=p)
    assert e.value.code == S.SL_EINVAL


def test_no_device_is_a_loud_error():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(S.SpinlatError) as e:
        _create()
    assert e.value.code == S.SL_ECUDA


def test_texture_grid_validation_needs_no_device():
    # argument checks come before any device work: a bad axis or cell is SL_EINVAL even
    # without a system on a GPU (NULL system first)
    import ctypes as C
    na, nb = C.c_int32(), C.c_int32()
    assert S.lib().sl_texture_map(None, 2, 4.7, C.byref(na), C.byref(nb), None, None) == S.SL_EINVAL
    assert S.lib().sl_set_atom_fields(None, None) == S.SL_EINVAL
    assert S.lib().sl_set_longitudinal(None, 1, 0.1, None) == S.SL_EINVAL


def test_carrier_selftest_argument_checks():
    import ctypes as C
    a, b = C.c_double(), C.c_double()
    assert S.lib().sl_selftest_carrier(0, 6.0, C.byref(a), C.byref(b)) == S.SL_EINVAL
    assert S.lib().sl_selftest_carrier(10, -1.0, C.byref(a), C.byref(b)) == S.SL_EINVAL


def test_bounded_wait_selftest_argument_checks():
    assert S.lib().sl_selftest_bounded_wait(0) == S.SL_EINVAL
    assert S.lib().sl_selftest_bounded_wait(1 << 23) == S.SL_EINVAL


def test_spin_sweep_entry_points_need_a_system():
    assert S.lib().sl_set_spin_sweep(None, 1) == S.SL_EINVAL
    assert S.lib().sl_get_sweep_colours(None, None, None, None) == S.SL_EINVAL
