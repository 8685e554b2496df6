"""Python binding of libspinlat (include/spinlat.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays to
pointers and C status codes to exceptions.  If the library cannot be loaded the
import of `lib()` raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

SL_OK, SL_EINVAL, SL_ENOMEM, SL_ENBR_OVERFLOW, SL_ENONFINITE, SL_ETIMEOUT, SL_ECUDA, SL_EINTERNAL = \
    0, -1, -2, -3, -4, -5, -6, -7
SL_PREC_FP64, SL_PREC_MIXED = 0, 1
_NAMES = {SL_EINVAL: "SL_EINVAL", SL_ENOMEM: "SL_ENOMEM", SL_ENBR_OVERFLOW: "SL_ENBR_OVERFLOW",
          SL_ENONFINITE: "SL_ENONFINITE", SL_ETIMEOUT: "SL_ETIMEOUT", SL_ECUDA: "SL_ECUDA",
          SL_EINTERNAL: "SL_EINTERNAL"}

EXPORTS = ["sl_default_options", "sl_create_system", "sl_step", "sl_energy_forces_fields", "sl_get_descriptors",
           "sl_get_state", "sl_set_state", "sl_get_neighbors", "sl_get_info", "sl_get_stream",
           "sl_destroy_system", "sl_last_error", "sl_batch_create", "sl_batch_step", "sl_batch_destroy",
           "sl_selftest_harmonics", "sl_step_profiled", "sl_measure_fma_peak", "sl_descriptors_energies_noalloc",
           "sl_estimate_device_bytes", "sl_get_midpoint_evaluations", "sl_set_atom_fields", "sl_texture_map",
           "sl_batch_graph_launches", "sl_batch_set", "sl_batch_stats", "sl_batch_reserve", "sl_batch_submit",
           "sl_batch_wait", "sl_autotune", "sl_set_longitudinal", "sl_selftest_carrier",
           "sl_selftest_bounded_wait", "sl_set_spin_sweep", "sl_get_sweep_colours", "sl_get_launch_config"]
KERNEL_GROUPS = ["first_half", "rebuild", "compact", "rad_fwd", "ang_fwd", "network", "backward", "second_half"]


class SpinlatError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class sl_nep_params(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("n_ch", C.c_int32), ("l_max", C.c_int32), ("basis_k", C.c_int32),
                ("rc_rad", C.c_double), ("rc_ang", C.c_double), ("n_hidden", C.c_int32),
                ("coeffs", C.c_void_p), ("q_scaler", C.c_void_p), ("w0", C.c_void_p), ("b0", C.c_void_p),
                ("w1", C.c_void_p), ("b1", C.c_double), ("mass_amu", C.c_void_p), ("moment_muB", C.c_void_p)]


class sl_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("seed", C.c_uint64), ("replica", C.c_uint64), ("skin", C.c_double),
                ("gamma_lattice_per_fs", C.c_double), ("lambda_spin", C.c_double), ("midpoint_iters", C.c_int32),
                ("nbr_cap_rad", C.c_int32), ("nbr_cap_ang", C.c_int32), ("steps_per_graph", C.c_int32),
                ("cuda_stream", C.c_void_p), ("device", C.c_int32), ("midpoint_tol", C.c_double),
                ("anderson_depth", C.c_int32), ("anderson_reg", C.c_double)]


_lib = None
_lock = threading.Lock()


def lib(path: str | None = None):
    """Load libspinlat.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or os.environ.get("SPINLAT_LIB") or _build.build()
            L = C.CDLL(p)
            P, I64, D, I32 = C.c_void_p, C.c_int64, C.c_double, C.c_int32
            L.sl_default_options.argtypes = [P]
            L.sl_default_options.restype = None
            L.sl_create_system.argtypes = [P, P, P, P, P, I64, P, P, P, P]
            L.sl_step.argtypes = [P, I64, D, D, P]
            L.sl_energy_forces_fields.argtypes = [P, P, P, P, P]
            L.sl_get_descriptors.argtypes = [P, P, P]
            L.sl_get_state.argtypes = [P, P, P, P, P, P, P, P]
            L.sl_set_state.argtypes = [P, P, P, P, P, P, P, C.c_uint64]
            L.sl_get_neighbors.argtypes = [P, I32, P, P, P, P]
            L.sl_get_info.argtypes = [P, P, P, P, P]
            L.sl_get_midpoint_evaluations.argtypes = [P, P]
            L.sl_set_atom_fields.argtypes = [P, P]
            L.sl_set_longitudinal.argtypes = [P, I32, D, P]
            L.sl_selftest_carrier.argtypes = [I32, D, P, P]
            L.sl_selftest_bounded_wait.argtypes = [I32]
            L.sl_set_spin_sweep.argtypes = [P, I32]
            L.sl_get_sweep_colours.argtypes = [P, P, P, P]
            L.sl_batch_graph_launches.argtypes = [P, P]
            L.sl_batch_set.argtypes = [P, I32, P]
            L.sl_batch_stats.argtypes = [P, P]
            L.sl_batch_reserve.argtypes = [P, I64]
            L.sl_batch_submit.argtypes = [P, P, P, P, P]
            L.sl_batch_wait.argtypes = [P]
            L.sl_autotune.argtypes = [P, I32, P, P, P]
            L.sl_get_launch_config.argtypes = [P, P, P]
            L.sl_texture_map.argtypes = [P, I32, D, P, P, P, P]
            L.sl_step_profiled.argtypes = [P, I64, D, D, P, P]
            L.sl_measure_fma_peak.argtypes = [I32, P, P]
            L.sl_descriptors_energies_noalloc.argtypes = [P, P, P, I64, P, P, P, P, P, P]
            L.sl_estimate_device_bytes.argtypes = [I64, P]
            L.sl_estimate_device_bytes.restype = C.c_int64
            L.sl_get_stream.argtypes = [P]
            L.sl_get_stream.restype = P
            L.sl_destroy_system.argtypes = [P]
            L.sl_destroy_system.restype = None
            L.sl_last_error.restype = C.c_char_p
            L.sl_batch_create.argtypes = [P, I32, P]
            L.sl_batch_step.argtypes = [P, P, P, P, P]
            L.sl_batch_destroy.argtypes = [P]
            L.sl_batch_destroy.restype = None
            L.sl_selftest_harmonics.argtypes = [I32, P, P]
            for f in ("sl_create_system", "sl_step", "sl_energy_forces_fields", "sl_get_descriptors",
                      "sl_get_state", "sl_set_state", "sl_get_neighbors", "sl_get_info", "sl_batch_create",
                      "sl_batch_step", "sl_selftest_harmonics", "sl_step_profiled", "sl_measure_fma_peak",
                      "sl_descriptors_energies_noalloc", "sl_get_midpoint_evaluations", "sl_set_atom_fields",
                      "sl_texture_map", "sl_batch_graph_launches", "sl_batch_set", "sl_batch_stats", "sl_batch_reserve",
                      "sl_batch_submit", "sl_batch_wait", "sl_autotune", "sl_set_longitudinal",
                      "sl_selftest_carrier", "sl_selftest_bounded_wait", "sl_set_spin_sweep",
                      "sl_get_sweep_colours", "sl_get_launch_config"):
                getattr(L, f).restype = C.c_int
            _lib = L
        return _lib


def _check(rc):
    if rc != SL_OK:
        raise SpinlatError(rc, lib().sl_last_error().decode())


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        a = a.reshape(shape)
    return a


class NepParams:
    """sl_nep_params built from a parameter dict (see nep_params.load); keeps arrays alive."""

    def __init__(self, p: dict):
        self._arrs = {k: _f64(p[k]).ravel() for k in ("coeffs", "q_scaler", "w0", "b0", "w1", "mass_amu",
                                                      "moment_muB")}
        s = sl_nep_params()
        s.n_species, s.n_ch, s.l_max, s.basis_k = int(p["n_species"]), int(p["n_ch"]), 4, int(p["basis_k"])
        s.rc_rad, s.rc_ang, s.n_hidden = float(p["rc_rad"]), float(p["rc_ang"]), int(p["n_hidden"])
        for k, a in self._arrs.items():
            setattr(s, k, a.ctypes.data)
        s.b1 = float(p["b1"])
        self.struct = s


def sl_default_options() -> sl_options:
    o = sl_options()
    lib().sl_default_options(C.byref(o))
    return o


class System:
    """One replica on the GPU.  Methods mirror the C entry points."""

    def __init__(self, positions, spins, box, periodic, species, params: dict, velocities=None, *,
                 precision=SL_PREC_FP64, seed=1234, replica=0, skin=1.0, gamma=0.01, lam=0.1,
                 cap_rad=160, cap_ang=64, steps_per_graph=10, stream=None, device=-1, midpoint_iters=0,
                 midpoint_tol=0.0, anderson_depth=0, anderson_reg=1e-10):
        pos = _f64(positions)
        n = pos.shape[0]
        sp = _f64(spins)
        spec = np.ascontiguousarray(species, dtype=np.int32)
        box_ = _f64(box)
        per = np.ascontiguousarray(periodic, dtype=np.int32)
        vel = None if velocities is None else _f64(velocities)
        self.params = NepParams(params)
        o = sl_default_options()
        o.precision, o.seed, o.replica, o.skin = int(precision), int(seed), int(replica), float(skin)
        o.gamma_lattice_per_fs, o.lambda_spin = float(gamma), float(lam)
        o.nbr_cap_rad, o.nbr_cap_ang, o.steps_per_graph = int(cap_rad), int(cap_ang), int(steps_per_graph)
        o.cuda_stream = stream
        o.device = int(device)
        o.midpoint_iters, o.midpoint_tol = int(midpoint_iters), float(midpoint_tol)
        o.anderson_depth, o.anderson_reg = int(anderson_depth), float(anderson_reg)
        self.options = o
        h = C.c_void_p()
        _check(lib().sl_create_system(_ptr(pos), _ptr(sp), _ptr(box_), _ptr(per), _ptr(spec), n, _ptr(vel),
                                      C.byref(self.params.struct), C.byref(o), C.byref(h)))
        self.handle = h
        self.n = n
        self.precision = int(precision)

    # -- C entry points
    def set_atom_fields(self, B_atoms=None):
        """Per-atom part of the external field ([n][3] tesla, caller order); None removes it."""
        b = None if B_atoms is None else _f64(B_atoms)
        if b is not None and b.shape != (self.n, 3):
            raise ValueError("B_atoms must have shape (n, 3)")
        _check(lib().sl_set_atom_fields(self.handle, _ptr(b)))

    def set_longitudinal(self, enable: bool = True, alpha: float = 0.1, landau=None):
        """Longitudinal moment mode: spin lengths become dynamical with damping alpha and the
        optional Landau onsite energy landau [n_species][2] = (a, b), eV; enable=False returns
        to unit spins."""
        lan = None if landau is None else _f64(landau).reshape(-1)
        if lan is not None and lan.shape != (4,):
            raise ValueError("landau must have shape (2, 2)")
        _check(lib().sl_set_longitudinal(self.handle, int(bool(enable)), float(alpha), _ptr(lan)))

    def set_spin_sweep(self, enable: bool = True):
        """Coloured Suzuki-Trotter spin sweep instead of the predictor-corrector spin update."""
        _check(lib().sl_set_spin_sweep(self.handle, int(bool(enable))))

    def sweep_colours(self, with_colours: bool = True):
        """(colours [n] caller order or None, number of colours, evaluations so far) of the
        last coloured step."""
        nc, ev = C.c_int32(), C.c_int64()
        col = np.zeros(self.n, np.int32) if with_colours else None
        _check(lib().sl_get_sweep_colours(self.handle, _ptr(col), C.byref(nc), C.byref(ev)))
        return col, nc.value, ev.value

    def texture(self, normal: int = 2, cell: float = 4.7):
        """(m [n_b][n_a][3], Q): coarse-grained film magnetisation and topological charge."""
        na, nb = C.c_int32(), C.c_int32()
        _check(lib().sl_texture_map(self.handle, int(normal), float(cell), C.byref(na), C.byref(nb), None, None))
        m = np.zeros((nb.value, na.value, 3))
        q = C.c_double()
        _check(lib().sl_texture_map(self.handle, int(normal), float(cell), C.byref(na), C.byref(nb), _ptr(m),
                                    C.byref(q)))
        return m, float(q.value)

    def autotune(self, repeats: int = 5) -> dict:
        """Pick the evaluation kernels' launch shapes by timing (sl_autotune)."""
        ch = np.zeros(4, dtype=np.int32)
        b, a = C.c_double(), C.c_double()
        _check(lib().sl_autotune(self.handle, int(repeats), _ptr(ch), C.byref(b), C.byref(a)))
        return dict(crad_block=int(ch[0]), ang_block=int(ch[1]), bwd_block=int(ch[2]), mlp_ctas_per_sm=int(ch[3]),
                    eval_ms_before=b.value, eval_ms_after=a.value)

    def launch_config(self) -> dict:
        """Current launch shapes of the evaluation kernels and the last autotuning landscape
        (sl_get_launch_config)."""
        cfg = np.zeros(8, dtype=np.int32)
        land = np.zeros(16)
        _check(lib().sl_get_launch_config(self.handle, _ptr(cfg), _ptr(land)))
        names = ("radial", "angular", "network", "backward")
        return dict(crad_block=int(cfg[0]), crad_minb=int(cfg[1]), ang_block=int(cfg[2]), ang_minb=int(cfg[3]),
                    bwd_block=int(cfg[4]), bwd_minb=int(cfg[5]), mlp_ctas_per_sm=int(cfg[6]),
                    landscape_ms=[{k: float(land[4 * c + g]) for g, k in enumerate(names)} for c in range(4)
                                  if land[4 * c] >= 0])

    def midpoint_evaluations(self) -> int:
        v = C.c_int64()
        _check(lib().sl_get_midpoint_evaluations(self.handle, C.byref(v)))
        return int(v.value)

    def step(self, n_steps: int, dt: float, T: float, B=(0.0, 0.0, 0.0)):
        Bv = _f64(B)
        _check(lib().sl_step(self.handle, int(n_steps), float(dt), float(T), _ptr(Bv)))

    def energy_forces_fields(self, want_virial=True):
        E = np.zeros(1)
        F = np.zeros((self.n, 3))
        H = np.zeros((self.n, 3))
        W = np.zeros(9) if want_virial else None
        _check(lib().sl_energy_forces_fields(self.handle, _ptr(E), _ptr(F), _ptr(H), _ptr(W)))
        return dict(E=float(E[0]), F=F, H=H, W=None if W is None else W.reshape(3, 3))

    def get_descriptors(self):
        q = np.zeros((self.n, 66))
        e = np.zeros(self.n)
        _check(lib().sl_get_descriptors(self.handle, _ptr(q), _ptr(e)))
        return q, e

    def get_state(self):
        p, v, s, f, h, r = (np.zeros((self.n, 3)) for _ in range(6))
        st = C.c_uint64()
        _check(lib().sl_get_state(self.handle, _ptr(p), _ptr(v), _ptr(s), _ptr(f), _ptr(h), _ptr(r), C.byref(st)))
        return dict(positions=p, velocities=v, spins=s, forces=f, fields=h, ref_positions=r, step=int(st.value))

    def set_state(self, positions, velocities, spins, forces=None, fields=None, step=0, ref_positions=None):
        p, v, s = _f64(positions), _f64(velocities), _f64(spins)
        f = None if forces is None else _f64(forces)
        h = None if fields is None else _f64(fields)
        r = None if ref_positions is None else _f64(ref_positions)
        _check(lib().sl_set_state(self.handle, _ptr(p), _ptr(v), _ptr(s), _ptr(f), _ptr(h), _ptr(r), int(step)))

    def get_neighbors(self, cap=256):
        cr = np.zeros(self.n, np.int32)
        ca = np.zeros(self.n, np.int32)
        lr = np.zeros((self.n, cap), np.int32)
        la = np.zeros((self.n, cap), np.int32)
        _check(lib().sl_get_neighbors(self.handle, cap, _ptr(cr), _ptr(lr), _ptr(ca), _ptr(la)))
        return [lr[i, :cr[i]].copy() for i in range(self.n)], [la[i, :ca[i]].copy() for i in range(self.n)]

    def info(self):
        n, p, b, k = C.c_int64(), C.c_int32(), C.c_int64(), C.c_int64()
        _check(lib().sl_get_info(self.handle, C.byref(n), C.byref(p), C.byref(b), C.byref(k)))
        return dict(n_atoms=n.value, precision=p.value, n_builds=b.value, n_launches=k.value)

    def step_profiled(self, n_steps: int, dt: float, T: float, B=(0.0, 0.0, 0.0)):
        """Steps without graphs, CUDA-event timed per kernel group; returns {group: ms summed}."""
        Bv = _f64(B)
        ms = np.zeros(len(KERNEL_GROUPS))
        _check(lib().sl_step_profiled(self.handle, int(n_steps), float(dt), float(T), _ptr(Bv), _ptr(ms)))
        return dict(zip(KERNEL_GROUPS, ms.tolist()))

    def stream(self) -> int:
        return int(lib().sl_get_stream(self.handle) or 0)

    def destroy(self):
        if getattr(self, "handle", None):
            lib().sl_destroy_system(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Batch:
    """Replicas stepped together (sl_batch_*), in fixed slots; None is an empty slot."""

    def __init__(self, systems):
        self.systems = list(systems)
        arr = (C.c_void_p * len(self.systems))(*[s.handle if s is not None else None for s in self.systems])
        h = C.c_void_p()
        _check(lib().sl_batch_create(arr, len(self.systems), C.byref(h)))
        self.handle = h

    def set(self, slot: int, system):
        """Put `system` into `slot` (None: empty the slot)."""
        _check(lib().sl_batch_set(self.handle, int(slot), system.handle if system is not None else None))
        self.systems[slot] = system

    def _args(self, n_steps, dt, T, B):
        k = len(self.systems)
        ns = np.array(np.broadcast_to(n_steps, (k,)), dtype=np.int64)
        ns[[i for i, x in enumerate(self.systems) if x is None]] = 0   # empty slots take no steps
        d = np.ascontiguousarray(np.broadcast_to(dt, (k,)), dtype=np.float64)
        t = np.ascontiguousarray(np.broadcast_to(T, (k,)), dtype=np.float64)
        b = np.ascontiguousarray(np.broadcast_to(np.asarray(B, dtype=np.float64), (k, 3)))
        return ns, d, t, b

    def step(self, n_steps, dt, T, B):
        ns, d, t, b = self._args(n_steps, dt, T, B)
        _check(lib().sl_batch_step(self.handle, _ptr(ns), _ptr(d), _ptr(t), _ptr(b)))

    def submit(self, n_steps, dt, T, B):
        """Queue the steps and return at once; wait() finishes them."""
        ns, d, t, b = self._args(n_steps, dt, T, B)
        _check(lib().sl_batch_submit(self.handle, _ptr(ns), _ptr(d), _ptr(t), _ptr(b)))

    def wait(self):
        _check(lib().sl_batch_wait(self.handle))

    def graph_launches(self) -> int:
        v = C.c_int64()
        _check(lib().sl_batch_graph_launches(self.handle, C.byref(v)))
        return int(v.value)

    def stats(self) -> dict:
        v = (C.c_int64 * 7)()
        _check(lib().sl_batch_stats(self.handle, v))
        return dict(graph_launches=v[0], fused_captures=v[1], fused_steps=v[2], kernel_launches=v[3],
                    fused_calls=v[4], replica_calls=v[5], atom_capacity=v[6])

    def reserve(self, atoms: int):
        """Size the fused launches for up to `atoms` atoms over all slots."""
        _check(lib().sl_batch_reserve(self.handle, int(atoms)))

    def destroy(self):
        if getattr(self, "handle", None):
            lib().sl_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def sl_create_system(*args, **kw) -> System:
    return System(*args, **kw)


def sl_selftest_harmonics(n_samples=1000):
    a, g = C.c_double(), C.c_double()
    _check(lib().sl_selftest_harmonics(int(n_samples), C.byref(a), C.byref(g)))
    return a.value, g.value


def sl_selftest_carrier(n_samples=100000, rc=6.0):
    """(relative error of f_k, of df_k/dr) of the FP32 radial carrier against FP64 on the device."""
    a, b = C.c_double(), C.c_double()
    _check(lib().sl_selftest_carrier(int(n_samples), float(rc), C.byref(a), C.byref(b)))
    return a.value, b.value


def sl_measure_fma_peak(precision=SL_PREC_MIXED):
    """(FLOP/s, elapsed ms) of the FMA microbenchmark on the current device."""
    f, t = C.c_double(), C.c_double()
    _check(lib().sl_measure_fma_peak(int(precision), C.byref(f), C.byref(t)))
    return f.value, t.value


def sl_descriptors_energies_noalloc(positions4_ptr: int, spins4_ptr: int, species_ptr: int, n: int, box, periodic,
                                    params: dict, q_ptr: int | None, energy_ptr: int, stream_ptr: int | None = None):
    """Descriptors and network energies of a small system without any device
    allocation.  All *_ptr are device addresses owned by the caller (positions4 and
    spins4 [n][4] float64, species [n] int32, q [n][66] float64 or None, energy [n]
    float64); see spinlat.h for the limits and the shared-scratch caveat."""
    P = NepParams(params)
    b = _f64(box)
    per = np.ascontiguousarray(periodic, dtype=np.int32)
    _check(lib().sl_descriptors_energies_noalloc(positions4_ptr, spins4_ptr, species_ptr, int(n), _ptr(b), _ptr(per),
                                                 C.byref(P.struct), q_ptr, energy_ptr, stream_ptr))


def sl_estimate_device_bytes(n: int, precision=SL_PREC_MIXED, cap_rad=160, cap_ang=64) -> int:
    o = sl_default_options()
    o.precision, o.nbr_cap_rad, o.nbr_cap_ang = int(precision), int(cap_rad), int(cap_ang)
    return int(lib().sl_estimate_device_bytes(int(n), C.byref(o)))


def system_from_workload(wl, params: dict, **kw) -> System:
    return System(wl.positions, wl.spins, wl.box, wl.periodic, wl.species, params, wl.velocities,
                  seed=kw.pop("seed", wl.seed), **kw)
