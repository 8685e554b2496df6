"""ctypes front end of the plain FP64 CPU oracle (oracle/nepspin_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test-suite, by the smoke check and by
the benchmark's CPU-baseline leg, never by the product path.  It shares no code
with the CUDA library.

Every function here forwards to the C oracle; see the header comment of
nepspin_oracle.c for the definitions (paper Sections 3, 5.1.1-5.1.3, 5.2.1-5.2.4)
and the readings taken where the paper prints no formula.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nepspin_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

KB = 8.617333262e-5
HBAR = 0.6582119569
MUB = 5.7883818060e-5
ACC = 9.6485332e-3


def build(force: bool = False) -> str:
    """Compile the oracle with the system C compiler (gcc), -ffp-contract=off."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["cc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("n_ch", C.c_int32), ("basis_k", C.c_int32),
                ("n_hidden", C.c_int32), ("rc_rad", C.c_double), ("rc_ang", C.c_double),
                ("coeffs", C.c_void_p), ("q_scaler", C.c_void_p), ("w0", C.c_void_p),
                ("b0", C.c_void_p), ("w1", C.c_void_p), ("b1", C.c_double),
                ("mass_amu", C.c_void_p), ("moment_muB", C.c_void_p), ("B_atoms", C.c_void_p),
                ("landau", C.c_void_p)]


class _Dyn(C.Structure):
    _fields_ = [("gamma_lattice", C.c_double), ("lambda_spin", C.c_double),
                ("seed", C.c_uint64), ("replica", C.c_uint64),
                ("midpoint_iters", C.c_int32), ("anderson_depth", C.c_int32),
                ("midpoint_tol", C.c_double), ("anderson_reg", C.c_double),
                ("longitudinal", C.c_int32), ("alpha_long", C.c_double), ("st_sweep", C.c_int32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            P, D, I = C.c_void_p, C.c_double, C.c_int64
            _lib.or_philox4x64_10.argtypes = [P, P, P]
            _lib.or_gauss4.argtypes = [C.c_uint64] * 5 + [P]
            _lib.or_chebyshev.argtypes = [D, C.c_int, P, P]
            _lib.or_carrier.argtypes = [D, D, C.c_int, P, P]
            _lib.or_neighbors.argtypes = [I, P, P, P, D, C.c_int, C.c_int32, P, P]
            _lib.or_descriptors.argtypes = [I, P, P, P, P, P, P, P]
            _lib.or_evaluate.argtypes = [I, P, P, P, P, P, P, P, P, P, P, P, P]
            _lib.or_evaluate_subset.argtypes = [I, P, P, P, P, P, P, P, I, P, P, P, P]
            _lib.or_run.argtypes = [I, P, P, P, P, P, P, P, P, I, D, D, P, C.c_uint64, P, P, C.c_int, P]
            _lib.or_rotate.argtypes = [P, P, D, P]
            for f in ("or_neighbors", "or_descriptors", "or_evaluate", "or_evaluate_subset", "or_run"):
                getattr(_lib, f).restype = C.c_int
            _lib.or_num_threads.restype = C.c_int
            _lib.or_set_num_threads.argtypes = [C.c_int]
            _lib.or_colour.argtypes = [I, P, P, P, D, P]
            _lib.or_colour.restype = C.c_int
            _lib.or_set_num_threads.restype = None
        return _lib


def _p(a):
    return a.ctypes.data if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Model:
    """NEP-SPIN parameters in the oracle's layout (see nep_params in the package)."""

    def __init__(self, p: dict, landau=None):
        """landau: optional [n_species][2] (a, b) of the onsite energy a|S|^2 + b|S|^4 (eV)."""
        self.landau = None if landau is None else _f64(landau).reshape(-1, 2).ravel().copy()
        self.n_species = int(p["n_species"])
        self.n_ch = int(p["n_ch"])
        self.basis_k = int(p["basis_k"])
        self.n_hidden = int(p["n_hidden"])
        self.rc_rad = float(p["rc_rad"])
        self.rc_ang = float(p["rc_ang"])
        self.coeffs = _f64(p["coeffs"]).ravel()
        self.q_scaler = _f64(p["q_scaler"]).ravel()
        self.w0 = _f64(p["w0"]).ravel()
        self.b0 = _f64(p["b0"]).ravel()
        self.w1 = _f64(p["w1"]).ravel()
        self.b1 = float(p["b1"])
        self.mass = _f64(p["mass_amu"]).ravel()
        self.moment = _f64(p["moment_muB"]).ravel()
        self.dim = 1 + 13 * self.n_ch

    def c_struct(self, B_atoms=None) -> _Params:
        """The C parameter block; B_atoms ([n][3] tesla, FP64 C-contiguous, kept alive by the
        caller) is the optional per-atom part of the external field."""
        s = _Params()
        s.n_species, s.n_ch, s.basis_k, s.n_hidden = self.n_species, self.n_ch, self.basis_k, self.n_hidden
        s.rc_rad, s.rc_ang = self.rc_rad, self.rc_ang
        s.coeffs, s.q_scaler, s.w0 = _p(self.coeffs), _p(self.q_scaler), _p(self.w0)
        s.b0, s.w1, s.b1 = _p(self.b0), _p(self.w1), self.b1
        s.mass_amu, s.moment_muB = _p(self.mass), _p(self.moment)
        s.B_atoms = None if B_atoms is None else _p(B_atoms)
        s.landau = _p(self.landau)
        return s


def _sys(pos, spin, species, box, periodic):
    return (_f64(pos), _f64(spin), np.ascontiguousarray(species, dtype=np.int32), _f64(box),
            np.ascontiguousarray(periodic, dtype=np.int32))


def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().or_philox4x64_10(_p(c), _p(k), _p(out))
    return out


def gauss4(step, atom, stream, seed, replica):
    out = np.zeros(4)
    lib().or_gauss4(step, atom, stream, seed, replica, _p(out))
    return out


def chebyshev(x, K):
    T, dT = np.zeros(K), np.zeros(K)
    lib().or_chebyshev(float(x), K, _p(T), _p(dT))
    return T, dT


def carrier(r, rc, K):
    f, df = np.zeros(K), np.zeros(K)
    lib().or_carrier(float(r), float(rc), K, _p(f), _p(df))
    return f, df


def rotate(S, w, dt):
    out = np.zeros(3)
    lib().or_rotate(_p(_f64(S)), _p(_f64(w)), float(dt), _p(out))
    return out


def neighbors(pos, box, periodic, cut, method=0, cap=256):
    pos, box, periodic = _f64(pos), _f64(box), np.ascontiguousarray(periodic, dtype=np.int32)
    n = pos.shape[0]
    counts = np.zeros(n, dtype=np.int32)
    lists = np.zeros((n, cap), dtype=np.int32)
    rc = lib().or_neighbors(n, _p(pos), _p(box), _p(periodic), float(cut), int(method), cap, _p(counts), _p(lists))
    if rc == -2:
        raise OverflowError("neighbour count above cap")
    if rc:
        raise RuntimeError(f"or_neighbors failed: {rc}")
    return [lists[i, :counts[i]].copy() for i in range(n)]


def descriptors(model: Model, pos, spin, species, box, periodic):
    pos, spin, species, box, periodic = _sys(pos, spin, species, box, periodic)
    q = np.zeros((pos.shape[0], model.dim))
    P = model.c_struct()
    rc = lib().or_descriptors(pos.shape[0], _p(pos), _p(spin), _p(species), _p(box), _p(periodic),
                              C.addressof(P), _p(q))
    if rc:
        raise RuntimeError(f"or_descriptors failed: {rc}")
    return q


def _batoms(B_atoms, n):
    if B_atoms is None:
        return None
    b = _f64(B_atoms)
    if b.shape != (n, 3):
        raise ValueError("B_atoms must have shape (n, 3)")
    return b


def evaluate(model: Model, pos, spin, species, box, periodic, B=(0.0, 0.0, 0.0), B_atoms=None):
    """Returns dict(E, Ei, F, H, W) at FP64; B_atoms is the optional per-atom field part."""
    pos, spin, species, box, periodic = _sys(pos, spin, species, box, periodic)
    n = pos.shape[0]
    E = np.zeros(1)
    Ei, F, H, W = np.zeros(n), np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(9)
    ba = _batoms(B_atoms, n)
    P = model.c_struct(ba)
    Bv = _f64(B)
    rc = lib().or_evaluate(n, _p(pos), _p(spin), _p(species), _p(box), _p(periodic), C.addressof(P), _p(Bv),
                           _p(E), _p(Ei), _p(F), _p(H), _p(W))
    if rc:
        raise RuntimeError(f"or_evaluate failed: {rc}")
    return dict(E=float(E[0]), Ei=Ei, F=F, H=H, W=W.reshape(3, 3))


def evaluate_subset(model: Model, pos, spin, species, box, periodic, sample, B=(0.0, 0.0, 0.0), B_atoms=None):
    pos, spin, species, box, periodic = _sys(pos, spin, species, box, periodic)
    sample = np.ascontiguousarray(sample, dtype=np.int64)
    m = sample.shape[0]
    F, H, Ei = np.zeros((m, 3)), np.zeros((m, 3)), np.zeros(m)
    ba = _batoms(B_atoms, pos.shape[0])
    P = model.c_struct(ba)
    Bv = _f64(B)
    rc = lib().or_evaluate_subset(pos.shape[0], _p(pos), _p(spin), _p(species), _p(box), _p(periodic),
                                  C.addressof(P), _p(Bv), m, _p(sample), _p(F), _p(H), _p(Ei))
    if rc:
        raise RuntimeError(f"or_evaluate_subset failed: {rc}")
    return dict(F=F, H=H, Ei=Ei)


class State:
    """Mutable dynamical state for or_run (arrays in caller atom order)."""

    def __init__(self, pos, vel, spin, species, box, periodic):
        self.pos, self.spin, self.species, self.box, self.periodic = _sys(pos, spin, species, box, periodic)
        self.pos = self.pos.copy()
        self.spin = self.spin.copy()
        self.vel = _f64(vel).copy()
        n = self.pos.shape[0]
        self.F = np.zeros((n, 3))
        self.H = np.zeros((n, 3))
        self.have_fh = False
        self.step = 0


def run(model: Model, st: State, n_steps: int, dt: float, T: float, B=(0.0, 0.0, 0.0), *,
        gamma=0.01, lam=0.1, seed=1234, replica=0, midpoint_iters=0, midpoint_tol=0.0, anderson_depth=0,
        anderson_reg=1e-10, B_atoms=None, longitudinal=False, alpha_long=0.0, st_sweep=False):
    """Advance st by n_steps steps (or_run).  midpoint_iters > 0 selects the self-consistent
    midpoint spin update (cap of the iteration, tolerance midpoint_tol, optional Anderson
    history anderson_depth with relative regularisation anderson_reg).  Returns st; the
    number of midpoint evaluations of the call is in st.last_iterations.  B_atoms is the
    optional per-atom part of the external field ([n][3] tesla).  longitudinal=True frees the
    moment lengths (Langevin form with longitudinal damping alpha_long; lam is then unused).
    st_sweep=True replaces the predictor-corrector spin update by the coloured Suzuki-Trotter
    sweep (or_colour colouring at the new positions, 2C + 1 evaluations per step)."""
    ba = _batoms(B_atoms, st.pos.shape[0])
    P = model.c_struct(ba)
    dyn = _Dyn(gamma, lam, seed, replica, int(midpoint_iters), int(anderson_depth), float(midpoint_tol),
               float(anderson_reg), int(bool(longitudinal)), float(alpha_long), int(bool(st_sweep)))
    Bv = _f64(B)
    it = np.zeros(1, dtype=np.int64)
    rc = lib().or_run(st.pos.shape[0], _p(st.pos), _p(st.vel), _p(st.spin), _p(st.species), _p(st.box),
                      _p(st.periodic), C.addressof(P), C.addressof(dyn), int(n_steps), float(dt), float(T),
                      _p(Bv), int(st.step), _p(st.F), _p(st.H), int(st.have_fh), _p(it))
    if rc:
        raise RuntimeError(f"or_run failed: {rc}")
    st.have_fh = True
    st.step += int(n_steps)
    st.last_iterations = int(it[0])
    return st


def num_threads() -> int:
    return int(lib().or_num_threads())


def colour(pos, box, periodic, rc):
    """Greedy colouring (index order) of the conflict graph d < 2 rc (or_colour): (colours, count)."""
    pos, box = _f64(pos), _f64(box)
    periodic = np.ascontiguousarray(periodic, dtype=np.int32)
    col = np.zeros(pos.shape[0], dtype=np.int32)
    nc = lib().or_colour(pos.shape[0], _p(pos), _p(box), _p(periodic), float(rc), _p(col))
    if nc < 0:
        raise RuntimeError(f"or_colour failed: {nc}")
    return col, int(nc)


def set_num_threads(t: int):
    lib().or_set_num_threads(int(t))


def kinetic_energy(vel, species, masses):
    m = np.asarray(masses)[np.asarray(species)]
    return 0.5 * float((m[:, None] * np.asarray(vel) ** 2).sum()) / ACC
