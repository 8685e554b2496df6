"""The C ABI used from plain C11 (tests/c_abi_client.c): the header compiles as C with
warnings as errors and the client links against the library (CPU); on a GPU the client's
results equal the Python binding's bit for bit and the FP64 oracle's to 1e-10."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_14073_gb300 import build as B
from paper_2606_14073_gb300 import nep_params, spinlat as S, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _compile(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = B.build()
    exe = tmp_path / "c_abi_client"
    cmd = [cc, "-std=c11", "-O2", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_abi_client.c"), "-L", os.path.dirname(lib), "-lspinlat",
           "-Wl,-rpath," + os.path.dirname(lib), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def _write_input(path, wl, p):
    with open(path, "wb") as f:
        f.write(np.int64(wl.n).tobytes())
        f.write(np.asarray(wl.box, np.float64).tobytes())
        f.write(np.asarray(wl.periodic, np.int32).tobytes())
        f.write(np.array([p["n_species"], p["n_ch"], 4, p["basis_k"], p["n_hidden"]], np.int32).tobytes())
        f.write(np.array([p["rc_rad"], p["rc_ang"], p["b1"]], np.float64).tobytes())
        for k in ("coeffs", "q_scaler", "w0", "b0", "w1", "mass_amu", "moment_muB"):
            f.write(np.ascontiguousarray(p[k], np.float64).tobytes())
        f.write(np.asarray(wl.species, np.int32).tobytes())
        for a in (wl.positions, wl.spins, wl.velocities):
            f.write(np.ascontiguousarray(a, np.float64).tobytes())


def test_c_client_compiles_and_links(tmp_path):
    exe = _compile(tmp_path)
    assert exe.exists()


@pytest.mark.gpu
def test_c_client_matches_python_binding_and_oracle(tmp_path):
    p = nep_params.load()
    wl = W.fege_small()
    exe = _compile(tmp_path)
    inp, outp = tmp_path / "in.bin", tmp_path / "out.bin"
    _write_input(inp, wl, p)
    r = subprocess.run([str(exe), str(inp), str(outp)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    raw = np.fromfile(outp, dtype=np.float64)
    n = wl.n
    E0, F0, H0 = raw[0], raw[1:1 + 3 * n].reshape(n, 3), raw[1 + 3 * n:1 + 6 * n].reshape(n, 3)
    pos1 = raw[1 + 6 * n:1 + 9 * n].reshape(n, 3)
    spin1 = raw[1 + 9 * n:1 + 12 * n].reshape(n, 3)
    E1 = raw[1 + 12 * n]
    step = int(raw[2 + 12 * n:3 + 12 * n].view(np.int64)[0])
    # the same calls through the Python binding
    s = S.System(wl.positions, wl.spins, wl.box, wl.periodic, wl.species, p, wl.velocities)
    r0 = s.energy_forces_fields(want_virial=False)
    assert r0["E"] == E0 and np.array_equal(r0["F"], F0) and np.array_equal(r0["H"], H0)
    s.step(10, 1.0, 300.0, (0.0, 0.0, 0.5))
    st = s.get_state()
    assert np.array_equal(st["positions"], pos1) and np.array_equal(st["spins"], spin1) and step == 10
    assert s.energy_forces_fields(want_virial=False)["E"] == E1
    s.destroy()
    # and the oracle at the start state
    ref = O.evaluate(O.Model(p), wl.positions, wl.spins, wl.species, wl.box, wl.periodic)
    assert abs(E0 - ref["E"]) <= 1e-10 * abs(ref["E"])
    assert np.abs(F0 - ref["F"]).max() <= 1e-10 * np.abs(ref["F"]).max()
    assert np.abs(H0 - ref["H"]).max() <= 1e-10 * np.abs(ref["H"]).max()
