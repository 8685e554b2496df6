"""Write the random-init NEP-SPIN parameter file used by every workload.

The paper's trained FeGe model is not available, so a random model of the same
shape stands in for it: 2 species, 5 radial/angular channels, 9 Chebyshev terms,
l_max = 4, cutoffs 6 / 4 A, 30 tanh hidden units (66-entry descriptor).

Recipe (numpy PCG64, seed 7):
  c ~ U(-1, 1)                                   [2][2][6][5][9]
  W0 ~ N(0, 1/66), magnetic columns (EX, DMI, ANI, SIA, SA) scaled by beta
  w1 ~ N(0, 1/30) * alpha,  b1 = 0
  s_v = 1/(max_v - min_v) of q_v over the 512-atom FeGe start state (1 where the
        range is zero, i.e. the onsite channel |S|^2 = 1)
  b0_h = sum_v W0_hv s_v mean_v(q_v)  (centres the pre-activations on that state)
alpha sets RMS|F| = 0.5 eV/A and beta sets the RMS transverse field to 0.05 eV
on that state (one refinement pass each; forces and fields are linear in alpha).

This script calls the oracle only; run it from the repository root:
    python -m oracle.make_nep_params
"""
from __future__ import annotations

import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from oracle import oracle as O  # noqa: E402
from paper_2606_14073_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2606_14073_gb300", "data", "nep_fege_random.npz")

NS, NCH, K, NH = 2, 5, 9, 30
D = 1 + 13 * NCH
F_TARGET = 0.5
HPERP_TARGET = 0.05


def magnetic_columns():
    cols = list(range(NCH + 4 * NCH + 1, D))          # EX, DMI, ANI, SIA, SA
    return np.array(cols)


def base(seed=W.PARAM_SEED):
    rng = np.random.Generator(np.random.PCG64(seed))
    coeffs = rng.uniform(-1.0, 1.0, size=(NS, NS, 6, NCH, K))
    w0 = rng.normal(0.0, np.sqrt(1.0 / D), size=(NH, D))
    w1 = rng.normal(0.0, np.sqrt(1.0 / NH), size=NH)
    return coeffs, w0, w1


def assemble(coeffs, w0, w1, scaler, qmean, alpha, beta):
    w0 = w0.copy()
    w0[:, magnetic_columns()] *= beta
    b0 = w0 @ (scaler * qmean)
    return dict(n_species=NS, n_ch=NCH, basis_k=K, n_hidden=NH, rc_rad=6.0, rc_ang=4.0,
                coeffs=coeffs, q_scaler=scaler, w0=w0, b0=b0, w1=w1 * alpha, b1=0.0,
                mass_amu=np.array(W.MASS_AMU), moment_muB=np.array(W.MOMENT_MUB))


def rms_force_field(p, wl):
    m = O.Model(p)
    r = O.evaluate(m, wl.positions, wl.spins, wl.species, wl.box, wl.periodic)
    F = r["F"]
    H = r["H"]
    Hperp = H - (H * wl.spins).sum(1, keepdims=True) * wl.spins
    return float(np.sqrt((F ** 2).sum(1).mean())), float(np.sqrt((Hperp ** 2).sum(1).mean()))


def main():
    wl = W.fege_small()
    coeffs, w0, w1 = base()
    probe = assemble(coeffs, w0, w1, np.ones(D), np.zeros(D), 1.0, 1.0)
    q = O.descriptors(O.Model(probe), wl.positions, wl.spins, wl.species, wl.box, wl.periodic)
    rng_ = q.max(0) - q.min(0)
    scaler = np.where(rng_ > 1e-12, 1.0 / np.where(rng_ > 1e-12, rng_, 1.0), 1.0)
    qmean = q.mean(0)
    alpha, beta = 1.0, 1.0
    for _ in range(3):
        f, h = rms_force_field(assemble(coeffs, w0, w1, scaler, qmean, alpha, beta), wl)
        alpha *= F_TARGET / f
        f, h = rms_force_field(assemble(coeffs, w0, w1, scaler, qmean, alpha, beta), wl)
        beta *= HPERP_TARGET / h
    p = assemble(coeffs, w0, w1, scaler, qmean, alpha, beta)
    f, h = rms_force_field(p, wl)
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    np.savez(OUT, **p, alpha=alpha, beta=beta, seed=W.PARAM_SEED)
    print(f"wrote {OUT}: alpha={alpha:.6g} beta={beta:.6g} rms|F|={f:.4f} eV/A rms|Hperp|={h:.4f} eV")


if __name__ == "__main__":
    main()
