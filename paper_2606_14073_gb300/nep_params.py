"""Loader for NEP-SPIN parameter files (.npz).

Layout (all float64 unless stated):
  n_species, n_ch, basis_k, n_hidden   ints (2, 5, 9, 30 for the FeGe model)
  rc_rad, rc_ang                       cutoffs in A (6, 4)
  coeffs      [ns][ns][6][n_ch][basis_k]  group order R, A, EX, DMI, ANI, SIA;
              index [t_i][t_j] = (centre species, neighbour species)
  q_scaler    [66]   descriptor scaler s_v
  w0          [n_hidden][66], b0 [n_hidden], w1 [n_hidden], b1 scalar
  mass_amu    [ns], moment_muB [ns]
Descriptor order: R(5), A(n,l)(20, n-major, l = 1..4), O(1), EX(5), DMI(5),
ANI(5), SIA(5), SA(n,l)(20).

The bundled file data/nep_fege_random.npz is a seeded random-init model of the
paper's FeGe network shape (its trained weights are not published).
"""
from __future__ import annotations

import os

import numpy as np

DEFAULT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "nep_fege_random.npz")


def load(path: str = DEFAULT) -> dict:
    z = np.load(path)
    out = {}
    for k in z.files:
        v = z[k]
        out[k] = v.item() if v.ndim == 0 else np.array(v)
    for k in ("n_species", "n_ch", "basis_k", "n_hidden"):
        out[k] = int(out[k])
    for k in ("rc_rad", "rc_ang", "b1"):
        out[k] = float(out[k])
    return out
