"""Texture diagnostics of a film: coarse-grained magnetisation and topological charge.

TEST INFRASTRUCTURE ONLY: used by the test-suite to check the library's on-device
diagnostics; the product path never imports it.

The paper follows helix-to-skyrmion textures in a thin FeGe stripe (Fig. 7 and
Section 8).  The quantities, written from their definitions:
  * the in-plane grid: the two axes other than the film normal, each cut into
    n = max(1, floor(L / cell)) equal cells; atoms beyond a non-periodic edge go to the
    edge cell;
  * m(cell) = sum of the spins in the column over the cell, normalised (left zero
    when the column is empty or the sum vanishes);
  * the lattice topological charge of Berg and Luescher (Nucl. Phys. B 190 (1981) 412):
    every plaquette (a, b) -> (a+1, b) -> (a+1, b+1) -> (a, b+1) is cut into the two
    counter-clockwise triangles (m00, m10, m11) and (m00, m11, m01); the signed solid
    angle of a triangle of unit vectors is 2 atan2(m1.(m2 x m3), 1 + m1.m2 + m2.m3 + m3.m1)
    (Van Oosterom and Strackee, IEEE Trans. Biomed. Eng. 30 (1983) 125), and
    Q = sum of the solid angles / (4 pi).  Plaquettes wrap across periodic axes and stop
    at non-periodic edges; triangles with an empty cell contribute nothing.
With this orientation a core-up skyrmion in a down background with vorticity +1 has
Q = +1, the continuum value of (1/4 pi) int m.(d_a m x d_b m) da db.
"""
from __future__ import annotations

import math

import numpy as np


def grid_axes(normal: int):
    return [a for a in range(3) if a != normal]


def grid_shape(box, normal: int, cell: float):
    a, b = grid_axes(normal)
    return max(1, int(math.floor(box[b] / cell))), max(1, int(math.floor(box[a] / cell)))


def magnetisation_map(pos, spin, box, periodic, normal: int = 2, cell: float = 4.7):
    """m[nb][na][3]: normalised column sums of the spins over the in-plane grid."""
    pos = np.asarray(pos, dtype=np.float64)
    spin = np.asarray(spin, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    a, b = grid_axes(normal)
    nb, na = grid_shape(box, normal, cell)
    idx = []
    for ax, n in ((a, na), (b, nb)):
        w = box[ax] / n
        k = np.floor(pos[:, ax] / w).astype(np.int64)
        k = np.mod(k, n) if periodic[ax] else np.clip(k, 0, n - 1)
        idx.append(k)
    ia, ib = idx
    acc = np.zeros((nb, na, 3))
    for c in range(3):
        np.add.at(acc[:, :, c], (ib, ia), spin[:, c])
    norm = np.linalg.norm(acc, axis=2)
    m = np.zeros_like(acc)
    ok = norm > 0
    m[ok] = acc[ok] / norm[ok][:, None]
    return m


def solid_angle(m1, m2, m3):
    """Signed solid angle of the spherical triangle of unit vectors (rows)."""
    num = np.einsum("...i,...i", m1, np.cross(m2, m3))
    den = 1.0 + np.einsum("...i,...i", m1, m2) + np.einsum("...i,...i", m2, m3) + np.einsum("...i,...i", m3, m1)
    return 2.0 * np.arctan2(num, den)


def topological_charge(m, periodic_a: bool, periodic_b: bool) -> float:
    """Berg-Luescher charge of a grid m[nb][na][3] of unit (or zero) vectors."""
    nb, na, _ = m.shape
    ra = range(na) if periodic_a else range(na - 1)
    rb = range(nb) if periodic_b else range(nb - 1)
    total = 0.0
    empty = np.linalg.norm(m, axis=2) == 0
    for j in rb:
        j1 = (j + 1) % nb
        for i in ra:
            i1 = (i + 1) % na
            m00, m10, m11, m01 = m[j, i], m[j, i1], m[j1, i1], m[j1, i]
            e00, e10, e11, e01 = empty[j, i], empty[j, i1], empty[j1, i1], empty[j1, i]
            if not (e00 or e10 or e11):
                total += float(solid_angle(m00, m10, m11))
            if not (e00 or e11 or e01):
                total += float(solid_angle(m00, m11, m01))
    return total / (4.0 * math.pi)


def texture(pos, spin, box, periodic, normal: int = 2, cell: float = 4.7):
    """(m map, Q) of the configuration."""
    m = magnetisation_map(pos, spin, box, periodic, normal, cell)
    a, b = grid_axes(normal)
    return m, topological_charge(m, bool(periodic[a]), bool(periodic[b]))
