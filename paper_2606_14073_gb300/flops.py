"""Algorithmic work of one NEP-SPIN evaluation, per atom.

Counts what the method has to compute (multiply-add = 2 FLOP, a transcendental
= 1), not what a kernel executes: the roofline fraction of a kernel is this
count divided by its measured time and by the ALU peak, so redundant work in a
kernel shows up as a lower fraction.

Inputs: N_R = mean number of neighbours inside rc_rad (6 A) and N_A inside rc_ang
(4 A) per atom; on the FeGe B20 crystal (8 atoms / 4.70^3 A^3) N_R ~ 69.7, N_A ~ 20.7.

descriptor (k_fwd):
  radial pair   geometry 13 + carrier 47 + spin products 31 + basis sums 81     = 172
  angular pair  geometry 13 + carrier 47 + g_n 90 + spin weight 10 + 24 solid
                harmonics 60 + 240 angular sums x 2                              = 700
  per atom      contraction with the coefficients for 2 neighbour species 900
                + 240 squared sums into q 720                                   = 1620
network (k_mlp): two 66x30 contractions (forward, input gradient) + tanh + scaling = 8206
backward (k_bwd):
  per atom      angular adjoints 720 + coefficient precontraction 900          = 1620
  radial pair   geometry 13 + carrier and slope 75 + 5 group values/slopes 162
                + spin functions and tangential gradients 130                    = 380
  angular pair  carrier and slope 75 + g_n, g_n' 180 + per harmonic 66 x 24
                + assembly 11                                                    = 1850
"""
from __future__ import annotations

FWD_RADIAL_PAIR = 172
FWD_ANGULAR_PAIR = 700
FWD_ATOM = 1620
NETWORK_ATOM = 2 * (66 * 30 * 2) + 66 + 30 * 5 + 30 * 2 + 66
BWD_ATOM = 1620
BWD_RADIAL_PAIR = 380
BWD_ANGULAR_PAIR = 1850


# split of the per-atom terms between the radial and angular kernels
FWD_ATOM_RAD = 900       # coefficient contraction, 2 neighbour species
FWD_ATOM_ANG = 720       # squared angular sums into q
BWD_ATOM_RAD = 900       # coefficient precontraction
BWD_ATOM_ANG = 720       # angular adjoints


def per_atom(n_r: float, n_a: float) -> dict:
    rad_fwd = FWD_ATOM_RAD + FWD_RADIAL_PAIR * n_r
    ang_fwd = FWD_ATOM_ANG + FWD_ANGULAR_PAIR * n_a
    ang_bwd = BWD_ATOM_ANG + BWD_ANGULAR_PAIR * n_a
    rad_bwd = BWD_ATOM_RAD + BWD_RADIAL_PAIR * n_r
    total = rad_fwd + ang_fwd + NETWORK_ATOM + ang_bwd + rad_bwd
    return dict(rad_fwd=rad_fwd, ang_fwd=ang_fwd, network=float(NETWORK_ATOM), ang_bwd=ang_bwd, rad_bwd=rad_bwd,
                descriptor=rad_fwd + ang_fwd, backward=ang_bwd + rad_bwd, total=total)


def crystal_counts() -> tuple[float, float]:
    import math
    rho = 8.0 / 4.70 ** 3
    return rho * 4.0 / 3.0 * math.pi * 6.0 ** 3, rho * 4.0 / 3.0 * math.pi * 4.0 ** 3
