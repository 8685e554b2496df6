"""Algorithmic work of one NEP-SPIN evaluation, per atom.

Counts what the method has to compute (add, subtract, multiply, divide = 1 FLOP each, so a
multiply-add is 2; a transcendental = 1), not what a kernel executes: the roofline fraction
of a kernel is this count divided by its measured time and by the ALU peak, so redundant
work in a kernel shows up as a lower fraction.  The numbers are counted, not estimated:
tests/test_flop_count.py runs a plain restatement of the method (harmonic form of the
angular channels, coefficient contractions hoisted out of the pair loops as Section 5.2.4
does with its precomputed fp.dC and fp.Cv products) over an operation-counting number
type, checks that it reproduces the oracle's descriptors, energies, forces and fields,
and requires the constants below to equal its counts.

Inputs: N_R = mean number of neighbours inside rc_rad (6 A) and N_A inside rc_ang (4 A)
per atom; on the FeGe B20 crystal (8 atoms / 4.70^3 A^3) N_R ~ 69.7, N_A ~ 20.7.

descriptor:
  radial pair   geometry 13 + carrier 41 + spin products 31 + basis sums 81       = 166
  angular pair  (geometry shared) carrier 41 + g_n 85 + spin weight 5
                + 24 solid harmonics 53 + 240 angular sums x 2                    = 664
  per atom      coefficient contraction, 2 neighbour species, 875 + onsite 5       = 880
                240 squared sums into q                                           = 680
network: scaling 66 + 30 pre-activations 3960 + tanh 30 + output 60 + gradient
         of the 30 units 90 + 66x30 input gradient 3894 + scaling 66              = 8166
backward:
  per atom      angular adjoints 2 kappa Fp B                                     = 480
                coefficient precontraction C^G_k = sum_n Fp c 810 + onsite 4      = 814
  radial pair   geometry 13 + carrier and slope 98 + group values and slopes 153
                + spin functions, force and field terms 129                       = 393
  angular pair  carrier and slope 98 + g_n, g_n' 170 + harmonics and gradients 157
                + 24 harmonic contractions and assembly 1243                      = 1668
gather: one record (force and field parts) per ordered in-cutoff pair            = 6
"""
from __future__ import annotations

FWD_RADIAL_PAIR = 166
FWD_ANGULAR_PAIR = 664
FWD_ATOM_RAD = 880       # coefficient contraction for 2 neighbour species, onsite channel
FWD_ATOM_ANG = 680       # squared angular sums into q
FWD_ATOM = FWD_ATOM_RAD + FWD_ATOM_ANG
NETWORK_ATOM = 8166
BWD_ATOM_RAD = 814       # coefficient precontraction, onsite field
BWD_ATOM_ANG = 480       # angular adjoints
BWD_ATOM = BWD_ATOM_RAD + BWD_ATOM_ANG
BWD_RADIAL_PAIR = 393
BWD_ANGULAR_PAIR = 1668
GATHER_PAIR = 6


def per_atom(n_r: float, n_a: float) -> dict:
    rad_fwd = FWD_ATOM_RAD + FWD_RADIAL_PAIR * n_r
    ang_fwd = FWD_ATOM_ANG + FWD_ANGULAR_PAIR * n_a
    ang_bwd = BWD_ATOM_ANG + BWD_ANGULAR_PAIR * n_a
    rad_bwd = BWD_ATOM_RAD + BWD_RADIAL_PAIR * n_r
    gather = GATHER_PAIR * n_r
    total = rad_fwd + ang_fwd + NETWORK_ATOM + ang_bwd + rad_bwd + gather
    return dict(rad_fwd=rad_fwd, ang_fwd=ang_fwd, network=float(NETWORK_ATOM), ang_bwd=ang_bwd, rad_bwd=rad_bwd,
                descriptor=rad_fwd + ang_fwd, backward=ang_bwd + rad_bwd, gather=gather, total=total)


def crystal_counts() -> tuple[float, float]:
    import math
    rho = 8.0 / 4.70 ** 3
    return rho * 4.0 / 3.0 * math.pi * 6.0 ** 3, rho * 4.0 / 3.0 * math.pi * 4.0 ** 3
