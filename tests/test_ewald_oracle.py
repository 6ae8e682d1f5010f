"""Pins of the oracle's Ewald sum (the long-range Coulomb part of Sec. II.B.2, Eqs. 9-10).

* Rock salt: a simple cubic lattice of alternating unit charges (spacing r0) has the
  Coulomb energy -(N/2) M K q^2 / r0 with the NaCl Madelung constant M = 1.747564594633.
* The total U_real + U_recip + U_self + U_excl does not depend on the splitting parameter
  alpha (for a neutral system, converged cut-offs): checked on the LJ electrolyte and on
  rigid waters, where the intramolecular exclusion correction enters.
* The reciprocal-space forces are minus the finite-difference gradient of U_recip.
"""
import itertools
import math

import numpy as np

from oracle import oracle as orc
from paper_2307_11447_gb300 import workloads as wl

MADELUNG_NACL = 1.747564594633182  # rock-salt Madelung constant (nearest-neighbour distance 1)


def _rock_salt(m):
    """m^3 sites of a simple cubic lattice, spacing 1, charges (-1)^(i+j+k), ordered as
    interleaved +/- pairs (the oracle types even atoms as cations)"""
    plus, minus = [], []
    for i, j, k in itertools.product(range(m), repeat=3):
        (plus if (i + j + k) % 2 == 0 else minus).append((i + 0.25, j + 0.25, k + 0.25))
    x = np.empty((m**3, 3))
    x[0::2] = plus
    x[1::2] = minus
    return x


def test_rock_salt_madelung_constant():
    m = 8
    x = _rock_salt(m)
    cfg = dict(wl.LJ_PHYSICS, L=float(m), kcoul=1.0, q=[1.0, -1.0], n_f=1)
    e = orc.ewald(orc.make_params(cfg), x, alpha=1.4, kmax=16, rcut=m / 2)
    expect = -0.5 * m**3 * MADELUNG_NACL
    print(f"\nrock salt: U {e['U']:.10f}, -(N/2) M {expect:.10f}")
    assert abs(e["U"] - expect) < 1e-9 * abs(expect)
    # the sign convention of a single term: one pair alone is -K/r plus image terms
    assert e["self"] < 0 and e["recip"] > 0


def test_total_is_independent_of_alpha_lj_electrolyte():
    cfg = dict(wl.CONFIGS["lj250"])
    L = cfg["L"]
    x = wl.lj_positions(cfg["n_pairs"], L, 3)
    p = orc.make_params(cfg)
    a = orc.ewald(p, x, alpha=1.1, kmax=20, rcut=L / 2)
    b = orc.ewald(p, x, alpha=1.5, kmax=27, rcut=L / 2)
    print(f"\nalpha 1.1: {a['U']:.10f} (recip {a['recip']:.6f}); alpha 1.5: {b['U']:.10f} (recip {b['recip']:.6f})")
    assert abs(a["U"] - b["U"]) < 1e-9 * abs(a["U"])
    assert abs(a["recip"] - b["recip"]) > 1.0  # the split itself moves a lot


def test_total_is_independent_of_alpha_rigid_water():
    L = 22.5
    cfg = wl.aq_config(200, 4, L, 10)
    x = wl.aqueous_positions(200, 4, L, 5)
    p = orc.make_params(cfg)
    # alpha rc >= 5.6 and k_max^2 / 4 alpha^2 >= 25: both sums converged below 1e-10
    a = orc.ewald(p, x, alpha=0.5, kmax=18, rcut=L / 2)
    b = orc.ewald(p, x, alpha=0.6, kmax=22, rcut=L / 2)
    print(f"\nwater alpha 0.5: {a['U']:.8f} (excl {a['excl']:.4f}); 0.6: {b['U']:.8f} (excl {b['excl']:.4f})")
    assert abs(a["U"] - b["U"]) < 1e-8 * abs(a["U"])
    assert a["excl"] != 0.0


def test_reciprocal_forces_are_minus_gradient():
    cfg = dict(wl.CONFIGS["lj250"])
    L = cfg["L"]
    x = wl.lj_positions(cfg["n_pairs"], L, 4)
    p = orc.make_params(cfg)
    alpha, kmax = 0.6, 10
    F = orc.ewald(p, x, alpha, kmax, 0.0, forces=True)["F_recip"]
    h = 1e-5
    for i in (0, 7, 100, 249):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, c] += h
            xm[i, c] -= h
            up = orc.ewald(p, xp, alpha, kmax, 0.0)["recip"]
            um = orc.ewald(p, xm, alpha, kmax, 0.0)["recip"]
            fd = -(up - um) / (2 * h)
            assert abs(F[i, c] - fd) < 1e-6 * (abs(fd) + 1.0), (i, c, F[i, c], fd)
