"""Long-range Coulomb term on the GPU (Sec. II.B.2, Eqs. 9-10) against the oracle's Ewald
sum on the same fixed-point positions.

Tolerances from the arithmetic: the GPU sums FP32 terms in tiles of 256 (FP64 across
tiles) with sin/cos of an exactly formed phase, so U_recip agrees to 1e-6 relative and
each atom's reciprocal-space force to 1e-5 (|F| + F_rms); the self energy is FP64 on both
sides (1e-12); the altitude screening multiplies everything by exp(-kappa_lr wbar).
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2307_11447_gb300 import lib as h4d
from paper_2307_11447_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TWO32 = 4294967296.0


def quantize(x, L):
    return np.mod(np.rint(np.mod(x, L) / L * TWO32), TWO32) * (L / TWO32)


def _check(cfg, x, alpha, kmax, n_water=0, f_scale=0.0):
    """f_scale: force scale added to the bound where the exact forces vanish (a perfect
    lattice), so that the relative criterion stays meaningful"""
    L = cfg["L"]
    x = quantize(x, L)
    o = orc.ewald(orc.make_params(cfg), x, alpha, kmax, 0.0, forces=True)
    ur, us, F = h4d.h4d_ewald_lr(h4d.make_params(cfg), L, x, alpha, kmax, n_water=n_water)
    Fo = o["F_recip"]
    frms = np.sqrt((Fo**2).sum(1).mean())
    err = np.linalg.norm(F - Fo, axis=1)
    bound = 1e-5 * (np.linalg.norm(Fo, axis=1) + frms + f_scale)
    print(f"\nU_recip gpu {ur:.10g} oracle {o['recip']:.10g} (rel {abs(ur - o['recip']) / abs(o['recip']):.1e}); "
          f"max force error / bound {(err / bound).max():.3f}")
    assert abs(ur - o["recip"]) <= 1e-6 * abs(o["recip"])
    assert abs(us - o["self"]) <= 1e-12 * abs(o["self"])
    assert np.all(err <= bound)
    return ur, us, F


def test_lj_electrolyte_long_range_term_matches_oracle():
    cfg = dict(wl.CONFIGS["lj250"])
    _check(cfg, wl.lj_positions(cfg["n_pairs"], cfg["L"], 6), alpha=0.6, kmax=10)


def test_rock_salt_long_range_term_matches_oracle():
    m = 6
    plus, minus = [], []
    for i, j, k in itertools.product(range(m), repeat=3):
        (plus if (i + j + k) % 2 == 0 else minus).append((i + 0.5, j + 0.5, k + 0.5))
    x = np.empty((m**3, 3))
    x[0::2], x[1::2] = plus, minus
    cfg = dict(wl.LJ_PHYSICS, L=float(m), kcoul=1.0, n_f=1)
    # every site is a centre of symmetry: the exact forces vanish; K q^2 / r0^2 = 1 sets the scale
    _check(cfg, x, alpha=1.2, kmax=12, f_scale=1.0)


def test_aqueous_long_range_term_matches_oracle():
    L = 22.5
    cfg = wl.aq_config(300, 4, L, 10)
    _check(cfg, wl.aqueous_positions(300, 4, L, 9), alpha=0.3, kmax=9, n_water=300)


def test_altitude_screening_scales_the_long_range_term():
    cfg = dict(wl.CONFIGS["lj250"])
    L = cfg["L"]
    x = quantize(wl.lj_positions(cfg["n_pairs"], L, 7), L)
    p = h4d.make_params(cfg)
    u0, s0, F0 = h4d.h4d_ewald_lr(p, L, x, 0.6, 8)
    u1, s1, F1 = h4d.h4d_ewald_lr(p, L, x, 0.6, 8, wbar=1.5, kappa_lr=0.7)
    g = np.exp(-0.7 * 1.5)
    assert u1 == pytest.approx(g * u0, rel=1e-12) and s1 == pytest.approx(g * s0, rel=1e-12)
    assert np.allclose(F1, g * F0, rtol=1e-12, atol=0)
