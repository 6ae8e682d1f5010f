"""h4d_eval_forces_static serves callers that cannot allocate device memory: it must give
the same forces and energy as h4d_eval_forces while keeping every device buffer in the
library's static scratch array.  Two different calls in a row check that the shared
array's leftover contents from one call do not leak into the next.  This file is
collected last on purpose."""
import math

import numpy as np
import pytest

from paper_2307_11447_gb300 import lib as h4d
from paper_2307_11447_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TWO32 = 4294967296.0


def _quantize(x, L):
    return np.mod(np.rint(np.mod(x, L) / L * TWO32), TWO32) * (L / TWO32)


def _close(Fa, Fb, Ua, Ub):
    frms = math.sqrt((Fb**2).sum(1).mean())
    err = np.linalg.norm(Fa - Fb, axis=1)
    assert np.all(err <= 1e-5 * (np.linalg.norm(Fb, axis=1) + frms))
    assert Ua == pytest.approx(Ub, rel=1e-10, abs=1e-9)


def test_static_scratch_matches_allocating_entry_point_twice():
    # call 1: 1000 ions at density 0.3 in 3D
    cfg1 = wl.lj_config(1000, 0.3, 100)
    x1 = _quantize(wl.lj_positions(500, cfg1["L"], 21), cfg1["L"])
    p1 = h4d.make_params(cfg1)
    Us1, Fs1 = h4d.h4d_eval_forces_static(p1, cfg1["L"], x1)
    Ua1, Fa1 = h4d.h4d_eval_forces(p1, cfg1["L"], x1)
    _close(Fs1, Fa1, Us1, Ua1)
    # call 2: a smaller box with two flyers at altitude and screening, right after call 1
    cfg2 = wl.lj_config(250, 0.2, 100, kappa_sr=0.7)
    x2 = _quantize(wl.lj_positions(125, cfg2["L"], 22), cfg2["L"])
    w2 = np.zeros(250)
    w2[[5, 40]] = 1.25
    p2 = h4d.make_params(cfg2)
    Us2, Fs2 = h4d.h4d_eval_forces_static(p2, cfg2["L"], x2, w2)
    Ua2, Fa2 = h4d.h4d_eval_forces(p2, cfg2["L"], x2, w2)
    _close(Fs2, Fa2, Us2, Ua2)
    assert Us2 != Us1


def test_static_scratch_rejects_oversized_systems():
    cfg = wl.lj_config(20000, 0.3, 100)
    x = wl.lj_positions(10000, cfg["L"], 3)
    with pytest.raises(h4d.H4DError) as ei:
        h4d.h4d_eval_forces_static(h4d.make_params(cfg), cfg["L"], x)
    assert ei.value.code == h4d.H4D_ECAPACITY


def test_static_scratch_rigid_water_and_empty_system():
    """the water path (O/H types, intramolecular exclusions, Kahan force sums) through the
    static scratch, and n = 0, which both entry points accept with U = 0"""
    L = 22.5
    cfg = wl.aq_config(300, 4, L, 10)
    x = _quantize(wl.aqueous_positions(300, 4, L, 12), L)
    p = h4d.make_params(cfg)
    Us, Fs = h4d.h4d_eval_forces_static(p, L, x, n_water=300)
    Ua, Fa = h4d.h4d_eval_forces(p, L, x, n_water=300)
    _close(Fs, Fa, Us, Ua)
    U0s, F0s = h4d.h4d_eval_forces_static(p, L, np.zeros((0, 3)))
    U0a, F0a = h4d.h4d_eval_forces(p, L, np.zeros((0, 3)))
    assert U0s == U0a == 0.0 and F0s.shape == F0a.shape == (0, 3)
