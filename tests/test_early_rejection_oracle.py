"""Early rejection (SI, "Simple, early rejection scheme") in the oracle.

Reading: a cube of volume V_ex centred on the flying cation; a pair whose anion lies
inside it (every axis of the minimum-image fixed-point offset within the half-edge) is
exchanged by an instantaneous MC move -- the trial without NEMD, Delta H = Delta U at
unchanged velocities, no kinetic part -- and any other pair by NEMD.  One rule classifies
insertions and deletions, so every pair geometry has a single kind of move in both
directions and the acceptance rule is unchanged; p_NE = 1 - V_ex/V is then the fraction of
uniform insertions that run NEMD.

Pins: the cube on fixed-point offsets (inside and outside near the half-edge, periodic
wrap, symmetry, the volume fraction it covers); instantaneous trials carry no protocol
work and their Delta H is the potential-energy difference of the two end states computed
directly; the trial's flag is the classification of its pair, for deletions and
insertions alike (a deletion type drawn at random with p_cv, the other way to read the
scheme, fails here).  The stationary <N> of an interacting electrolyte with and without
the scheme is compared as a consistency check; on this dilute system it cannot tell the
two readings apart.
"""
import math

import numpy as np

from oracle import oracle as orc
from paper_2307_11447_gb300 import analysis as an
from paper_2307_11447_gb300 import workloads as wl


def _params(L, edge, **extra):
    cfg = dict(wl.LJ_PHYSICS)
    cfg.update(L=L, n_f=10, v_ex=edge**3, seed=21, replica=0)
    cfg.update(extra)
    return orc.make_params(cfg)


def test_excluded_cube_geometry():
    L, edge = 10.0, 2.0
    p = _params(L, edge)
    c = np.array([5.0, 5.0, 5.0])
    assert orc.in_excluded_volume(p, c, c + [0.999, -0.999, 0.5])
    assert not orc.in_excluded_volume(p, c, c + [1.001, 0.0, 0.0])
    assert not orc.in_excluded_volume(p, c, c + [0.0, 0.0, -1.001])
    assert not orc.in_excluded_volume(p, c, c + [0.9, 0.9, 1.2])
    # minimum image across the periodic boundary
    assert orc.in_excluded_volume(p, [0.2, 5.0, 5.0], [9.5, 5.0, 5.5])
    assert not orc.in_excluded_volume(p, [0.2, 5.0, 5.0], [8.9, 5.0, 5.0])
    # off: no cube at all
    assert not orc.in_excluded_volume(_params(L, 0.0), c, c)
    rng = np.random.default_rng(1)
    xc = rng.random((20000, 3)) * L
    xa = rng.random((20000, 3)) * L
    inside = np.array([orc.in_excluded_volume(p, a, b) for a, b in zip(xc, xa)])
    assert np.array_equal(inside, [orc.in_excluded_volume(p, b, a) for a, b in zip(xc, xa)])
    # it covers V_ex / V of the box (0.008 here; 4 standard errors)
    frac = edge**3 / L**3
    assert abs(inside.mean() - frac) < 4 * math.sqrt(frac * (1 - frac) / inside.size)


def test_instant_trials_skip_nemd_and_exchange_the_potential_energy():
    cfg = wl.lj_config(40, 0.2, 20)
    L = cfg["L"]
    cfg.update(seed=4, replica=3, beta_mu=-2.0, v_ex=(0.5 * L) ** 3)
    p = orc.make_params(cfg)
    st = orc.State(p, wl.lj_positions(20, L, 5), None, 20, 40)
    orc.init_velocities(p, st)
    orc.md(p, st, 100)
    kinds = {0: 0, 1: 0}
    checked = 0
    for _ in range(160):
        n = 2 * st.n_pairs
        x0 = st.positions()[:n].copy()
        r = orc.trial(p, st)
        if r["status"] != 0:
            continue
        kinds[int(r["instant"])] += 1
        if r["move"] == 0:
            ci, ai = 2 * r["cation"], 2 * r["anion"] + 1
            assert bool(r["instant"]) == orc.in_excluded_volume(p, x0[ci], x0[ai])
            if r["instant"]:
                # the (N-1)-pair end state: the last pair moves into the freed slots, which
                # keeps the species of every index (cation even, anion odd)
                x_end = x0.copy()
                x_end[ci], x_end[ai] = x0[n - 2], x0[n - 1]
                dU = orc.energy_forces(p, x_end[: n - 2])[0] - orc.energy_forces(p, x0)[0]
                assert r["w_prot"] == 0.0
                assert abs(r["dH"] - dU) <= 1e-9 * (1.0 + abs(dU))
                checked += 1
        elif r["accepted"]:
            x1 = st.positions()[: n + 2]
            assert bool(r["instant"]) == orc.in_excluded_volume(p, x1[n], x1[n + 1])
            if r["instant"]:
                dU = orc.energy_forces(p, x1)[0] - orc.energy_forces(p, x0)[0]
                assert r["w_prot"] == 0.0
                assert abs(r["dH"] - dU) <= 1e-9 * (1.0 + abs(dU))
                checked += 1
        if not r["instant"]:
            assert r["w_prot"] != 0.0
    assert kinds[0] >= 20 and kinds[1] >= 5 and checked >= 5, (kinds, checked)


def _mean_n(v_ex, n_trials):
    L = 8.0
    cfg = dict(wl.LJ_PHYSICS)
    cfg.update(L=L, n_f=10, beta_mu=-9.0, v_ex=v_ex, seed=8, replica=1)
    p = orc.make_params(cfg)
    x = wl.lj_positions(8, L, 3)
    st = orc.State(p, np.concatenate([x, np.zeros((2 * 32 - x.shape[0], 3))]), None, 4, 32)
    orc.init_velocities(p, st)
    recs = orc.run_cycles(p, st, n_trials, 5)
    n = recs["n_after"][1000:]
    return an.block_stats(n, 40), recs


def test_stationary_n_is_unchanged_by_early_rejection():
    (m0, se0), _ = _mean_n(0.0, 24000)
    (m1, se1), recs = _mean_n((0.55 * 8.0) ** 3, 24000)
    frac_instant = recs["instant"][recs["status"] == 0].mean()
    print(f"<N> without {m0:.3f} +- {se0:.3f}, with early rejection {m1:.3f} +- {se1:.3f} "
          f"({100 * frac_instant:.1f}% instantaneous)")
    assert frac_instant > 0.1
    assert abs(m1 - m0) < 4 * math.hypot(se0, se1)
