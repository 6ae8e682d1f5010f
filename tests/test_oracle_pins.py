"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible mistake in the oracle (a dropped shift, a wrong
sign, a transposed index, a wrong power of (N+1)/V, a wrong altitude schedule) fails it.
None of these tests needs a GPU.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

from oracle import oracle as orc
from paper_2307_11447_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def lj_params(**kw):
    cfg = dict(wl.LJ_PHYSICS)
    cfg.update(L=10.0, n_f=20, beta_mu=0.0)
    cfg.update(kw)
    return orc.make_params(cfg), cfg


# ---------------------------------------------------------------------------------------
# Philox4x64-10: known answers from numpy's independent implementation
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("key", [(0, 0), (1, 2), (123456789, 987654321), (2**64 - 1, 7)])
@pytest.mark.parametrize("ctr", [(0, 0, 0, 0), (5, 0, 0, 0), (2**64 - 1, 0, 3, 0), (9, 8, 7, 6)])
def test_philox_matches_numpy(key, ctr):
    ref = np.random.Philox(key=np.array(key, np.uint64), counter=np.array(ctr, np.uint64)).random_raw(4)
    # numpy increments the 256-bit counter before producing a block
    c = sum(int(ctr[i]) << (64 * i) for i in range(4)) + 1
    c1 = [(c >> (64 * i)) & (2**64 - 1) for i in range(4)]
    assert np.array_equal(orc.philox(c1, key), ref)


# ---------------------------------------------------------------------------------------
# Pair potential (Eqs. 9-11, 19-20)
# ---------------------------------------------------------------------------------------
def _erf_table():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "erfc_table.txt")) if l.strip() and not l.startswith("#")]
    return {float(a): float(b) for a, b in rows}


def test_coulomb_against_printed_erf_table():
    tab = _erf_table()
    p, cfg = lj_params(eps=[0.0, 0.0])
    a, rc, K = cfg["alpha"], cfg["rc_coul"], cfg["kcoul"]
    shift = (1.0 - tab[1.20]) / rc  # alpha * rc = 1.2
    for x in (0.30, 0.50, 1.00):
        r = x / a
        u, _ = orc.pair(p, 0, 1, r)
        assert u == pytest.approx(-K * ((1.0 - tab[x]) / r - shift), rel=1e-9, abs=1e-11)
        u, _ = orc.pair(p, 0, 0, r)  # like charges repel
        assert u == pytest.approx(+K * ((1.0 - tab[x]) / r - shift), rel=1e-9, abs=1e-11)


def test_lj_minimum_and_shift():
    p, cfg = lj_params(q=[0.0, 0.0])
    rc = cfg["rc_lj"]
    shift = 4.0 * (rc**-12 - rc**-6)
    rmin = 2.0 ** (1.0 / 6.0)
    u, du = orc.pair(p, 0, 1, rmin)
    assert du == pytest.approx(0.0, abs=1e-12)
    assert u == pytest.approx(-1.0 - shift, rel=1e-12)
    u, _ = orc.pair(p, 0, 1, 1.0)
    assert u == pytest.approx(-shift, abs=1e-12)
    u, du = orc.pair(p, 0, 1, rc * (1 - 1e-12))
    assert abs(u) < 1e-9  # continuous at the cut-off
    u, du = orc.pair(p, 0, 1, rc * (1 + 1e-9))
    assert u == 0.0 and du == 0.0


def test_lorentz_berthelot_mixing():
    cfg = dict(wl.AQ_PHYSICS)
    cfg.update(L=40.0, n_f=10, q=[0.0, 0.0, 0.0, 0.0])
    p = orc.make_params(cfg)
    s = 0.5 * (2.16 + 3.166)
    e = math.sqrt(1.475 * 0.650)
    rmin = 2 ** (1 / 6) * s
    shift = 4 * e * ((s / 10.0) ** 12 - (s / 10.0) ** 6)
    u, du = orc.pair(p, 0, 2, rmin)
    assert du == pytest.approx(0.0, abs=1e-12)
    assert u == pytest.approx(-e - shift, rel=1e-12)
    u, du = orc.pair(p, 2, 3, 2.0)  # H carries no LJ
    assert u == 0.0 and du == 0.0


def test_dudr_matches_finite_difference():
    p, _ = lj_params(kappa_sr=0.7)
    for ti, tj in ((0, 1), (0, 0), (1, 1)):
        for r in (0.85, 1.1, 2.0, 3.3):
            for g in (1.0, 0.3):
                h = 1e-6
                up, _ = orc.pair(p, ti, tj, r + h, g)
                um, _ = orc.pair(p, ti, tj, r - h, g)
                _, du = orc.pair(p, ti, tj, r, g)
                assert du == pytest.approx((up - um) / (2 * h), rel=1e-6, abs=1e-7)


def _random_config(n, L, seed, min_dist=0.9):
    return wl._pick_far(np.random.default_rng(seed), L, [], n, min_dist)


def test_forces_are_minus_gradient_with_flyers():
    """F = -grad U by central differences (h = 1e-5) in a 4D configuration with two flyers
    at nonzero altitude and short-range screening switched on."""
    p, cfg = lj_params(L=7.0, kappa_sr=0.8)
    x = _random_config(16, 7.0, 3)
    w = np.zeros(16)
    fly = np.zeros(16, np.uint8)
    fly[[4, 9]] = 1
    w[[4, 9]] = 0.7
    U, F = orc.energy_forces(p, x, w, fly)
    h = 1e-5
    for i in range(16):
        for c in range(3):
            xp = x.copy(); xp[i, c] += h
            xm = x.copy(); xm[i, c] -= h
            Up, _ = orc.energy_forces(p, xp, w, fly)
            Um, _ = orc.energy_forces(p, xm, w, fly)
            assert F[i, c] == pytest.approx(-(Up - Um) / (2 * h), rel=1e-5, abs=1e-6)
    assert np.abs(F.sum(0)).max() < 1e-10  # Newton's third law in 3D


def test_four_d_distance_single_pair():
    """A flyer at altitude w straight above a 3D particle sees the 3D pair energy at r = w."""
    p, _ = lj_params(L=12.0)
    for w0 in (0.95, 1.5, 2.2, 3.9):
        x = np.array([[3.0, 3.0, 3.0], [3.0, 3.0, 3.0]])
        w = np.array([w0, 0.0])
        fly = np.array([1, 0], np.uint8)
        U, F = orc.energy_forces(p, x, w, fly)
        u3, _ = orc.pair(p, 0, 1, w0)
        assert U == pytest.approx(u3, rel=1e-13)
        assert np.abs(F).max() == 0.0  # no 3D component when the 3D separation is zero


def test_screening_only_between_flyer_and_non_flyer():
    p0, _ = lj_params(L=12.0, kappa_sr=0.0)
    p1, _ = lj_params(L=12.0, kappa_sr=1.3)
    x = np.array([[1.0, 1.0, 1.0], [2.2, 1.0, 1.0], [1.0, 2.4, 1.0]])
    fly = np.array([1, 1, 0], np.uint8)
    w = np.array([0.5, 0.5, 0.0])
    U0, _ = orc.energy_forces(p0, x, w, fly)
    U1, _ = orc.energy_forces(p1, x, w, fly)
    # the flyer-flyer pair (Delta w = 0) keeps its full 3D interaction; flyer-solvent pairs
    # have their Coulomb part multiplied by exp(-kappa w)
    u01, _ = orc.pair(p0, 0, 1, 1.2)
    r02 = math.sqrt(1.4**2 + 0.25)
    r12 = math.sqrt(1.2**2 + 1.4**2 + 0.25)
    uc02 = orc.pair(orc.make_params(dict(wl.LJ_PHYSICS, L=12.0, n_f=1, eps=[0, 0])), 0, 0, r02)[0]
    uc12 = orc.pair(orc.make_params(dict(wl.LJ_PHYSICS, L=12.0, n_f=1, eps=[0, 0])), 1, 0, r12)[0]
    g = math.exp(-1.3 * 0.5)
    assert U1 - U0 == pytest.approx((g - 1.0) * (uc02 + uc12), rel=1e-12)
    assert U0 == pytest.approx(u01 + orc.pair(p0, 0, 0, r02)[0] + orc.pair(p0, 1, 0, r12)[0], rel=1e-12)


def test_three_d_recovered_when_all_w_zero():
    p, _ = lj_params(L=8.0, kappa_sr=0.0)
    x = _random_config(30, 8.0, 5)
    fly = np.zeros(30, np.uint8)
    fly[[3, 4]] = 1
    U3, F3 = orc.energy_forces(p, x)
    U4, F4 = orc.energy_forces(p, x, np.zeros(30), fly)
    assert U4 == U3 and np.array_equal(F3, F4)


def test_minimum_image_across_the_boundary():
    p, _ = lj_params(L=10.0)
    x = np.array([[0.2, 5.0, 5.0], [9.5, 5.0, 5.0]])
    U, F = orc.energy_forces(p, x)
    u, du = orc.pair(p, 0, 1, 0.7)
    assert U == pytest.approx(u, rel=1e-12)
    assert F[0, 0] == pytest.approx(-du, rel=1e-12)  # pushed towards +x (away from the image at -0.5)


def test_cell_list_equals_brute_force():
    cfg = dict(wl.LJ_PHYSICS, L=14.0, n_f=1)
    x = _random_config(400, 14.0, 11)
    pb = orc.make_params(cfg, use_cells=0)
    pc = orc.make_params(cfg, use_cells=1)
    Ub, Fb = orc.energy_forces(pb, x)
    Uc, Fc = orc.energy_forces(pc, x)
    assert Uc == pytest.approx(Ub, rel=1e-12)
    assert np.abs(Fc - Fb).max() < 1e-10 * max(1.0, np.abs(Fb).max())


def test_neighbor_criterion_against_float_distances():
    L = 9.0
    x = np.random.default_rng(2).random((300, 3)) * L
    i, j = orc.neighbor_pairs(x, L, 2.8)
    got = set(zip(i.tolist(), j.tolist()))
    d = x[:, None, :] - x[None, :, :]
    d -= L * np.round(d / L)
    r = np.sqrt((d * d).sum(-1))
    for a in range(300):
        for b in range(a + 1, 300):
            if r[a, b] < 2.8 - 1e-7:
                assert (a, b) in got
            elif r[a, b] > 2.8 + 1e-7:
                assert (a, b) not in got


# ---------------------------------------------------------------------------------------
# Protocol (Eq. 2, Eqs. S6-S7)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("sched,n", [("linear", 1.0), ("wv", 2.0), ("wx", 3.0)])
def test_schedules_boundary_values_and_time_reversal(sched, n):
    p, cfg = lj_params(n_f=40, schedule=sched, sched_n=n)
    wmax = cfg["w_max"]
    assert orc.altitude(p, True, 0) == pytest.approx(wmax)
    assert orc.altitude(p, True, 40) == pytest.approx(0.0, abs=1e-15)
    assert orc.altitude(p, False, 0) == pytest.approx(0.0, abs=1e-15)
    assert orc.altitude(p, False, 40) == pytest.approx(wmax)
    for k in range(41):
        # deletion is the time reverse of insertion
        assert orc.altitude(p, False, k) == pytest.approx(orc.altitude(p, True, 40 - k), abs=1e-14)
    if sched == "linear":  # constant vertical velocity (Eq. 2)
        dw = np.diff([orc.altitude(p, True, k) for k in range(41)])
        assert np.allclose(dw, -wmax / 40)


# ---------------------------------------------------------------------------------------
# Integrator
# ---------------------------------------------------------------------------------------
def _lj_state(n_pairs, L, seed, **kw):
    p, cfg = lj_params(L=L, **kw)
    x = _random_config(2 * n_pairs, L, seed, 1.0)
    st = orc.State(p, x, None, n_pairs, n_pairs + 2)
    orc.init_velocities(p, st)
    return p, st


def test_nve_energy_drift_scales_as_dt_squared():
    p, st0 = _lj_state(20, 6.0, 1, dt=0.002, tau_t=0.1)
    orc.md(p, st0, 300)  # relax the random start
    flucts = []
    for dt, n in ((0.004, 200), (0.002, 400)):
        p2, _ = lj_params(L=6.0, dt=dt)
        st = orc.State(p2, st0.positions(), st0.velocities(), 20, 22)
        _, tr = orc.nve(p2, st, n, trace=True)
        flucts.append(tr.std())
    ratio = flucts[0] / flucts[1]
    assert 3.0 < ratio < 5.3, ratio


@pytest.mark.parametrize("fw", [0.0, 1.0])
def test_nemd_is_time_reversible(fw):
    """Insertion schedule forward, negate momenta, deletion schedule: back to the start
    (also with a different w_max for the anion, fw > 0)."""
    p, st = _lj_state(12, 6.0, 4, dt=0.003, n_f=60, tau_t=0.1, kappa_sr=0.5, fw=fw)
    orc.md(p, st, 200)
    x0, v0 = st.positions(), st.velocities()
    fly = [4, 7]
    orc.nemd_path(p, st, fly, True)
    st.v[: st.n_atoms] *= -1
    orc.nemd_path(p, st, fly, False)
    st.v[: st.n_atoms] *= -1
    dx = st.positions() - x0
    dx -= 6.0 * np.round(dx / 6.0)
    assert np.abs(dx).max() < 1e-10
    assert np.abs(st.velocities() - v0).max() < 1e-10


def test_shadow_work_vanishes_as_dt_squared():
    """Delta H - W_protocol is the integration error; halving dt divides it by ~4."""
    p, st0 = _lj_state(12, 6.0, 8, dt=0.002, tau_t=0.1)
    orc.md(p, st0, 200)
    fly = [2, 5]
    out = []
    for dt, nf in ((0.004, 50), (0.002, 100), (0.001, 200)):
        p2, _ = lj_params(L=6.0, dt=dt, n_f=nf)
        st = orc.State(p2, st0.positions(), st0.velocities(), 12, 14)
        fl = np.zeros(24, np.uint8); fl[fly] = 1
        w = np.zeros(24); w[fly] = orc.altitude(p2, True, 0)
        U0, _ = orc.energy_forces(p2, st.positions(), w, fl)
        K0 = orc.kinetic(p2, st.velocities(), fl)
        wprot, U1 = orc.nemd_path(p2, st, fly, True)
        K1 = orc.kinetic(p2, st.velocities(), fl)
        out.append(abs((U1 + K1) - (U0 + K0) - wprot))
    assert out[0] / out[1] == pytest.approx(4.0, rel=0.35)
    assert out[1] / out[2] == pytest.approx(4.0, rel=0.35)


def test_rattle_keeps_water_rigid():
    cfg = dict(wl.AQ_PHYSICS)
    cfg.update(L=12.0, n_f=10, n_water=4, dt=1.0)
    p = orc.make_params(cfg)
    rng = np.random.default_rng(1)
    x = []
    for m in range(4):
        o = np.array([3.0 + 6 * (m % 2), 3.0 + 6 * (m // 2), 6.0])
        th = math.radians(109.47)
        x += [o, o + [1.0, 0, 0], o + [math.cos(th), math.sin(th), 0]]
    x = np.array(x) + rng.normal(scale=0.0, size=(12, 3))
    st = orc.State(p, x, None, 0, 1)
    orc.init_velocities(p, st)
    orc.md(p, st, 50)
    xs = st.positions()
    for m in range(4):
        o, h1, h2 = xs[3 * m: 3 * m + 3]
        dist = lambda a, b: np.linalg.norm((a - b) - 12.0 * np.round((a - b) / 12.0))
        assert dist(o, h1) == pytest.approx(1.0, abs=1e-7)
        assert dist(o, h2) == pytest.approx(1.0, abs=1e-7)
        assert dist(h1, h2) == pytest.approx(cfg["d_hh"], abs=1e-7)


@pytest.mark.parametrize("fw", [0.0, 0.5, 1.0])
def test_species_wmax_two_flyer_protocol_work_closed_form(fw):
    """SI, different w_max per species: the anion starts at w_max + 0.5 (sig_c + sig_a) fw
    and both flyers reach w = 0 together.  With only the two (frozen) flyers in the box the
    protocol work telescopes to u(r, 0) - u(r, dw0), dw0 = 0.5 (sig_c + sig_a) fw: the
    flyer-flyer term is the only one, unscreened (both fly), and its altitude gap closes
    linearly."""
    cfg = dict(wl.LJ_PHYSICS)
    cfg.update(L=12.0, n_f=40, fw=fw, kappa_sr=0.7)
    p = orc.make_params(cfg)
    x = np.array([[3.0, 3.0, 3.0], [4.4, 3.3, 2.8]])
    st = orc.State(p, x, None, 1, 1)
    w, _ = orc.nemd_path(p, st, [0, 1], True)
    r = float(np.linalg.norm(x[1] - x[0]))
    dw0 = 0.5 * (cfg["sig"][0] + cfg["sig"][1]) * fw
    u0, _ = orc.pair(p, 0, 1, r)
    u1, _ = orc.pair(p, 0, 1, math.sqrt(r * r + dw0 * dw0))
    assert w == pytest.approx(u0 - u1, abs=1e-12)
