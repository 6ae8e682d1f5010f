"""Thermal velocities in the oracle: the CSVR thermostat of equilibrium MD (Bussi, Donadio
and Parrinello 2007; the paper leaves the NVT thermostat open, the reading taken is CSVR)
and the Maxwell-Boltzmann draws of the initial velocities and of inserted ions (Sec. II.A).

Pin: without forces the thermostat alone must sample the canonical kinetic energy, K ~
Gamma(dof/2, k_B T) with dof = 3 n (no constraints): mean dof/2 kT, variance dof/2 (kT)^2,
and the whole distribution (Kolmogorov-Smirnov on samples thinned well beyond the
thermostat's relaxation time).  A chi-square draw with the wrong number of degrees of
freedom moves the mean by kT/2; a wrong sign or factor in the stochastic term changes the
variance.
"""
import math

import numpy as np
from scipy import stats

from oracle import oracle as orc
from paper_2307_11447_gb300 import analysis as an
from paper_2307_11447_gb300 import workloads as wl


def test_csvr_samples_the_canonical_kinetic_energy():
    # few degrees of freedom: a chi-square draw off by one shifts <K> by kT/2 whatever dof
    # is, while the noise of <K> grows with dof
    n_pairs = 2
    cfg = dict(wl.LJ_PHYSICS)
    # free particles: no pair interactions, so only the thermostat changes K
    cfg.update(L=20.0, n_f=1, q=[0.0, 0.0], eps=[0.0, 0.0], tau_t=0.05, beta=1.25, seed=3, replica=7)
    p = orc.make_params(cfg)
    x = np.random.default_rng(0).random((2 * n_pairs, 3)) * cfg["L"]
    st = orc.State(p, x, None, n_pairs, n_pairs)
    orc.init_velocities(p, st)
    dof = 3 * 2 * n_pairs
    kT = 1.0 / cfg["beta"]
    orc.md(p, st, 200)
    K = np.empty(100000)
    for k in range(K.size):
        orc.md(p, st, 1)
        K[k] = orc.kinetic(p, st.velocities())
    mean, se = an.block_stats(K, 40)
    print(f"<K> {mean:.4f} +- {se:.4f} (exact {dof / 2 * kT:.4f}); Var K {K.var():.4f} "
          f"(exact {dof / 2 * kT**2:.4f})")
    assert abs(mean - dof / 2 * kT) < 4 * se
    assert abs(K.var() / (dof / 2 * kT**2) - 1.0) < 0.1
    # relaxation time tau_t = 10 steps: every 100th sample is independent
    thin = K[::100][:600]
    ks = stats.kstest(thin, stats.gamma(a=dof / 2, scale=kT).cdf)
    assert ks.pvalue > 1e-3, ks
    # the thermostat is reproducible: the same seed and counters give the same K
    st2 = orc.State(p, x, None, n_pairs, n_pairs)
    orc.init_velocities(p, st2)
    orc.md(p, st2, 200 + K.size)
    assert math.isclose(orc.kinetic(p, st2.velocities()), K[-1], rel_tol=1e-12)


def test_initial_velocities_are_maxwell_boltzmann_per_species():
    """orc_init_velocities (Sec. II.A): every Cartesian component of an atom of mass m is
    N(0, kT/m); checked per species with unequal masses"""
    n_pairs = 2000
    cfg = dict(wl.LJ_PHYSICS)
    cfg.update(L=60.0, n_f=1, mass=[1.0, 3.5], beta=0.8, seed=12, replica=1)
    p = orc.make_params(cfg)
    x = np.random.default_rng(1).random((2 * n_pairs, 3)) * cfg["L"]
    st = orc.State(p, x, None, n_pairs, n_pairs)
    orc.init_velocities(p, st)
    v = st.velocities()
    for t, m in enumerate(cfg["mass"]):
        z = (v[t::2] * math.sqrt(m * cfg["beta"])).ravel()
        ks = stats.kstest(z, stats.norm.cdf)
        assert ks.pvalue > 1e-3, (t, ks)
        assert abs(z.mean()) < 4 / math.sqrt(z.size)


def test_inserted_ions_carry_maxwell_boltzmann_velocities():
    """the flyers' velocities drawn at an insertion (trial blocks 3-4) and kept on
    acceptance: per species N(0, kT/m) over many accepted insertions of an ideal pair gas"""
    cfg = dict(wl.LJ_PHYSICS)
    cfg.update(L=10.0, n_f=1, q=[0.0, 0.0], eps=[0.0, 0.0], mass=[2.0, 0.5], beta=1.0,
               beta_mu=math.log(1e4 / 1e6), seed=6, replica=2)
    p = orc.make_params(cfg)
    cap = 400
    st = orc.State(p, np.random.default_rng(2).random((2 * cap, 3)) * cfg["L"], None, 0, cap)
    orc.init_velocities(p, st)
    vc, va = [], []
    for _ in range(3000):
        n0 = st.n_pairs
        r = orc.trial(p, st)
        if r["move"] == 1 and r["accepted"]:
            v = st.velocities()
            vc.append(v[2 * n0].copy())
            va.append(v[2 * n0 + 1].copy())
    assert len(vc) > 300
    for vs, m in ((vc, cfg["mass"][0]), (va, cfg["mass"][1])):
        z = (np.array(vs) * math.sqrt(m * cfg["beta"])).ravel()
        ks = stats.kstest(z, stats.norm.cdf)
        assert ks.pvalue > 1e-3, (m, ks)


def test_rigid_water_velocities_are_equipartitioned():
    """orc_init_velocities on rigid waters: Maxwell-Boltzmann draws with the bond-parallel
    components removed (the RATTLE projection, mass-weighted) leave each molecule with
    3/2 kT of translational and 3/2 kT of rotational kinetic energy on average, and the
    constraints satisfied"""
    cfg = dict(wl.AQ_PHYSICS)
    nw, L = 400, 30.0
    x = wl.aqueous_positions(nw, 0, L, 5)
    kT = 1.0 / cfg["beta"]
    m = np.array(cfg["mass"])[[2, 3, 3]]
    kt, kr = [], []
    for seed in range(20):
        c = dict(cfg)
        c.update(L=L, n_water=nw, n_f=1, seed=seed, replica=0)
        p = orc.make_params(c)
        st = orc.State(p, x, None, 0, 1)
        orc.init_velocities(p, st)
        v = st.velocities().reshape(nw, 3, 3)
        M = m.sum()
        V = (v * m[None, :, None]).sum(1) / M
        k_t = 0.5 * M * (V**2).sum(1) * cfg["mvv2e"]
        k = 0.5 * (m[None, :, None] * v**2).sum((1, 2)) * cfg["mvv2e"]
        kt.append(k_t)
        kr.append(k - k_t)
        # rigid: every bond's relative velocity is perpendicular to the bond
        xm = x.reshape(nw, 3, 3)
        for a, b in ((0, 1), (0, 2), (1, 2)):
            d = xm[:, b] - xm[:, a]
            dv = v[:, b] - v[:, a]
            assert np.abs((d * dv).sum(1)).max() < 1e-9 * np.abs(dv).max()
    kt, kr = np.concatenate(kt) / kT, np.concatenate(kr) / kT
    for k in (kt, kr):
        assert abs(k.mean() - 1.5) < 4 * math.sqrt(1.5 / k.size), (kt.mean(), kr.mean())
