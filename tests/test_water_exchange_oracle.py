"""Pins of the oracle's rigid-water exchange (Sec. II.A: the exchange rule with one flying
particle, V/(N+1) once; Sec. II.C: a flying rigid water with Maxwell-Boltzmann velocities
drawn in its molecular frame; Sec. II.B.1 read for a molecule: the flyer is frozen in 3D,
position and orientation).

* Ideal gas of rigid waters (every interaction off): P(N) is Poisson with <N> = zV and
  Var N/<N> = 1 (z = e^{beta mu}); the pair factor (squared) gives a Bessel law instead.
* An inserted water: both O-H bonds and the H-H distance of the model, velocities of a
  rigid body (no relative velocity along any bond), centre-of-mass velocity N(0, kT/M) per
  axis, body-frame angular velocity N(0, kT/I_k) about each principal axis (moments from
  the geometry by an eigen-decomposition here), a uniform orientation (the symmetry axis
  and the H-H axis uniform on the sphere) and a uniform position.
* Two interacting waters (capacity two, LJ sites on O and H, no charges): P(1)/P(0) = zV
  and P(2)/P(1) = (z/2)(V + B) with B = int d^3r <e^{-beta u} - 1> over the separation of
  the O atoms and both orientations, estimated by Monte Carlo here from the pair potential
  of Eq. 19 written out in numpy.
* Layout: a rejection restores the state; an accepted insertion adds the water after the
  last water and moves the ions up by three atoms; an accepted deletion moves the last
  water into the deleted slot and the ions down by three.
"""
import math
import multiprocessing as mp
import os

import numpy as np
import pytest
from scipy import special, stats

from oracle import oracle as orc
from paper_2307_11447_gb300 import workloads as wl


def _water_cfg(L, **kw):
    cfg = wl.aq_config(0, 0, L, 2)
    cfg.update(exchange="water", tau_t=0.0, rc_lj=min(4.5, 0.45 * L), rc_coul=min(4.5, 0.45 * L))
    cfg.update(kw)
    return cfg


def _ideal(L, **kw):
    return _water_cfg(L, q=[0.0] * 4, eps=[0.0] * 4, **kw)


def _chain(job):
    cfg, n0, cap, cycles, seed, v_scale = job
    p = orc.make_params(dict(cfg, seed=seed, replica=0, n_water=n0))
    x = wl.aqueous_positions(n0, 0, cfg["L"], seed) if n0 else np.zeros((0, 3))
    rng = np.random.default_rng(seed)
    st = orc.State(p, x, v_scale * rng.normal(size=(3 * n0, 3)) if n0 else None, 0, 0, cap_water=cap)
    if n0 and v_scale:
        orc.init_velocities(p, st)
    recs = orc.run_cycles(p, st, cycles, 0)
    return recs["n_after"], recs["accepted"], recs["move"]


def _run(cfg, n0, cap, cycles, chains, seed0, v_scale=0.0):
    jobs = [(cfg, n0, cap, cycles, seed0 + k, v_scale) for k in range(chains)]
    with mp.get_context("spawn").Pool(min(chains, os.cpu_count() or 1)) as pool:
        return pool.map(_chain, jobs)


def test_ideal_water_gas_is_poisson():
    L, lam = 10.0, 3.0
    cfg = _ideal(L, beta_mu=math.log(lam / L**3))
    res = _run(cfg, 3, 24, 30000, 8, 300)
    n = np.concatenate([r[0][1000:] for r in res]).astype(float)
    means = np.array([r[0][1000:].mean() for r in res])
    se = means.std(ddof=1) / math.sqrt(len(means))
    print(f"\n<N> {n.mean():.4f} +- {se:.4f} (zV {lam}), Var/<N> {n.var() / n.mean():.4f}")
    assert abs(n.mean() - lam) < 4 * se + 1e-3, (n.mean(), lam, se)
    assert abs(n.var() / n.mean() - 1.0) < 0.05, n.var() / n.mean()
    k = np.arange(15)
    pk = np.exp(k * math.log(lam) - lam - special.gammaln(k + 1))
    hist = np.bincount(n.astype(int), minlength=25)[:15] / n.size
    assert np.abs(hist - pk).max() < 0.01


def _inserted_waters(cfg, n_trials):
    """positions and velocities of the water inserted by each insertion trial from an
    empty box (z large enough that every insertion is accepted)"""
    p = orc.make_params(dict(cfg, seed=11, replica=0, n_water=0))
    st = orc.State(p, np.zeros((0, 3)), None, 0, 0, cap_water=1)
    xs, vs = [], []
    for k in range(n_trials):
        st.s.n_water = 0
        st.s.trial_ctr = k
        r = orc.trial(p, st)
        if r["move"] == 1:
            assert r["accepted"] == 1 and r["status"] == 0 and st.n_water == 1
            xs.append(st.positions()[:3])
            vs.append(st.velocities()[:3])
    return np.array(xs), np.array(vs)


def test_inserted_water_geometry_orientation_and_velocities():
    L = 10.0
    cfg = _ideal(L, beta_mu=math.log(1e6))
    x, v = _inserted_waters(cfg, 6000)
    assert len(x) > 2500
    d_oh, d_hh = cfg["d_oh"], cfg["d_hh"]
    mO, mH = cfg["mass"][2], cfg["mass"][3]
    kT = 1.0 / (cfg["beta"] * cfg["mvv2e"])

    def mi(d):
        return d - L * np.round(d / L)

    r1, r2 = mi(x[:, 1] - x[:, 0]), mi(x[:, 2] - x[:, 0])
    # geometry of the model to the resolution of the 32-bit grid
    assert np.abs(np.linalg.norm(r1, axis=1) - d_oh).max() < 1e-7
    assert np.abs(np.linalg.norm(r2, axis=1) - d_oh).max() < 1e-7
    assert np.abs(np.linalg.norm(r1 - r2, axis=1) - d_hh).max() < 1e-7
    # velocities of a rigid body: no relative velocity along any bond
    for a, b, rab in ((1, 0, r1), (2, 0, r2), (1, 2, r1 - r2)):
        along = np.einsum("ij,ij->i", v[:, a] - v[:, b], rab)
        assert np.abs(along).max() < 1e-9
    # centre of mass velocity
    M = mO + 2 * mH
    com_off = (mH * r1 + mH * r2) / M  # centre of mass relative to the O
    vcom = (mO * v[:, 0] + mH * v[:, 1] + mH * v[:, 2]) / M
    for d in range(3):
        assert stats.kstest(vcom[:, d] / math.sqrt(kT / M), "norm").pvalue > 1e-3
    # body axes: y along the symmetry axis, x along H1 - H2, z = x cross y
    ey = com_off / np.linalg.norm(com_off, axis=1, keepdims=True)
    ex = (r1 - r2) / np.linalg.norm(r1 - r2, axis=1, keepdims=True)
    ez = np.cross(ex, ey)
    # principal moments of the model about its centre of mass (eigen-decomposition)
    sh = 0.5 * d_hh / d_oh
    body = np.array([[0.0, 0.0, 0.0], [d_oh * sh, d_oh * math.sqrt(1 - sh * sh), 0.0],
                     [-d_oh * sh, d_oh * math.sqrt(1 - sh * sh), 0.0]])
    m = np.array([mO, mH, mH])
    rb = body - (m[:, None] * body).sum(0) / m.sum()
    I = sum(mk * (np.dot(r, r) * np.eye(3) - np.outer(r, r)) for mk, r in zip(m, rb))
    evals, evecs = np.linalg.eigh(I)
    assert np.allclose(np.abs(evecs), np.eye(3)[:, np.argsort(np.diag(I))], atol=1e-12)  # body axes are principal
    Ib = np.diag(I)
    # angular velocity from the atoms' velocities relative to the centre of mass:
    # u_a = omega x s_a for the three atoms, solved by least squares
    s = np.stack([-com_off, r1 - com_off, r2 - com_off], 1)
    u = v - vcom[:, None, :]
    omegas = []
    for k in range(len(x)):
        A = np.concatenate([np.array([[0, s[k, a, 2], -s[k, a, 1]], [-s[k, a, 2], 0, s[k, a, 0]],
                                      [s[k, a, 1], -s[k, a, 0], 0]]) for a in range(3)])
        w, *_ = np.linalg.lstsq(A, u[k].reshape(-1), rcond=None)
        omegas.append(w)
    om = np.array(omegas)
    resid = np.abs(np.cross(om[:, None, :], s) - u).max()
    assert resid < 1e-9
    for e, Ik in ((ex, Ib[0]), (ey, Ib[1]), (ez, Ib[2])):
        wk = np.einsum("ij,ij->i", om, e)
        assert stats.kstest(wk / math.sqrt(kT / Ik), "norm").pvalue > 1e-3
    # equipartition: 3/2 kT translational and 3/2 kT rotational on average
    ktr = 0.5 * M * (vcom**2).sum(1) / kT
    krot = 0.5 * sum(Ik * np.einsum("ij,ij->i", om, e) ** 2 for e, Ik in ((ex, Ib[0]), (ey, Ib[1]), (ez, Ib[2]))) / kT
    assert stats.kstest(ktr, stats.gamma(1.5).cdf).pvalue > 1e-3
    assert stats.kstest(krot, stats.gamma(1.5).cdf).pvalue > 1e-3
    # uniform orientation and position
    for e in (ey, ex, ez):
        for d in range(3):
            assert stats.kstest(e[:, d], stats.uniform(-1, 2).cdf).pvalue > 1e-3
    for d in range(3):
        assert stats.kstest(x[:, 0, d] / L, "uniform").pvalue > 1e-3


def _lj_numpy(cfg, ta, tb, r):
    """truncated-shifted LJ of Eq. 19 with Lorentz-Berthelot mixing"""
    sig = 0.5 * (cfg["sig"][ta] + cfg["sig"][tb])
    eps = math.sqrt(cfg["eps"][ta] * cfg["eps"][tb])
    rc = cfg["rc_lj"]
    if eps == 0.0:
        return np.zeros_like(r)
    sr6 = (sig / r) ** 6
    src6 = (sig / rc) ** 6
    u = 4 * eps * (sr6 * sr6 - sr6) - 4 * eps * (src6 * src6 - src6)
    return np.where(r < rc, u, 0.0)


def _random_rotations(rng, n):
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)


def _second_virial(cfg, n=2_000_000, seed=5):
    """B = int d^3r <e^{-beta u} - 1>: O-O separations uniform in the ball beyond which no
    atom pair is inside the cut-off, both orientations uniform"""
    rng = np.random.default_rng(seed)
    d_oh, d_hh = cfg["d_oh"], cfg["d_hh"]
    sh = 0.5 * d_hh / d_oh
    body = np.array([[0.0, 0.0, 0.0], [d_oh * sh, d_oh * math.sqrt(1 - sh * sh), 0.0],
                     [-d_oh * sh, d_oh * math.sqrt(1 - sh * sh), 0.0]])
    types = [2, 3, 3]
    R = cfg["rc_lj"] + 2 * d_oh
    acc = 0.0
    for chunk in range(n // 200_000):
        m = 200_000
        r = rng.normal(size=(m, 3))
        r *= (R * rng.random(m) ** (1 / 3) / np.linalg.norm(r, axis=1))[:, None]
        a = np.einsum("mij,kj->mki", _random_rotations(rng, m), body)
        b = np.einsum("mij,kj->mki", _random_rotations(rng, m), body) + r[:, None, :]
        u = np.zeros(m)
        for i in range(3):
            for j in range(3):
                u += _lj_numpy(cfg, types[i], types[j], np.linalg.norm(b[:, j] - a[:, i], axis=1))
        acc += np.sum(np.exp(-cfg["beta"] * u) - 1.0)
    return 4.0 / 3.0 * math.pi * R**3 * acc / n


def test_numpy_pair_potential_matches_oracle():
    cfg = _water_cfg(12.0, q=[0.0] * 4, sig=[2.16, 4.83, 3.166, 1.6], eps=[1.475, 0.0535, 0.65, 0.4])
    p = orc.make_params(cfg)
    for ta, tb in ((2, 2), (2, 3), (3, 3)):
        for r in (1.3, 2.0, 3.1, 4.0, 4.49):
            u, _ = orc.pair(p, ta, tb, r)
            assert _lj_numpy(cfg, ta, tb, np.array([r]))[0] == pytest.approx(u, rel=1e-12, abs=1e-14)


def test_two_waters_quadrature():
    L = 12.0
    V = L**3
    z = 2.0 / V
    # LJ sites on O and H, no charges; rc < L/2 - 2 d_oh: an atom pair whose vector wraps
    # differently from the O-O minimum image is out of range either way
    cfg = _water_cfg(L, q=[0.0] * 4, sig=[2.16, 4.83, 3.166, 1.6], eps=[1.475, 0.0535, 0.65, 0.4],
                     beta_mu=math.log(z), rc_lj=3.9, rc_coul=3.9)
    B = _second_virial(cfg)
    res = _run(cfg, 1, 2, 150000, 16, 700)
    n = np.concatenate([r[0][1000:] for r in res])
    c = np.bincount(n, minlength=3).astype(float)
    r10, r21 = c[1] / c[0], c[2] / c[1]
    per = np.array([np.bincount(r[0][1000:], minlength=3) for r in res], float)
    s21 = np.std(per[:, 2] / per[:, 1], ddof=1) / math.sqrt(len(res))
    s10 = np.std(per[:, 1] / per[:, 0], ddof=1) / math.sqrt(len(res))
    exact21 = 0.5 * z * (V + B)
    print(f"\nP1/P0 {r10:.4f} +- {s10:.4f} (zV {z * V:.4f}); P2/P1 {r21:.4f} +- {s21:.4f} "
          f"(exact {exact21:.4f}, ideal {0.5 * z * V:.4f}, B/V {B / V:.4f})")
    assert abs(r10 - z * V) < 4 * s10
    assert abs(r21 - exact21) < 4 * s21
    assert abs(r21 - 0.5 * z * V) > 4 * s21


def _layout_state(cfg, n_w, n_p, cap_w, seed):
    L = cfg["L"]
    p = orc.make_params(dict(cfg, n_water=n_w, n_pairs=n_p))
    x = wl.aqueous_positions(n_w, n_p, L, seed)
    st = orc.State(p, x, np.zeros_like(x), n_p, n_p, cap_water=cap_w)
    return p, st


def test_water_layout_on_reject_insert_and_delete():
    L = 14.0
    base = _ideal(L, n_f=3)
    # never accepted: the state is restored after every trial
    p, st = _layout_state(dict(base, beta_mu=0.0, no_accept=1, seed=3), 6, 3, 10, 4)
    x0 = st.positions()
    for _ in range(8):
        r = orc.trial(p, st)
        assert r["accepted"] == 0 and st.n_water == 6 and r["status"] == 0
        assert np.array_equal(st.positions(), x0)
    # insertions always accepted (non-interacting atoms at rest: NEMD moves nothing)
    p, st = _layout_state(dict(base, beta_mu=50.0, seed=5), 4, 3, 40, 6)
    for _ in range(30):
        before = st.positions()
        N = st.n_water
        r = orc.trial(p, st)
        if r["move"] == 1:
            assert r["accepted"] == 1 and st.n_water == N + 1
            after = st.positions()
            # waters kept (the constraint step pulls an inserted water's H atoms, placed on the
            # 32-bit grid, onto the exact geometry: a few grid quanta), ions moved up
            assert np.allclose(after[: 3 * N], before[: 3 * N], rtol=0, atol=1e-8)
            assert np.array_equal(after[3 * N + 3:], before[3 * N:])
            assert len(after) == len(before) + 3
            st.v[:] = 0.0  # the inserted water came with thermal velocities: keep all at rest
    assert st.n_water > 8
    # deletions always accepted: the last water fills the slot, the ions move down by three
    p, st = _layout_state(dict(base, beta_mu=-50.0, seed=7), 8, 3, 10, 8)
    seen = 0
    for _ in range(30):
        before = st.positions()
        N = st.n_water
        r = orc.trial(p, st)
        if r["move"] == 0 and N > 0:
            assert r["accepted"] == 1 and st.n_water == N - 1
            k = r["cation"]
            after = st.positions()
            expect = np.concatenate([before[: 3 * (N - 1)], before[3 * N:]])
            if k < N - 1:
                expect[3 * k: 3 * k + 3] = before[3 * (N - 1): 3 * N]
            assert np.allclose(after, expect, rtol=0, atol=1e-8)
            assert np.array_equal(after[3 * (N - 1):], before[3 * N:])
            seen += 1
    assert seen >= 5 and st.n_water < 8
