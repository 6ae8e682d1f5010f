"""Pins of the oracle's single-particle exchange (Sec. II.A: the pair acceptance rule
translated to one flying particle, the phase-space factor V/(N+1) appearing once).

* Ideal single-species gas (LJ and charges off): the grand-canonical law is Poisson,
  P(N) = (zV)^N e^{-zV} / N! with z = e^{beta mu} (Lambda = 1), so <N> = zV and
  Var N / <N> = 1.  The pair rule (factor squared) gives the Bessel law instead and fails.
* Two interacting particles (capacity two, flyer frozen in 3D): P(1)/P(0) = zV and
  P(2)/P(1) = (z/2) (V + B), B = int_box (e^{-beta u(r)} - 1) d^3r by quadrature, which
  fixes the reading of Delta H (end-state Hamiltonians) for one flyer.
* Rejection restores the state; an accepted deletion removes the chosen particle by
  swapping the last one into its slot.
"""
import math
import multiprocessing as mp
import os

import numpy as np
import pytest
from scipy import integrate, special

from oracle import oracle as orc
from paper_2307_11447_gb300 import workloads as wl


def _fluid(L, **kw):
    cfg = dict(wl.LJ_PHYSICS)
    cfg.update(L=L, exchange="single", q=[0.0, 0.0], rc_coul=2.5, n_f=1, tau_t=0.0)
    cfg.update(kw)
    return cfg


def _chain(job):
    cfg, n0, cap, cycles, seed = job
    p = orc.make_params(dict(cfg, seed=seed, replica=0))
    rng = np.random.default_rng(seed)
    st = orc.State(p, rng.random((cap, 3)) * cfg["L"], np.zeros((cap, 3)), n0, cap)
    recs = orc.run_cycles(p, st, cycles, 0)
    return recs["n_after"], recs["accepted"], recs["move"]


def _run(cfg, n0, cap, cycles, chains, seed0):
    jobs = [(cfg, n0, cap, cycles, seed0 + k) for k in range(chains)]
    with mp.get_context("spawn").Pool(min(chains, os.cpu_count() or 1)) as pool:
        return pool.map(_chain, jobs)


def test_ideal_gas_is_poisson():
    L, lam = 8.0, 12.0
    cfg = _fluid(L, eps=[0.0, 0.0], beta_mu=math.log(lam / L**3))
    res = _run(cfg, 12, 60, 40000, 8, 100)
    n = np.concatenate([r[0][2000:] for r in res]).astype(float)
    means = np.array([r[0][2000:].mean() for r in res])
    se = means.std(ddof=1) / math.sqrt(len(means))
    assert abs(n.mean() - lam) < 4 * se + 1e-3, (n.mean(), lam, se)
    assert abs(n.var() / n.mean() - 1.0) < 0.05, n.var() / n.mean()
    k = np.arange(30)
    pk = np.exp(k * math.log(lam) - lam - special.gammaln(k + 1))
    hist = np.bincount(n.astype(int), minlength=40)[:30] / n.size
    assert np.abs(hist - pk).max() < 0.01
    # the pair factor (V/(N+1))^2 would give the Bessel law, whose variance is about half
    assert n.var() / n.mean() > 0.8


def test_two_particles_quadrature():
    L = 6.0
    V = L**3
    z = 2.0 / V
    cfg = _fluid(L, beta_mu=math.log(z), skin=0.3)
    p = orc.make_params(cfg)

    def integrand(r):
        u, _ = orc.pair(p, 0, 0, r)
        return (math.exp(-u) - 1.0) * 4 * math.pi * r * r

    B, _ = integrate.quad(integrand, 0.6, 2.5, limit=200, points=[1.0, 1.12])
    B += -4.0 / 3.0 * math.pi * 0.6**3  # e^{-beta u} < 1e-30 below 0.6 sigma
    res = _run(cfg, 1, 2, 200000, 16, 500)
    n = np.concatenate([r[0][1000:] for r in res])
    c = np.bincount(n, minlength=3).astype(float)
    r10, r21 = c[1] / c[0], c[2] / c[1]
    # error of the ratios from the spread over chains
    per = np.array([np.bincount(r[0][1000:], minlength=3) for r in res], float)
    s21 = np.std(per[:, 2] / per[:, 1], ddof=1) / math.sqrt(len(res))
    s10 = np.std(per[:, 1] / per[:, 0], ddof=1) / math.sqrt(len(res))
    exact21 = 0.5 * z * (V + B)
    print(f"\nP1/P0 {r10:.4f} (zV {z * V:.4f}); P2/P1 {r21:.4f} +- {s21:.4f} (exact {exact21:.4f}, "
          f"ideal {0.5 * z * V:.4f}, B/V {B / V:.4f})")
    assert abs(r10 - z * V) < 4 * s10
    assert abs(r21 - exact21) < 4 * s21
    # the interaction is resolved: the ideal value lies outside the error bars
    assert abs(r21 - 0.5 * z * V) > 4 * s21


def test_rejection_restores_and_deletion_swaps_last():
    L = 8.0
    cfg = _fluid(L, n_f=5)
    rng = np.random.default_rng(5)
    x0 = wl.lj_positions(6, L, 9)[:10]  # 10 particles
    v0 = rng.normal(size=(10, 3))
    # never accept: the state after each trial is the start state up to the reversals
    p = orc.make_params(dict(cfg, beta_mu=0.0, no_accept=1, seed=3))
    st = orc.State(p, x0, v0, 10, 12)
    for _ in range(6):
        r = orc.trial(p, st)
        assert r["accepted"] == 0 and st.n_pairs == 10
        assert np.array_equal(st.positions(), x0)
        assert np.allclose(np.abs(st.velocities()), np.abs(v0), rtol=0, atol=0)
    # always accept deletions (beta mu very negative) of particles at rest without
    # interactions, so NEMD moves nothing: the chosen particle disappears and the last one
    # takes its slot
    p = orc.make_params(dict(cfg, beta_mu=-1e6, eps=[0.0, 0.0], seed=4))
    st = orc.State(p, x0, np.zeros_like(v0), 10, 12)
    for _ in range(20):
        before = st.positions()
        r = orc.trial(p, st)
        if r["move"] == 0 and r["accepted"]:
            k, N = r["cation"], r["n_before"]
            after = st.positions()
            assert len(after) == N - 1
            expect = before.copy()
            expect[k] = before[N - 1]
            assert np.array_equal(after, expect[: N - 1])
            return
    pytest.fail("no deletion was accepted")
