"""Single-particle exchange on the GPU (Sec. II.A: the pair rule translated to one flying
particle) against the oracle and against exact laws.

* Single trials of an LJ fluid (one species, charges 0) from the same seeded state and
  Philox key as the oracle: the same move, the same chosen particle, beta Delta M within
  the trial-work tolerance (1e-3 kT within 20 kT of the acceptance boundary, at least half
  of those within 2e-5 kT, 1e-3 relative beyond), identical decisions away from ties.
* Ideal single-species gas: Poisson law, <N> = zV and Var N/<N> = 1.
* Two interacting particles: P(1)/P(0) = zV and P(2)/P(1) = (z/2)(V + B), B by quadrature.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import oracle as orc
from paper_2307_11447_gb300 import lib as h4d
from paper_2307_11447_gb300 import workloads as wl

from .parity_util import trial_work_bound

pytestmark = pytest.mark.gpu

TWO32 = 4294967296.0


def quantize(x, L):
    y = np.mod(x, L)
    return np.mod(np.rint(y / L * TWO32), TWO32) * (L / TWO32)


def _fluid(L, **kw):
    cfg = dict(wl.LJ_PHYSICS)
    cfg.update(L=L, exchange="single", q=[0.0, 0.0], rc_coul=2.5)
    cfg.update(kw)
    return cfg


def test_single_particle_trials_match_oracle():
    L, N = 9.0, 300  # LJ fluid at density 0.41
    cfg = _fluid(L, n_f=80, beta_mu=-2.0, seed=41, replica=0)
    po = orc.make_params(cfg, use_cells=1)
    st = orc.State(po, quantize(wl.lj_positions(N // 2, L, 17), L), None, N, N + 40)
    orc.init_velocities(po, st)
    orc.md(po, st, 300)
    x0, v0 = quantize(st.positions(), L), st.velocities()
    ctx = h4d.Context(h4d.make_params(cfg), [dict(L=L, n_pairs=N, cap_pairs=N + 40, x=x0, v=v0)], seed=41)
    moves, near = set(), []
    for k in range(10):
        ctx.h4d_set_state(0, N, x0, v0)
        ctx.h4d_run_trials(1, 0)
        rg = ctx.h4d_get_work(0, 1)[0]
        so = orc.State(po, x0, v0, N, N + 40)
        so.s.trial_ctr = k
        ro = orc.trial(po, so)
        moves.add(int(ro["move"]))
        assert rg["move"] == ro["move"] and rg["status"] == ro["status"] == 0
        assert rg["cation"] == ro["cation"] and rg["anion"] == -1
        err = abs(rg["beta_dM"] - ro["beta_dM"])
        nr = abs(ro["x_acc"]) < 20
        assert err <= trial_work_bound(ro["beta_dM"], ro["x_acc"]), (k, rg["beta_dM"], ro["beta_dM"])
        if nr:
            near.append(err)
        if abs(ro["ln_u"] - ro["x_acc"]) > 1e-3:
            assert rg["accepted"] == ro["accepted"]
    assert moves == {0, 1}
    assert not near or np.mean(np.array(near) <= 2e-5) >= 0.5, near


def _n_series(ctx, R, cycles):
    out = [[] for _ in range(R)]
    done = 0
    while done < cycles:
        k = min(1000, cycles - done)
        ctx.h4d_run_trials(k, 0)
        for r in range(R):
            out[r].extend(ctx.h4d_get_work(r, k)["n_after"].tolist())
        done += k
    return np.array(out)


def test_gpu_single_species_ideal_gas_is_poisson():
    L, lam, R = 9.0, 15.0, 64
    cfg = _fluid(L, n_f=2, eps=[0.0, 0.0], beta_mu=math.log(lam / L**3))
    rng = np.random.default_rng(3)
    reps = [dict(L=L, n_pairs=15, cap_pairs=80, x=rng.random((15, 3)) * L) for _ in range(R)]
    ctx = h4d.Context(h4d.make_params(cfg), reps, seed=11)
    n = _n_series(ctx, R, 4000)[:, 300:]
    per = n.mean(1)
    se = per.std(ddof=1) / math.sqrt(R)
    print(f"\n<N> {n.mean():.3f} +- {se:.3f} (zV {lam}); Var/<N> {n.var() / n.mean():.4f}")
    assert abs(n.mean() - lam) < 4 * se + 1e-3
    assert abs(n.var() / n.mean() - 1.0) < 0.04
    k = np.arange(35)
    pk = np.exp(k * math.log(lam) - lam - special.gammaln(k + 1))
    hist = np.bincount(n.ravel(), minlength=40)[:35] / n.size
    assert np.abs(hist - pk).max() < 0.01


def test_gpu_two_particles_quadrature():
    L = 6.0  # the smallest box the cut-off allows, so that B/V is about 4%
    V = L**3
    z = 2.0 / V
    cfg = _fluid(L, n_f=1, beta_mu=math.log(z))
    p = orc.make_params(cfg)

    def integrand(r):
        u, _ = orc.pair(p, 0, 0, r)
        return (math.exp(-u) - 1.0) * 4 * math.pi * r * r

    B, _ = integrate.quad(integrand, 0.6, 2.5, limit=200, points=[1.0, 1.12])
    B += -4.0 / 3.0 * math.pi * 0.6**3
    R = 128
    rng = np.random.default_rng(4)
    reps = [dict(L=L, n_pairs=1, cap_pairs=2, x=rng.random((2, 3)) * L) for _ in range(R)]
    ctx = h4d.Context(h4d.make_params(cfg), reps, seed=12)
    n = _n_series(ctx, R, 6000)[:, 200:]
    per = np.array([np.bincount(row, minlength=3) for row in n], float)
    r10, r21 = per[:, 1].sum() / per[:, 0].sum(), per[:, 2].sum() / per[:, 1].sum()
    s10 = np.std(per[:, 1] / per[:, 0], ddof=1) / math.sqrt(R)
    s21 = np.std(per[:, 2] / per[:, 1], ddof=1) / math.sqrt(R)
    exact = 0.5 * z * (V + B)
    print(f"\nP1/P0 {r10:.4f} +- {s10:.4f} (zV 2); P2/P1 {r21:.4f} +- {s21:.4f} (exact {exact:.4f}, B/V {B / V:.4f})")
    assert abs(r10 - z * V) < 4 * s10
    assert abs(r21 - exact) < 4 * s21
