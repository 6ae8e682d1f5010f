"""Chain-level pins of the oracle: the Metropolis rule of Eqs. 3-8 must reproduce exactly
known grand-canonical laws.

* ideal 1:1 pair gas (LJ and charges off, Delta H = 0 in free flight):
  P(N) = lam^N/(N!)^2 / I_0(2 sqrt(lam)), lam = exp(beta mu) V^2 / Lambda_s^6;
  <N> = sqrt(lam) I_1/I_0 and chi = Var N / <N> -> 1/2 (Eq. 1 discussion).
* two ions with capacity one pair (flyers frozen, no other particles, so Delta H = u_ac):
  P(1)/P(0) = exp(beta mu) V int_box exp(-beta u(r)) d^3r.  This pins the reading that
  H_start of an insertion leaves the flyers out entirely; the other reading would give
  exp(beta mu) V^2.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import oracle as orc
from paper_2307_11447_gb300 import analysis as an
from paper_2307_11447_gb300 import workloads as wl


def _ideal_params(L, beta_mu, n_f=2):
    cfg = dict(wl.LJ_PHYSICS)
    cfg.update(L=L, n_f=n_f, beta_mu=beta_mu, q=[0.0, 0.0], eps=[0.0, 0.0], seed=11, replica=0)
    return orc.make_params(cfg)


def _run_chain(p, n0, cap, n_trials, n_eq=0):
    x = np.random.default_rng(3).random((2 * cap, 3)) * p.L
    st = orc.State(p, x, None, n0, cap)
    orc.init_velocities(p, st)
    return orc.run_cycles(p, st, n_trials, n_eq)


def test_bessel_law_closed_form():
    for lam in (0.5, 30.0, 400.0):
        mean, var = an.ideal_pair_gas(lam)
        s = math.sqrt(lam)
        assert mean == pytest.approx(s * special.i1e(2 * s) / special.i0e(2 * s), rel=1e-10)
    mean, var = an.ideal_pair_gas(1e6)
    assert var / mean == pytest.approx(0.5, rel=2e-3)


def test_ideal_pair_gas_follows_bessel_law():
    L = 10.0
    lam = 30.0
    p = _ideal_params(L, math.log(lam / L**6))
    recs = _run_chain(p, 5, 40, 30000)
    n = recs["n_after"][2000:]
    mean, se = an.block_stats(n, 30)
    exact_mean, exact_var = an.ideal_pair_gas(lam)
    assert abs(mean - exact_mean) < 4 * se + 1e-3, (mean, exact_mean, se)
    hist = np.bincount(n, minlength=20)[:12] / n.size
    k = np.arange(12)
    pk = np.exp(k * math.log(lam) - 2 * special.gammaln(k + 1))
    pk /= np.exp(np.arange(200) * math.log(lam) - 2 * special.gammaln(np.arange(200) + 1)).sum()
    assert np.abs(hist - pk).max() < 0.02
    assert np.all(recs["status"][recs["move"] == 1] == 0)


def test_ideal_pair_gas_chi_half():
    L = 10.0
    lam = 400.0
    p = _ideal_params(L, math.log(lam / L**6))
    recs = _run_chain(p, 20, 80, 30000)
    n = recs["n_after"][2000:]
    chi, se = an.chi_osmotic(n, 30)
    exact_mean, exact_var = an.ideal_pair_gas(lam)
    assert exact_var / exact_mean == pytest.approx(0.5, abs=0.02)
    assert abs(chi - exact_var / exact_mean) < 4 * se + 0.01, (chi, se)


def test_two_ion_quadrature_pins_delta_h_reading():
    cfg = dict(wl.LJ_PHYSICS)
    L = 10.0
    V = L**3
    beta_mu = -13.6
    cfg.update(L=L, n_f=1, beta_mu=beta_mu, seed=5, replica=2)
    p = orc.make_params(cfg)

    def integrand(r):
        u, _ = orc.pair(p, 0, 1, r)
        return (math.exp(-u) - 1.0) * 4 * math.pi * r * r

    inner, _ = integrate.quad(integrand, 0.5, 4.0, limit=200, points=[1.0, 2.5])
    inner += -4.0 / 3.0 * math.pi * 0.5**3  # exp(-u) = 0 inside r < 0.5 to double precision
    ratio_exact = math.exp(beta_mu) * V * (V + inner)
    recs = _run_chain(p, 0, 1, 60000)
    n = recs["n_after"][1000:]
    frac1 = n.mean()
    _, se = an.block_stats(n, 30)
    ratio = frac1 / (1 - frac1)
    dratio = se / (1 - frac1) ** 2
    assert abs(ratio - ratio_exact) < 4 * dratio, (ratio, ratio_exact, dratio)
    # the other reading (flyers' mutual energy in H_start) would give exp(beta mu) V^2
    assert abs(math.exp(beta_mu) * V * V - ratio) > 6 * dratio


def test_records_are_self_consistent():
    cfg = wl.lj_config(40, 0.2, 20)
    cfg.update(seed=3, replica=1, beta_mu=-3.0)
    p = orc.make_params(cfg)
    x = wl.lj_positions(20, cfg["L"], 9)
    st = orc.State(p, x, None, 20, 40)
    orc.init_velocities(p, st)
    orc.md(p, st, 100)
    recs = orc.run_cycles(p, st, 30, 20)
    V = cfg["L"] ** 3
    for r in recs:
        if r["status"] != 0:
            continue
        if r["move"] == 1:
            assert r["beta_dM"] == pytest.approx(r["dH"] - 2 * math.log(V / (r["n_before"] + 1)))
            assert r["x_acc"] == pytest.approx(-r["beta_dM"] + cfg["beta_mu"])
        else:
            assert r["beta_dM"] == pytest.approx(-r["dH"] - 2 * math.log(V / r["n_before"]))
            assert r["x_acc"] == pytest.approx(r["beta_dM"] - cfg["beta_mu"])
        assert bool(r["accepted"]) == (r["ln_u"] < r["x_acc"])
        assert r["n_after"] == r["n_before"] + (0 if not r["accepted"] else (1 if r["move"] == 1 else -1))
    assert st.n_pairs == recs["n_after"][-1]


def test_bar_recovers_mu_from_gaussian_crooks_pair():
    rng = np.random.default_rng(0)
    mu, s2 = -4.0, 6.0
    ins = rng.normal(mu + s2 / 2, math.sqrt(s2), 200000)
    dele = rng.normal(mu - s2 / 2, math.sqrt(s2), 150000)
    assert an.bar_mu(ins, dele) == pytest.approx(mu, abs=0.03)
    # Eq. 21 on a Crooks-consistent Gaussian equals the erfc closed form of Sec. II.E
    assert an.p_acc(ins, mu, True) == pytest.approx(an.p_acc_gauss(s2 / 2), rel=0.02)
    assert an.p_acc(dele, mu, False) == pytest.approx(an.p_acc_gauss(s2 / 2), rel=0.02)
    assert abs(an.alpha2(ins)) < 0.02
