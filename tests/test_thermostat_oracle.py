"""The CSVR thermostat of the oracle's equilibrium MD (Bussi, Donadio and Parrinello 2007;
the paper leaves the NVT thermostat open, the reading taken is CSVR).

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
