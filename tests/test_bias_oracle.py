"""Pins of the oracle's bimodal flyer-distance bias (Sec. II.B.3): the inverse error
function against scipy, the density's normalisation on the box (Eq. 16), the sampler
against the density, and detailed balance -- the exact ideal pair-gas law reached with
the biased insertion and the B^ins-weighted deletion (Eqs. 17-18).  CPU only."""
import math
import multiprocessing as mp

import numpy as np
import pytest
from scipy import integrate, special

from oracle import oracle as orc
from paper_2307_11447_gb300 import workloads as wl


def test_erfinv_matches_scipy():
    y = np.concatenate([np.linspace(-0.99999, 0.99999, 401), [1e-300, 0.0, 0.5, -0.75]])
    got = np.array([orc.erfinv(v) for v in y])
    assert np.allclose(got, special.erfinv(y), rtol=1e-12, atol=1e-15)
    # near +-1 the double y fixes 1 - |y| only to ~1e-4 relative: any x whose erf is within
    # one ulp of y is as good a draw; the Newton steps land within that band
    for v in (1 - 1e-12, -1 + 1e-12, 1 - 1e-9):
        x = orc.erfinv(v)
        assert abs(math.erf(x) - v) <= 4e-16
        assert x == pytest.approx(special.erfinv(v), rel=1e-5)


@pytest.mark.parametrize("alpha,xb,L", [(5.0, 0.8, 10.77), (5.0, 0.8, 6.0), (0.5, 2.0, 8.0), (20.0, 1.2, 4.0)])
def test_density_is_normalised_on_the_box_and_bimodal(alpha, xb, L):
    f = lambda x: orc.bias_density(alpha, xb, L, x)
    total, _ = integrate.quad(f, -L / 2, L / 2, points=[-xb, xb], limit=200)
    assert total == pytest.approx(1.0, abs=1e-10)
    assert f(0.3) == pytest.approx(f(-0.3), rel=1e-14)
    # peaks at +-xb when the modes are well separated
    if alpha * xb * xb > 2:
        assert f(xb) > f(xb + 0.05) and f(xb) > f(xb - 0.05)


def test_sampler_follows_the_density():
    alpha, xb, L = 5.0, 0.8, 6.0
    rng = np.random.default_rng(0)
    words = rng.integers(0, 2**63, size=(100000, 2), dtype=np.uint64) * 2 + rng.integers(0, 2, size=(100000, 2), dtype=np.uint64)
    x = np.array([orc.bias_offset(alpha, xb, L, int(a), int(b)) for a, b in words])
    assert np.all((x >= -L / 2) & (x < L / 2))
    edges = np.linspace(-L / 2, L / 2, 61)
    hist, _ = np.histogram(x, edges)
    expect = np.array([integrate.quad(lambda t: orc.bias_density(alpha, xb, L, t), a, b)[0]
                       for a, b in zip(edges[:-1], edges[1:])]) * len(x)
    ok = expect > 5
    chi2 = (((hist - expect) ** 2) / expect)[ok].sum()
    dof = ok.sum() - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof), (chi2, dof)


def _biased_chain(seed):
    L, lam = 6.0, 10.0
    cfg = dict(wl.LJ_PHYSICS)
    cfg.update(L=L, n_f=2, beta_mu=math.log(lam / L**6), q=[0.0, 0.0], eps=[0.0, 0.0], seed=seed,
               bias_alpha=5.0, bias_xb=0.8)
    p = orc.make_params(cfg)
    st = orc.State(p, np.random.default_rng(seed).random((6, 3)) * L, None, 3, 16)
    orc.init_velocities(p, st)
    return orc.run_cycles(p, st, 12000, 0)


def test_biased_exchange_keeps_the_ideal_pair_gas_law():
    """P(N) = lam^N / (N!)^2 / I0(2 sqrt(lam)) with the bias on: the insertion factor
    B^del/B^ins (end state) and the deletion factor B^ins/B^del (start state) are right.
    Eight independent chains; each bin within 4 standard errors of the chain means."""
    with mp.get_context("spawn").Pool(8) as pool:
        res = pool.map(_biased_chain, range(8))
    lnq = np.concatenate([r["ln_q"][r["status"] == 0] for r in res])
    assert lnq.std() > 0.3  # the bias factor is far from one
    lam = 10.0
    k = np.arange(9)
    pk = np.exp(k * math.log(lam) - 2 * special.gammaln(k + 1)) / special.i0(2 * math.sqrt(lam))
    H = np.array([np.bincount(r["n_after"][500:], minlength=20)[:9] / (len(r) - 500) for r in res])
    m, se = H.mean(0), H.std(0, ddof=1) / math.sqrt(len(H))
    z = (m - pk) / np.maximum(se, 1e-4)
    print("P(N) biased chains", np.round(m, 4), "exact", np.round(pk, 4), "z", np.round(z, 1))
    assert np.all(np.abs(z) < 4)
