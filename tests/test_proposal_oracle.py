"""Pins of the learned-proposal oracle (CPU only): gradients against finite differences,
feature counting and field against closed forms, proposal normalisation."""
import math

import numpy as np
import pytest

from oracle import proposal as pr


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    w = pr.init_weights(1) + 0.01 * rng.normal(size=pr.N_WEIGHTS)
    Xc, Xa = rng.normal(size=(7, 96)), rng.normal(size=(7, 96))
    yc, ya = rng.random(7), rng.random(7)
    loss, g = pr.bce_loss_grad(w, Xc, Xa, yc, ya)
    h = 1e-6
    for k in rng.choice(pr.N_WEIGHTS, 60, replace=False):
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        num = (pr.bce_loss_grad(wp, Xc, Xa, yc, ya)[0] - pr.bce_loss_grad(wm, Xc, Xa, yc, ya)[0]) / (2 * h)
        assert g[k] == pytest.approx(num, rel=1e-5, abs=1e-8)


def test_feature_counts_sum_rule_and_single_charge_field():
    L, G = 12.0, 4
    rng = np.random.default_rng(1)
    x = rng.random((30, 3)) * L
    types = np.array([0, 1] * 10 + [2] * 10)
    charges = [1.0, -1.0, -0.8, 0.4]
    F = pr.features(x, types, charges, L, G)
    # every atom is counted once in each of the 27 cells around it
    for s, n_s in ((0, 10), (1, 10), (2, 10)):
        assert F[:, s * 27:(s + 1) * 27].sum() == pytest.approx(0.25 * 27 * n_s)
    assert np.all(F[:, 84:] == 0)
    # one unit charge: the field at the centre of its own cell
    xs = np.array([[1.0, 2.0, 2.5]])
    F1 = pr.features(xs, np.array([0]), charges, L, G)
    c = (np.floor(xs[0] / L * G) + 0.5) * (L / G)
    d = c - xs[0]
    r = np.linalg.norm(d)
    own = int(np.floor(xs[0, 0] / 3) * 16 + np.floor(xs[0, 1] / 3) * 4 + np.floor(xs[0, 2] / 3))
    assert F1[own, 81:84] == pytest.approx(0.1 * d / r**3)
    assert F1[own, 13] == 0.25  # centre neighbour slot of the cation channel


def test_proposal_is_normalised_and_mixes_uniform():
    rng = np.random.default_rng(2)
    logits = rng.normal(size=(512, 2)) * 5
    q = pr.proposal_q(logits)
    assert q.sum(0) == pytest.approx([1.0, 1.0])
    assert q.min() >= pr.EPS_MIX / 512 - 1e-15
    flat = pr.proposal_q(np.zeros((512, 2)))
    assert np.allclose(flat, 1 / 512)


# ---------------------------------------------------------------------------------------
# the C oracle's proposal (used inside its trials) against the numpy statement
# ---------------------------------------------------------------------------------------
from oracle import oracle as orc  # noqa: E402
from paper_2307_11447_gb300 import workloads as wl  # noqa: E402


def _aq_state():
    cfg = wl.aq_config(60, 6, 12.5, 10, n_eq=0, cap_pairs=8, beta_mu=-40.0)
    x = wl.aqueous_positions(60, 6, 12.5, 3)
    return cfg, orc.make_params(cfg), x


def test_c_features_equal_numpy_features_with_exclusions():
    cfg, p, x = _aq_state()
    types = np.array([orc.atom_type(p, a) for a in range(len(x))])
    for ex in ((-1, -1), (180, 185)):
        Fc = orc.proposal_features(p, 4, x, ex)
        Fn = pr.features(x, types, cfg["q"], cfg["L"], 4, exclude=[e for e in ex if e >= 0])
        assert np.allclose(Fc, Fn, rtol=1e-12, atol=1e-13)


def test_c_logits_equal_numpy_forward_fp64_and_bf16():
    cfg, p, x = _aq_state()
    w = pr.init_weights(5)
    types = np.array([orc.atom_type(p, a) for a in range(len(x))])
    F = pr.features(x, types, cfg["q"], cfg["L"], 4)
    for emulate in (False, True):
        lc = orc.proposal_logits(p, orc.make_proposal(4, w, bf16=emulate), x)
        ln = pr.forward(w, F, emulate_bf16=emulate)[0]
        assert np.allclose(lc, ln, rtol=1e-6 if emulate else 1e-12, atol=1e-7 if emulate else 1e-12)
    # the emulated precision stays within the forward error bound of bfloat16 operands
    la = pr.forward(w, F, emulate_bf16=True)[0]
    lf = pr.forward(w, F)[0]
    assert np.abs(la - lf).max() < 0.05 * np.abs(lf).max()


def test_zero_network_gives_unit_proposal_factor():
    cfg = dict(wl.LJ_PHYSICS)
    cfg.update(L=6.0, n_f=2, beta_mu=math.log(10 / 6.0**6), q=[0.0, 0.0], eps=[0.0, 0.0])
    p = orc.make_params(cfg)
    st = orc.State(p, np.random.default_rng(0).random((6, 3)) * 6.0, None, 3, 12)
    orc.init_velocities(p, st)
    q = orc.make_proposal(3, np.zeros(pr.N_WEIGHTS), bf16=False)
    recs = orc.run_cycles_prop(p, q, st, 200, 0)
    assert np.abs(recs["ln_q"]).max() < 1e-12
    ok = recs["status"] == 0
    assert np.all(recs["cell_c"][ok] >= 0) and np.all(recs["cell_c"][ok] < 27)


def _ideal_chain(seed):
    L, lam = 6.0, 10.0
    cfg = dict(wl.LJ_PHYSICS)
    cfg.update(L=L, n_f=2, beta_mu=math.log(lam / L**6), q=[0.0, 0.0], eps=[0.0, 0.0], seed=seed)
    p = orc.make_params(cfg)
    st = orc.State(p, np.random.default_rng(seed).random((6, 3)) * L, None, 3, 16)
    orc.init_velocities(p, st)
    # a strongly count-dependent network: far from uniform and different in every state
    w = pr.unpack(pr.init_weights(11 + seed))
    w["W1"] *= 6.0
    w["W3"] *= 6.0
    q = orc.make_proposal(4, pr.pack(w), bf16=False)
    return orc.run_cycles_prop(p, q, st, 12000, 0)


def test_learned_proposal_keeps_the_ideal_pair_gas_law():
    """detailed balance with a state-dependent proposal: P(N) = lam^N/(N!)^2 / I0(2 sqrt(lam))
    (Eqs. 3-8 with the proposal ratio) whatever the network, if the factor is right"""
    from scipy import special
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(4) as pool:
        res = pool.map(_ideal_chain, range(4))
    n = np.concatenate([r["n_after"][500:] for r in res])
    lnq = np.concatenate([r["ln_q"] for r in res])
    print('ln q spread', lnq.std())
    assert lnq.std() > 0.5  # the proposal is far from uniform
    lam = 10.0
    k = np.arange(9)
    pk = np.exp(k * math.log(lam) - 2 * special.gammaln(k + 1)) / special.i0(2 * math.sqrt(lam))
    hist = np.bincount(n, minlength=20)[:9] / n.size
    print("P(N) chain", np.round(hist, 4), "exact", np.round(pk, 4))
    assert np.abs(hist - pk).max() < 0.02
    mean_exact = (k * pk).sum()
    blocks = np.array([r["n_after"][500:].mean() for r in res])
    assert abs(n.mean() - mean_exact) < 4 * blocks.std(ddof=1) / 2 + 0.02
