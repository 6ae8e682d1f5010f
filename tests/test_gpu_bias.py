"""The bimodal flyer-distance bias (Sec. II.B.3, Eqs. 14-18) on the GPU against the oracle.

Tolerances: the deleted anion (picked by the B^ins-weighted draw) identical; ln q within
1e-9 for deletions (start state, identical positions) and 1e-5 for insertions (end state
after FP32-force dynamics); beta dM as in the other trial tests (1e-3 kT within 20 kT of
the acceptance boundary, at least half within 2e-5 kT); the ideal pair-gas law within 4
standard errors of the replica means per N.
"""
import math

import numpy as np
import pytest
from scipy import special

from oracle import oracle as orc
from paper_2307_11447_gb300 import lib as h4d
from paper_2307_11447_gb300 import workloads as wl

from .test_gpu_proposal import _lj_state, work_close

pytestmark = pytest.mark.gpu

BIAS = dict(bias_alpha=5.0, bias_xb=0.8)  # the paper's alpha*_b and x*_b


def test_biased_trials_match_oracle():
    cfg, _, x0, v0 = _lj_state(1)
    cfg.update(BIAS)
    po = orc.make_params(cfg, use_cells=0)
    L, n_pairs = cfg["L"], cfg["n_pairs"]
    ctx = h4d.Context(h4d.make_params(cfg), [dict(L=L, n_pairs=n_pairs, cap_pairs=cfg["cap_pairs"], x=x0, v=v0)],
                      seed=cfg["seed"])
    ctx.h4d_set_bias(BIAS["bias_alpha"], BIAS["bias_xb"])
    moves, near = set(), []
    for k in range(12):
        ctx.h4d_set_state(0, n_pairs, x0, v0)
        ctx.h4d_run_trials(1, 0)
        rg = ctx.h4d_get_work(0, 1)[0]
        st = orc.State(po, x0, v0, n_pairs, cfg["cap_pairs"])
        st.s.trial_ctr = k
        ro = orc.trial(po, st)
        moves.add(int(ro["move"]))
        print(f"trial {k}: move {ro['move']} anion gpu {rg['anion']} oracle {ro['anion']} ln q gpu {rg['ln_q']:.9f} "
              f"oracle {ro['ln_q']:.9f} dM diff {rg['beta_dM'] - ro['beta_dM']:+.2e}")
        assert rg["move"] == ro["move"] and rg["status"] == ro["status"] == 0
        assert rg["cation"] == ro["cation"] and rg["anion"] == ro["anion"]
        assert abs(rg["ln_q"] - ro["ln_q"]) <= (1e-5 if ro["move"] == 1 else 1e-9)
        assert work_close(rg["beta_dM"], ro["beta_dM"], ro["x_acc"]), (k, rg["beta_dM"], ro["beta_dM"])
        if abs(ro["x_acc"]) < 20:
            near.append(abs(rg["beta_dM"] - ro["beta_dM"]))
        if abs(ro["ln_u"] - ro["x_acc"]) > 1e-3:
            assert rg["accepted"] == ro["accepted"]
        xg, _ = ctx.h4d_get_state(0)
        xo = st.positions()
        d = xg - xo
        d -= L * np.round(d / L)
        assert xg.shape == xo.shape and np.abs(d).max() < 1e-4
    assert moves == {0, 1}
    assert np.mean(np.array(near) <= 2e-5) >= 0.5, near
    recs = ctx.h4d_get_work(0, 12)
    assert np.abs(recs["ln_q"]).max() > 0.1  # the bias is active


def test_gpu_ideal_pair_gas_with_bias():
    L, lam = 10.0, 30.0
    cfg = dict(wl.LJ_PHYSICS)
    cfg.update(L=L, n_f=2, beta_mu=math.log(lam / L**6), q=[0.0, 0.0], eps=[0.0, 0.0])
    rng = np.random.default_rng(4)
    R = 64
    reps = [dict(L=L, n_pairs=5, cap_pairs=40, x=rng.random((10, 3)) * L) for _ in range(R)]
    ctx = h4d.Context(h4d.make_params(cfg), reps, seed=41)
    ctx.h4d_set_bias(BIAS["bias_alpha"], BIAS["bias_xb"])
    ns = [[] for _ in range(R)]
    for _ in range(3):
        ctx.h4d_run_trials(1000, 0)
        for r in range(R):
            ns[r].append(ctx.h4d_get_work(r, 1000)["n_after"])
    n = np.array([np.concatenate(v) for v in ns])[:, 300:]
    k = np.arange(12)
    pk = np.exp(k * math.log(lam) - 2 * special.gammaln(k + 1)) / special.i0(2 * math.sqrt(lam))
    H = np.array([np.bincount(row, minlength=40)[:12] / row.size for row in n])
    m, se = H.mean(0), H.std(0, ddof=1) / math.sqrt(R)
    z = (m - pk) / np.maximum(se, 1e-4)
    print("P(N) with bias", np.round(m, 4), "exact", np.round(pk, 4), "z", np.round(z, 1))
    assert np.all(np.abs(z) < 4)


def test_bias_api_rejects_bad_settings():
    cfg, _, x0, v0 = _lj_state(1)
    ctx = h4d.Context(h4d.make_params(cfg), [dict(L=cfg["L"], n_pairs=cfg["n_pairs"], cap_pairs=cfg["cap_pairs"],
                                                  x=x0, v=v0)], seed=1)
    with pytest.raises(h4d.H4DError):
        ctx.h4d_set_bias(-1.0, 0.8)
    ctx.h4d_set_bias(5.0, 0.8)
    with pytest.raises(h4d.H4DError):  # one placement rule at a time
        ctx.h4d_proposal(h4d.H4D_PROPOSAL_LEARNED, 1.5, 0.1, 0)
    ctx.h4d_set_bias(0.0, 0.0)
    ctx.h4d_proposal(h4d.H4D_PROPOSAL_LEARNED, 1.5, 0.1, 0)
    with pytest.raises(h4d.H4DError):
        ctx.h4d_set_bias(5.0, 0.8)


def test_bias_effect_on_acceptance_is_measured():
    """fixed-N trials of the 250-ion electrolyte with and without the bias, mean Metropolis
    acceptance at the beta mu that balances insertions and deletions (printed; the bias
    must leave the acceptance finite and the factor active)"""
    cfg = dict(wl.CONFIGS["lj250"])
    cfg.update(beta_mu=0.0)
    L, R = cfg["L"], 64
    reps = [dict(L=L, n_pairs=cfg["n_pairs"], cap_pairs=cfg["cap_pairs"], x=wl.lj_positions(cfg["n_pairs"], L, 90 + r))
            for r in range(R)]
    out = {}
    for name, bias in (("uniform", (0.0, 0.0)), ("bimodal", (5.0, 0.8))):
        ctx = h4d.Context(h4d.make_params(cfg), reps, seed=7)
        ctx.h4d_run_md(500)
        ctx.h4d_set_no_accept(1)
        ctx.h4d_set_bias(*bias)
        ctx.h4d_run_trials(60, 20)
        recs = [ctx.h4d_get_work(r, 60) for r in range(R)]
        rec = np.concatenate(recs)
        rec = rec[rec["status"] == 0]
        out[name] = rec
    ins_u = out["uniform"]["x_acc"][out["uniform"]["move"] == 1]
    del_u = out["uniform"]["x_acc"][out["uniform"]["move"] == 0]
    f = lambda m: np.exp(np.minimum(ins_u + m, 0)).mean() - np.exp(np.minimum(del_u - m, 0)).mean()
    lo, hi = -100.0, 100.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if f(mid) < 0 else (lo, mid)
    mu = 0.5 * (lo + hi)
    acc = {}
    for name, rec in out.items():
        ins = rec["move"] == 1
        x = np.where(ins, rec["x_acc"] + mu, rec["x_acc"] - mu)
        acc[name] = np.exp(np.minimum(x, 0)).mean()
    print(f"balanced beta mu {mu:.3f}; mean acceptance uniform {acc['uniform']:.4f}, bimodal bias "
          f"{acc['bimodal']:.4f} ({acc['bimodal'] / acc['uniform']:.2f}x)")
    assert 0 < acc["uniform"] < 1 and 0 < acc["bimodal"] < 1
    assert np.abs(out["bimodal"]["ln_q"]).max() > 0.1
