"""The learned insertion-site proposal on the GPU against the oracle.

Tolerances (each derived from the arithmetic of the two sides):
  * features: counts bit-exact; field |dE| <= 2e-5 (FP32 contributions summed in fixed
    point on the GPU, FP64 in the oracle);
  * logits against the oracle evaluated in the kernel's precision (bf16 operands, binary32
    sums): |dl| <= 2^-6 l_abs + 1e-5, l_abs the forward pass on absolute values (a change
    of one bfloat16 ulp in any operand moves a logit by at most 2^-8 l_abs);
  * gradients against the oracle with the same forward precision and an exact backward:
    |dg| <= 2^-6 g_abs + 1e-7 max g_abs elementwise, g_abs the backward pass on absolute
    values (the GPU rounds dL/dlogit, dz2 and dz1 to bfloat16: three roundings of 2^-9);
  * trials: the cells drawn are identical, ln q within 1e-4; beta dM within 1e-3 kT for
    trials within 20 kT of the acceptance boundary and at least half of them within
    2e-5 kT (FP32 pair forces alone produce that spread, tests/test_oracle_tolerance.py:
    a pair that lands within binary32 rounding of a cut-off is counted in a different
    step; trials from one state replay the same bulk trajectory, so such an event can be
    shared by several of them), else within 1e-3 relative (insertions onto an overlap
    exchange up to 1e6 kT under forces of 1e20 that FP32 and FP64 integrate apart; their
    acceptance is zero on both sides);
  * detailed balance: the ideal pair gas with a strongly state-dependent network keeps
    P(N) = lam^N / (N!)^2 / I0(2 sqrt(lam)) within 0.01 per N.
"""
import math

import numpy as np
import pytest
from scipy import special

from oracle import oracle as orc
from oracle import proposal as pr
from paper_2307_11447_gb300 import lib as h4d
from paper_2307_11447_gb300 import workloads as wl

from .parity_util import trial_work_bound

pytestmark = pytest.mark.gpu

TWO32 = 4294967296.0


def quantize(x, L):
    y = np.mod(x, L)
    return np.mod(np.rint(y / L * TWO32), TWO32) * (L / TWO32)


def work_close(g, o, x_acc):
    return abs(g - o) <= trial_work_bound(o, x_acc)


def f32_weights(seed, scale1=1.0, scale3=1.0):
    w = pr.unpack(pr.init_weights(seed))
    rng = np.random.default_rng(seed + 100)
    w["b1"] = rng.normal(0, 0.1, w["b1"].shape)
    w["b2"] = rng.normal(0, 0.1, w["b2"].shape)
    w["b3"] = rng.normal(0, 0.1, w["b3"].shape)
    w["W1"] *= scale1
    w["W3"] *= scale3
    return pr.pack(w).astype(np.float32).astype(np.float64)


# ---------------------------------------------------------------------------------------
# training kernels: loss and gradient
# ---------------------------------------------------------------------------------------
def _records(n, seed):
    """feature rows shaped like the grid's: counts/4 in the first 81 slots, a field, zeros"""
    rng = np.random.default_rng(seed)
    f = np.zeros((n, 2, 96), np.float32)
    f[:, :, :81] = 0.25 * rng.poisson(0.8, (n, 2, 81))
    f[:, :, 81:84] = rng.normal(0, 0.3, (n, 2, 3))
    t = rng.random((n, 2)).astype(np.float32)
    t[:, 1] = t[:, 0]  # one target per record
    return f, t


@pytest.mark.parametrize("n", [1, 7, 64, 1000])
def test_gradient_matches_oracle(n):
    w = f32_weights(3)
    f, t = _records(n, n)
    Xc, Xa = f[:, 0].astype(np.float64), f[:, 1].astype(np.float64)
    tc, ta = t[:, 0].astype(np.float64), t[:, 1].astype(np.float64)
    loss_o, g_o = pr.bce_loss_grad(w, Xc, Xa, tc, ta, emulate_bf16=True)
    _, g_abs = pr.bce_loss_grad(w, Xc, Xa, tc, ta, absolute=True, emulate_bf16=True)
    loss_g, g_g = h4d.h4d_proposal_grad(w, f, t)
    assert loss_g == pytest.approx(loss_o, rel=1e-5)
    err = np.abs(g_g - g_o)
    bound = 2.0**-6 * g_abs + 1e-7 * g_abs.max()
    worst = int(np.argmax(err / bound))
    print(f"n={n}: loss gpu {loss_g:.6f} oracle {loss_o:.6f}; max err/bound {err[worst] / bound[worst]:.3f}")
    assert np.all(err <= bound), (worst, g_g[worst], g_o[worst], bound[worst])
    # and against the plain FP64 gradient: the bf16 forward stays close in norm
    _, g64 = pr.bce_loss_grad(w, Xc, Xa, tc, ta)
    assert np.linalg.norm(g_g - g64) < 0.05 * np.linalg.norm(g64)


def test_gradient_of_a_bias_only_network_is_the_mean_residual():
    """with all weights but b3 zero, every logit is b3 and dL/db3 = mean(sigmoid(b3) - t)"""
    w = np.zeros(pr.N_WEIGHTS)
    w[-2:] = [0.3, -0.7]
    f, t = _records(33, 5)
    loss, g = h4d.h4d_proposal_grad(w, f, t)
    sig = 1 / (1 + np.exp(-np.array([0.3, -0.7])))
    expect = [(sig[0] - t[:, 0]).mean(), (sig[1] - t[:, 1]).mean()]
    assert g[-2:] == pytest.approx(expect, rel=1e-2, abs=1e-6)
    assert np.all(g[:-2] == 0.0)


# ---------------------------------------------------------------------------------------
# grid features and logits of a replica's state
# ---------------------------------------------------------------------------------------
NW, NP, LAQ = 400, 10, 24.0


def _aq_ctx(weights, cell_len=2.8, records=0, mode=h4d.H4D_PROPOSAL_LEARNED):
    cfg = wl.aq_config(NW, NP, LAQ, 20, n_eq=0, cap_pairs=16, beta_mu=-40.0, seed=4, replica=0)
    x = quantize(wl.aqueous_positions(NW, NP, LAQ, 2), LAQ)
    ctx = h4d.Context(h4d.make_params(cfg), [dict(L=LAQ, n_pairs=NP, cap_pairs=16, x=x, n_water=NW)], seed=4)
    ctx.h4d_proposal(mode, cell_len, 0.1, records)
    if weights is not None:
        ctx.h4d_proposal_set_weights(weights)
    return cfg, x, ctx


def test_features_and_logits_match_oracle():
    w = f32_weights(7)
    cfg, x, ctx = _aq_ctx(w)
    lg, ft = ctx.h4d_proposal_logits(0, features=True)
    p = orc.make_params(cfg)
    G = int(round(len(lg) ** (1 / 3)))
    assert G == 8 and len(lg) == 512
    Fo = orc.proposal_features(p, G, x)
    assert np.array_equal(ft[:, :81], Fo[:, :81].astype(np.float32))
    assert np.abs(ft[:, 81:84] - Fo[:, 81:84]).max() <= 2e-5
    assert np.all(ft[:, 84:] == 0)
    lo = orc.proposal_logits(p, orc.make_proposal(G, w, bf16=True), x)
    l_abs = pr.forward_abs(w, Fo)
    err = np.abs(lg - lo)
    bound = 2.0**-6 * l_abs + 1e-5
    print("logit max err", err.max(), "max err/bound", (err / bound).max())
    assert np.all(err <= bound)


def _lj_state(seed, n_f=30):
    cfg = dict(wl.CONFIGS["lj250"])
    cfg.update(seed=seed, replica=0, beta_mu=-8.0, n_f=n_f)
    L = cfg["L"]
    po = orc.make_params(cfg, use_cells=0)
    st = orc.State(po, quantize(wl.lj_positions(cfg["n_pairs"], L, seed), L), None, cfg["n_pairs"], cfg["cap_pairs"])
    orc.init_velocities(po, st)
    orc.md(po, st, 200)
    return cfg, po, quantize(st.positions(), L), st.velocities()


def test_uniform_mode_records_match_oracle():
    """uniform placement with recording: the record of each trial holds the features of the
    cells of the exchanged ions in the N-pair state of the move and the exponent y"""
    cfg, po, x0, v0 = _lj_state(5)
    L, n_pairs = cfg["L"], cfg["n_pairs"]
    ctx = h4d.Context(h4d.make_params(cfg), [dict(L=L, n_pairs=n_pairs, cap_pairs=cfg["cap_pairs"], x=x0, v=v0)],
                      seed=5)
    ctx.h4d_proposal(h4d.H4D_PROPOSAL_UNIFORM, 1.5, 0.1, 64)
    G = max(3, int(math.floor(L / 1.5)))
    q = orc.make_proposal(G, None)
    moves, near = set(), []
    for k in range(8):
        ctx.h4d_set_state(0, n_pairs, x0, v0)
        ctx.h4d_run_trials(1, 0)
        rg = ctx.h4d_get_work(0, 1)[0]
        fg, yg, mg, sg = ctx.h4d_proposal_records(0)
        sto = orc.State(po, x0, v0, n_pairs, cfg["cap_pairs"])
        sto.s.trial_ctr = k
        ro, fo, yo = orc.trial_prop(po, q, sto, want_site=True)
        moves.add(int(ro["move"]))
        assert rg["move"] == ro["move"] and rg["cell_c"] == ro["cell_c"] and rg["cell_a"] == ro["cell_a"]
        assert rg["ln_q"] == 0.0 and ro["ln_q"] == 0.0
        assert mg[-1] == ro["move"] and sg[-1] == 0
        assert np.array_equal(fg[-1][:, :81], fo[:, :81].astype(np.float32))
        assert np.abs(fg[-1][:, 81:84] - fo[:, 81:84]).max() <= 2e-5
        assert work_close(yg[-1], yo, ro["x_acc"]), (k, yg[-1], yo)
        if abs(ro["x_acc"]) < 20:
            near.append(abs(yg[-1] - yo))
    assert moves == {0, 1}
    assert np.mean(np.array(near) <= 2e-5) >= 0.5, near


# ---------------------------------------------------------------------------------------
# trials with the learned proposal
# ---------------------------------------------------------------------------------------
def test_learned_trials_match_oracle():
    cfg, po, x0, v0 = _lj_state(6)
    L, n_pairs = cfg["L"], cfg["n_pairs"]
    w = f32_weights(9, scale1=3.0, scale3=3.0)
    ctx = h4d.Context(h4d.make_params(cfg), [dict(L=L, n_pairs=n_pairs, cap_pairs=cfg["cap_pairs"], x=x0, v=v0)],
                      seed=6)
    ctx.h4d_proposal(h4d.H4D_PROPOSAL_LEARNED, 1.5, 0.1, 0)
    ctx.h4d_proposal_set_weights(w)
    G = max(3, int(math.floor(L / 1.5)))
    q = orc.make_proposal(G, w, bf16=True)
    moves, near = set(), []
    for k in range(10):
        ctx.h4d_set_state(0, n_pairs, x0, v0)
        ctx.h4d_run_trials(1, 0)
        rg = ctx.h4d_get_work(0, 1)[0]
        sto = orc.State(po, x0, v0, n_pairs, cfg["cap_pairs"])
        sto.s.trial_ctr = k
        ro = orc.trial_prop(po, q, sto)
        moves.add(int(ro["move"]))
        print(f"trial {k}: move {ro['move']} cells gpu ({rg['cell_c']},{rg['cell_a']}) oracle "
              f"({ro['cell_c']},{ro['cell_a']}) ln q gpu {rg['ln_q']:.6f} oracle {ro['ln_q']:.6f} "
              f"dM diff {rg['beta_dM'] - ro['beta_dM']:+.2e}")
        assert rg["move"] == ro["move"] and rg["status"] == ro["status"] == 0
        assert rg["cell_c"] == ro["cell_c"] and rg["cell_a"] == ro["cell_a"]
        assert abs(rg["ln_q"] - ro["ln_q"]) <= 1e-4
        assert work_close(rg["beta_dM"], ro["beta_dM"], ro["x_acc"]), (k, rg["beta_dM"], ro["beta_dM"])
        assert work_close(rg["x_acc"], ro["x_acc"], ro["x_acc"])
        if abs(ro["x_acc"]) < 20:
            near.append(abs(rg["beta_dM"] - ro["beta_dM"]))
        if abs(ro["ln_u"] - ro["x_acc"]) > 1e-3:
            assert rg["accepted"] == ro["accepted"]
        xg, _ = ctx.h4d_get_state(0)
        xo = sto.positions()
        d = xg - xo
        d -= L * np.round(d / L)
        # a cut-off flip (see the work tolerance) moves an atom by at most
        # n_f dt (dF dt / m) ~ 4e-5 sigma over the trajectory
        assert xg.shape == xo.shape and np.abs(d).max() < 1e-4
    assert moves == {0, 1}
    assert np.mean(np.array(near) <= 2e-5) >= 0.5, near
    # the network is far from uniform: the factor moves the exponent by order one
    recs = ctx.h4d_get_work(0, 10)
    assert np.abs(recs["ln_q"]).max() > 0.5


def test_gpu_ideal_pair_gas_with_learned_proposal():
    """detailed balance with a state-dependent proposal on the GPU: the exact law survives"""
    L, lam = 10.0, 30.0
    cfg = dict(wl.LJ_PHYSICS)
    cfg.update(L=L, n_f=2, beta_mu=math.log(lam / L**6), q=[0.0, 0.0], eps=[0.0, 0.0])
    rng = np.random.default_rng(3)
    reps = [dict(L=L, n_pairs=5, cap_pairs=40, x=rng.random((10, 3)) * L) for _ in range(64)]
    ctx = h4d.Context(h4d.make_params(cfg), reps, seed=31)
    ctx.h4d_proposal(h4d.H4D_PROPOSAL_LEARNED, 2.5, 0.1, 0)
    ctx.h4d_proposal_set_weights(f32_weights(12, scale1=6.0, scale3=6.0))
    ns, lnq = [[] for _ in range(64)], []
    for _ in range(3):
        ctx.h4d_run_trials(1000, 0)
        for r in range(64):
            rec = ctx.h4d_get_work(r, 1000)
            ns[r].append(rec["n_after"])
            lnq.append(rec["ln_q"])
    n = np.array([np.concatenate(v) for v in ns])[:, 300:]
    spread = np.concatenate(lnq).std()
    k = np.arange(12)
    pk = np.exp(k * math.log(lam) - 2 * special.gammaln(k + 1)) / special.i0(2 * math.sqrt(lam))
    hist = np.bincount(n.ravel(), minlength=20)[:12] / n.size
    print("ln q spread", spread, "P(N)", np.round(hist, 4), "exact", np.round(pk, 4))
    assert spread > 0.5
    assert np.abs(hist - pk).max() < 0.01


# ---------------------------------------------------------------------------------------
# training on self-generated records, and what it gains
# ---------------------------------------------------------------------------------------
def test_training_step_follows_the_gradient_and_lowers_the_loss():
    cfg = dict(wl.lj_config(250, 0.35, 20, cap_pairs=160))
    cfg.update(beta_mu=-4.0)
    L = cfg["L"]
    reps = [dict(L=L, n_pairs=125, cap_pairs=cfg["cap_pairs"], x=wl.lj_positions(125, L, 40 + r)) for r in range(32)]
    ctx = h4d.Context(h4d.make_params(cfg), reps, seed=2)
    ctx.h4d_run_md(200)
    ctx.h4d_proposal(h4d.H4D_PROPOSAL_UNIFORM, 1.5, 0.1, 256)
    ctx.h4d_set_no_accept(1)
    ctx.h4d_run_trials(40, 5)
    feats, ys = [], []
    for r in range(32):
        f, y, m, s = ctx.h4d_proposal_records(r)
        assert len(y) == 40 and np.all((s == 0) | (s == 3))
        ok = s == 0  # training skips trials whose work was not finite
        feats.append(f[ok])
        ys.append(y[ok])
    y = np.concatenate(ys)
    y0 = float(np.percentile(y, 90))
    w0 = f32_weights(21)
    ctx.h4d_proposal_set_weights(w0)
    # full-batch step from zero Adam moments: w1 - w0 = -lr g / (|g| + 1e-8) elementwise;
    # the batch is every valid record in ring order (replica by replica, oldest first)
    tgt = np.exp(np.minimum(y - y0, 0.0))
    f_all = np.concatenate(feats)
    loss0, g = h4d.h4d_proposal_grad(w0, f_all, np.stack([tgt, tgt], 1))
    lr = 1e-3
    loss_step = ctx.h4d_train_proposal(1, 1 << 20, lr, y0, seed=1)
    assert loss_step == pytest.approx(loss0, rel=1e-5)
    w1 = ctx.h4d_proposal_get_weights()
    big = np.abs(g) > 1e-4 * np.abs(g).max()
    assert np.all(np.sign(w1 - w0)[big] == -np.sign(g)[big])
    assert np.abs(w1 - w0).max() <= lr * 1.001
    # more steps lower the loss
    losses = [ctx.h4d_train_proposal(50, 512, 3e-3, y0, seed=s) for s in range(4)]
    print("training loss", loss0, losses)
    assert losses[-1] < 0.9 * loss0


def _fixed_n_records(ctx, R, cycles):
    ctx.h4d_run_trials(cycles, 3)
    return [ctx.h4d_get_work(r, cycles) for r in range(R)]


def _mean_acceptance(recs, beta_mu):
    """per replica, the mean Metropolis acceptance min(1, e^x) of its trials re-evaluated at
    beta_mu (records were taken at beta_mu = 0): x = -beta dM + beta mu - ln q for an
    insertion and beta dM - beta mu + ln q for a deletion"""
    out = []
    for rec in recs:
        ok = rec["status"] == 0
        ins = rec["move"][ok] == 1
        x = np.where(ins, rec["x_acc"][ok] + beta_mu, rec["x_acc"][ok] - beta_mu)
        out.append(np.exp(np.minimum(x, 0.0)).mean())
    return np.array(out)


def _balanced_mu(recs):
    """beta mu at which uniform insertions and deletions are accepted equally often"""
    ins = np.concatenate([r["x_acc"][(r["status"] == 0) & (r["move"] == 1)] for r in recs])
    dele = np.concatenate([r["x_acc"][(r["status"] == 0) & (r["move"] == 0)] for r in recs])
    f = lambda m: np.exp(np.minimum(ins + m, 0)).mean() - np.exp(np.minimum(dele - m, 0)).mean()
    lo, hi = -200.0, 200.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if f(mid) < 0 else (lo, mid)
    return 0.5 * (lo + hi)


def test_trained_proposal_gains_acceptance():
    """dense LJ electrolyte with a short switching protocol: uniform insertions mostly land on
    occupied space; the network trained on the method's own records (0.5 sigma cells, target
    shift y0 = median exponent) steers them to cavities.  Fixed-N sampling from the same
    ensemble gives both proposals' trials; their mean Metropolis acceptance is compared at
    the beta mu where uniform insertions and deletions are accepted equally often (the
    equilibrium condition of Eqs. 3-8 at this N)."""
    cfg = dict(wl.lj_config(300, 0.45, 20, cap_pairs=200))
    cfg.update(beta_mu=0.0)
    L = cfg["L"]
    R = 64
    reps = [dict(L=L, n_pairs=150, cap_pairs=cfg["cap_pairs"], x=wl.lj_positions(150, L, 70 + r)) for r in range(R)]
    ctx = h4d.Context(h4d.make_params(cfg), reps, seed=3)
    ctx.h4d_run_md(300)
    ctx.h4d_set_no_accept(1)
    ctx.h4d_proposal(h4d.H4D_PROPOSAL_UNIFORM, 0.5, 0.1, 512)
    base = _fixed_n_records(ctx, R, 200)
    mu = _balanced_mu(base)
    y = np.concatenate([ctx.h4d_proposal_records(r)[1] for r in range(R)])
    y0 = float(np.median(y))
    ctx.h4d_proposal_set_weights(f32_weights(5))
    for s in range(10):
        loss = ctx.h4d_train_proposal(100, 1024, 2e-3, y0, seed=s)
    ctx.h4d_proposal(h4d.H4D_PROPOSAL_LEARNED, 0.5, 0.1, 0)
    lrn = _fixed_n_records(ctx, R, 200)
    pb, pl = _mean_acceptance(base, mu), _mean_acceptance(lrn, mu)
    se = math.sqrt(pb.var(ddof=1) / R + pl.var(ddof=1) / R)
    print(f"records {len(y)}, final loss {loss:.4f}, balanced beta mu {mu:.3f}; mean acceptance uniform "
          f"{pb.mean():.5f}, learned {pl.mean():.5f}; gain {pl.mean() / pb.mean():.2f}x (se {se:.5f})")
    assert pl.mean() - pb.mean() > 3 * se
    assert pl.mean() > 2.0 * pb.mean()
