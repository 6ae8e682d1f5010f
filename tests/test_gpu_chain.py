"""Chain-level checks of the GPU engine.

* exact laws (no oracle needed): the ideal 1:1 pair gas must follow
  P(N) = lam^N/(N!)^2 / I_0(2 sqrt(lam)) and two ions with capacity one pair must satisfy
  P(1)/P(0) = exp(beta mu) V int exp(-beta u) d^3r (Eqs. 3-8 with the reading of Delta H);
* statistical parity with the FP64 oracle on an interacting LJ electrolyte: <N>,
  chi_osmotic = Var N/<N> (Eq. 1 at fixed V) and the insertion/deletion acceptance rates
  agree within 2 combined standard errors (the z-scores are printed);
* fixed-N work sampling never accepts;
* checkpoint/resume continues bit-identically.
"""
import math
import multiprocessing as mp
import os

import numpy as np
import pytest
from scipy import integrate, special

from oracle import oracle as orc
from paper_2307_11447_gb300 import analysis as an
from paper_2307_11447_gb300 import lib as h4d
from paper_2307_11447_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _ctx(cfg, n_rep, n0, cap, seed, x_seed=3):
    rng = np.random.default_rng(x_seed)
    reps = []
    for r in range(n_rep):
        x = rng.random((2 * cap, 3)) * cfg["L"]
        reps.append(dict(L=cfg["L"], n_pairs=n0, cap_pairs=cap, x=x[: 2 * n0]))
    return h4d.Context(h4d.make_params(cfg), reps, seed=seed)


def _n_series(ctx, n_rep, cycles):
    """run cycles in chunks (records keep the last 1024 per replica) and collect N"""
    out = [[] for _ in range(n_rep)]
    done = 0
    while done < cycles:
        k = min(1000, cycles - done)
        ctx.h4d_run_trials(k, ctx._n_eq)
        for r in range(n_rep):
            rec = ctx.h4d_get_work(r, k)
            out[r].extend(rec["n_after"].tolist())
        done += k
    return np.array(out)


def test_gpu_ideal_pair_gas_bessel_law():
    L, lam = 10.0, 30.0
    cfg = dict(wl.LJ_PHYSICS)
    cfg.update(L=L, n_f=2, beta_mu=math.log(lam / L**6), q=[0.0, 0.0], eps=[0.0, 0.0])
    ctx = _ctx(cfg, 64, 5, 40, seed=17)
    ctx._n_eq = 0
    n = _n_series(ctx, 64, 3000)[:, 300:]
    exact_mean, exact_var = an.ideal_pair_gas(lam)
    per_chain = n.mean(1)
    se = per_chain.std(ddof=1) / math.sqrt(len(per_chain))
    assert abs(n.mean() - exact_mean) < 4 * se + 1e-3, (n.mean(), exact_mean, se)
    k = np.arange(12)
    pk = np.exp(k * math.log(lam) - 2 * special.gammaln(k + 1)) / special.i0(2 * math.sqrt(lam))
    hist = np.bincount(n.ravel(), minlength=20)[:12] / n.size
    assert np.abs(hist - pk).max() < 0.01


def test_gpu_two_ion_quadrature():
    L, beta_mu = 10.0, -13.6
    V = L**3
    cfg = dict(wl.LJ_PHYSICS)
    cfg.update(L=L, n_f=1, beta_mu=beta_mu)
    p = orc.make_params(cfg)

    def integrand(r):
        u, _ = orc.pair(p, 0, 1, r)
        return (math.exp(-u) - 1.0) * 4 * math.pi * r * r

    inner, _ = integrate.quad(integrand, 0.5, 4.0, limit=200, points=[1.0, 2.5])
    inner += -4.0 / 3.0 * math.pi * 0.5**3
    ratio_exact = math.exp(beta_mu) * V * (V + inner)
    ctx = _ctx(cfg, 64, 0, 1, seed=23)
    ctx._n_eq = 0
    n = _n_series(ctx, 64, 4000)[:, 200:]
    f = n.mean(1)
    frac, se = f.mean(), f.std(ddof=1) / math.sqrt(len(f))
    ratio, dratio = frac / (1 - frac), se / (1 - frac) ** 2
    assert abs(ratio - ratio_exact) < 4 * dratio, (ratio, ratio_exact, dratio)


# ---------------------------------------------------------------------------------------
# interacting electrolyte: GPU vs oracle statistics
# ---------------------------------------------------------------------------------------
STAT_CFG = dict(wl.lj_config(100, 0.1, 100), beta_mu=-10.5, cap_pairs=120)
STAT_CYCLES, STAT_NEQ, STAT_BURN = 400, 20, 100


def _oracle_chain(seed):
    cfg = dict(STAT_CFG)
    cfg.update(seed=seed, replica=0)
    p = orc.make_params(cfg)
    x = wl.lj_positions(50, cfg["L"], 1000 + seed)
    st = orc.State(p, x, None, 50, cfg["cap_pairs"])
    orc.init_velocities(p, st)
    orc.md(p, st, 200)
    recs = orc.run_cycles(p, st, STAT_CYCLES, STAT_NEQ)
    return recs["n_after"], recs["move"], recs["accepted"]


def test_gpu_statistics_match_oracle():
    n_or = 16
    with mp.get_context("spawn").Pool(min(n_or, os.cpu_count() or 1)) as pool:
        res = pool.map(_oracle_chain, range(n_or))
    cfg = dict(STAT_CFG)
    reps = [dict(L=cfg["L"], n_pairs=50, cap_pairs=cfg["cap_pairs"], x=wl.lj_positions(50, cfg["L"], 5000 + r))
            for r in range(128)]
    ctx = h4d.Context(h4d.make_params(cfg), reps, seed=99)
    ctx.h4d_run_md(200)
    ctx._n_eq = STAT_NEQ
    ctx.h4d_run_trials(STAT_CYCLES, STAT_NEQ)
    gn, gchi, gacc_i, gacc_d = [], [], [], []
    for r in range(128):
        rec = ctx.h4d_get_work(r, STAT_CYCLES)
        gn.append(rec["n_after"][STAT_BURN:].mean())
        gchi.append(an.chi_osmotic(rec["n_after"][STAT_BURN:])[0])
        ins = rec["move"][STAT_BURN:] == 1
        acc = rec["accepted"][STAT_BURN:] == 1
        gacc_i.append(acc[ins].mean() if ins.any() else 0.0)
        gacc_d.append(acc[~ins].mean() if (~ins).any() else 0.0)
    on = [r[0][STAT_BURN:].mean() for r in res]
    ochi = [an.chi_osmotic(r[0][STAT_BURN:])[0] for r in res]
    oacc_i = [r[2][STAT_BURN:][r[1][STAT_BURN:] == 1].mean() for r in res]
    oacc_d = [r[2][STAT_BURN:][r[1][STAT_BURN:] == 0].mean() for r in res]

    def z(a, b):
        a, b = np.asarray(a), np.asarray(b)
        se = math.sqrt(a.var(ddof=1) / a.size + b.var(ddof=1) / b.size)
        return abs(a.mean() - b.mean()) / max(se, 1e-12), a.mean(), b.mean()

    zn, zi, zd, zc = z(gn, on), z(gacc_i, oacc_i), z(gacc_d, oacc_d), z(gchi, ochi)
    print(f"<N> gpu {zn[1]:.3f} oracle {zn[2]:.3f} z={zn[0]:.2f}; acc_ins gpu {zi[1]:.4f} oracle {zi[2]:.4f} "
          f"z={zi[0]:.2f}; acc_del gpu {zd[1]:.4f} oracle {zd[2]:.4f} z={zd[0]:.2f}; "
          f"chi gpu {zc[1]:.3f} oracle {zc[2]:.3f} z={zc[0]:.2f}")
    assert zn[0] < 2 and zi[0] < 2 and zd[0] < 2 and zc[0] < 2
    assert zi[1] > 0.01  # the comparison is not vacuous


def test_gpu_fixed_n_mode_never_accepts():
    cfg = dict(STAT_CFG)
    reps = [dict(L=cfg["L"], n_pairs=50, cap_pairs=cfg["cap_pairs"], x=wl.lj_positions(50, cfg["L"], 77 + r))
            for r in range(8)]
    ctx = h4d.Context(h4d.make_params(cfg, beta_mu=50.0), reps, seed=5)
    ctx.h4d_set_no_accept(1)
    ctx.h4d_run_md(100)
    ctx.h4d_run_trials(40, 5)
    for r in range(8):
        rec = ctx.h4d_get_work(r, 40)
        assert rec["accepted"].sum() == 0 and np.all(rec["n_after"] == 50)
        assert np.isfinite(rec["beta_dM"]).all()


def test_gpu_checkpoint_resume_is_bit_identical(tmp_path):
    cfg = dict(STAT_CFG)
    reps = [dict(L=cfg["L"], n_pairs=50, cap_pairs=cfg["cap_pairs"], x=wl.lj_positions(50, cfg["L"], 300 + r))
            for r in range(4)]
    a = h4d.Context(h4d.make_params(cfg), reps, seed=8)
    a.h4d_run_md(50)
    a.h4d_run_trials(5, 10)
    path = str(tmp_path / "ck.bin")
    a.h4d_save(path)
    a.h4d_run_trials(6, 10)
    b = h4d.Context(h4d.make_params(cfg), reps, seed=123)  # seed is restored from the file
    b.h4d_load(path)
    b.h4d_run_trials(6, 10)
    for r in range(4):
        xa, va = a.h4d_get_state(r)
        xb, vb = b.h4d_get_state(r)
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
        wa, wb = a.h4d_get_work(r, 11), b.h4d_get_work(r, 11)
        assert wa.tobytes() == wb.tobytes()
        ca, cb = a.h4d_get_counts(r), b.h4d_get_counts(r)
        for k in ("n_pairs", "cycles", "accepted_ins", "accepted_del", "md_steps"):
            assert ca[k] == cb[k]


def _fixed_n_bdm(cfg, n_pairs, move, R, seed0):
    reps = [dict(L=cfg["L"], n_pairs=n_pairs, cap_pairs=cfg["cap_pairs"], x=wl.lj_positions(n_pairs, cfg["L"], seed0 + r))
            for r in range(R)]
    ctx = h4d.Context(h4d.make_params(cfg), reps, seed=seed0)
    ctx.h4d_run_md(300)
    ctx.h4d_set_no_accept(1)
    ctx.h4d_run_trials(300, 20)
    out = []
    for r in range(R):
        rec = ctx.h4d_get_work(r, 300)
        ok = (rec["status"] == 0) & (rec["move"] == move)
        out.append(rec["beta_dM"][ok])
    return out


def test_bar_mu_from_fixed_n_work_balances_grand_canonical_occupation():
    """SI Sec. S1: the BAR estimate of beta mu from fixed-N insertion work at N and
    deletion work at N+1 (Crooks, Eq. S1) is the beta mu at which grand-canonical chains
    occupy N and N+1 equally: P(N+1)/P(N) = 1 within the errors of both (the BAR error
    from a bootstrap over replicas, the occupation ratio from replica means)"""
    # a dense liquid state point (200 ions at rho 0.3), where P(N) is narrow and unimodal
    # (the dilute electrolyte of the other chain tests sits near liquid-vapour coexistence,
    # where grand-canonical chains wander far from any one N)
    cfg = dict(wl.lj_config(200, 0.3, 300, cap_pairs=140, beta_mu=0.0))
    N, R = 100, 64
    ins = _fixed_n_bdm(cfg, N, 1, R, 700)
    dele = _fixed_n_bdm(cfg, N + 1, 0, R, 900)
    mu = an.bar_mu(np.concatenate(ins), np.concatenate(dele))
    rng = np.random.default_rng(0)
    boots = []
    for _ in range(40):
        a = rng.integers(0, R, R)
        b = rng.integers(0, R, R)
        boots.append(an.bar_mu(np.concatenate([ins[i] for i in a]), np.concatenate([dele[j] for j in b])))
    s_mu = float(np.std(boots, ddof=1))
    RG = 128
    reps = [dict(L=cfg["L"], n_pairs=N, cap_pairs=cfg["cap_pairs"], x=wl.lj_positions(N, cfg["L"], 1100 + r))
            for r in range(RG)]
    ctx = h4d.Context(h4d.make_params(cfg, beta_mu=mu), reps, seed=77)
    ctx.h4d_run_md(300)
    ctx._n_eq = 20
    n = _n_series(ctx, RG, 1500)[:, 300:]
    c_n = (n == N).sum(1).astype(float)
    c_n1 = (n == N + 1).sum(1).astype(float)
    ratio = c_n1.sum() / c_n.sum()
    # delta method on the replica totals
    m1, m0 = c_n1.mean(), c_n.mean()
    cov = np.cov(c_n1, c_n)
    var_ln = (cov[0, 0] / m1**2 + cov[1, 1] / m0**2 - 2 * cov[0, 1] / (m1 * m0)) / RG
    tol = 3.0 * math.sqrt(var_ln + s_mu**2)
    print(f"BAR beta mu {mu:.3f} +- {s_mu:.3f} from {sum(map(len, ins))} + {sum(map(len, dele))} trials; "
          f"GC at that mu: P(N+1)/P(N) = {ratio:.3f} (ln {math.log(ratio):+.3f}, tolerance {tol:.3f}), <N> {n.mean():.2f}")
    assert abs(math.log(ratio)) < tol
