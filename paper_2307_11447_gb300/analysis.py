"""Host-side analysis of nonequilibrium work samples and particle-number series.

* ``bar_mu``     -- chemical potential from insertion/deletion work samples through the
  Bennett acceptance ratio equation solved by Newton's method (SI Sec. S1, Eq. S2; the
  Crooks relation of Eq. S1 read as P_ins/P_del = exp(beta(Delta M - mu))).
* ``p_acc``      -- acceptance estimated from fixed-N work samples (Eq. 21).
* ``p_acc_gauss`` -- the Gaussian-work limit erfc(sqrt(beta <Delta H>)/2) (Sec. II.E).
* ``alpha2``     -- non-Gaussian parameter of a work distribution (Eq. 22).
* ``block_stats`` -- mean and standard error by block averaging, used for <N> and for
  chi_osmotic = V <(delta rho)^2> / <rho> = Var(N)/<N> at fixed V (Eq. 1).
* ``efficiency`` -- E_f = P_acc/N_f and E_f^t = P_acc/(N_eq + N_f) (Sec. II.A).
* ``jackknife``  -- delete-one-group jackknife estimate and standard error of any statistic
  of independent groups (Markov chains), for ratios such as Var(N)/<N> and for BAR.
* ``pooled_n_stats`` -- <N>, chi_osmotic = Var(N)/<N> of the pooled N series of many chains
  and the acceptance rate, each with its jackknife standard error over chains.
* ``time_to_se`` -- wall time a run needs to reach a target standard error of <N>.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special


def bar_mu(bdm_ins: np.ndarray, bdm_del: np.ndarray, iters: int = 200) -> float:
    """beta*mu solving sum_i f(beta(C + dM_i) - beta mu) = sum_j f(-(beta(C + dM_j) - beta mu))
    with f(x) = 1/(1+e^x) and C = ln(N_ins/N_del)/beta; inputs are beta*Delta M.  Both sides
    are taken as log-sums (ln f(x) = -softplus(x)), so the root stays defined when the two
    work distributions barely overlap; the left side grows and the right side falls with
    beta mu, so bisection finds the unique root."""
    a = np.asarray(bdm_ins, np.float64)
    b = np.asarray(bdm_del, np.float64)
    c = math.log(a.size / b.size)

    def g(mu):
        left = special.logsumexp(-np.logaddexp(0.0, c + a - mu))
        right = special.logsumexp(-np.logaddexp(0.0, -(c + b - mu)))
        return left - right

    lo = min(a.min(), b.min()) - 50.0
    hi = max(a.max(), b.max()) + 50.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if g(mid) < 0.0:
            lo = mid
        else:
            hi = mid
        if hi - lo < 1e-12:
            break
    return float(0.5 * (lo + hi))


def p_acc(bdm: np.ndarray, beta_mu: float, insertion: bool) -> float:
    """Eq. 21: <min(1, exp(-beta dM + beta mu))> for insertions and
    <min(1, exp(beta dM - beta mu))> for deletions."""
    x = np.asarray(bdm, np.float64) - beta_mu
    e = -x if insertion else x
    return float(np.mean(np.exp(np.minimum(e, 0.0))))


def p_acc_gauss(beta_mean_dH: float) -> float:
    """Gaussian work limit of the acceptance (Sec. II.E)."""
    return float(special.erfc(0.5 * math.sqrt(max(beta_mean_dH, 0.0))))


def alpha2(bdm: np.ndarray) -> float:
    """Eq. 22: <(beta dM)^4> / (3 <(beta dM)^2>^2) - 1 about the mean."""
    d = np.asarray(bdm, np.float64)
    d = d - d.mean()
    m2 = (d * d).mean()
    return float((d**4).mean() / (3.0 * m2 * m2) - 1.0)


def block_stats(series: np.ndarray, n_blocks: int = 20):
    """Mean of a correlated series and its standard error from n_blocks block means."""
    s = np.asarray(series, np.float64)
    nb = max(2, min(n_blocks, s.size))
    m = s.size // nb
    blocks = s[: m * nb].reshape(nb, m).mean(1)
    return float(s.mean()), float(blocks.std(ddof=1) / math.sqrt(nb))


def chi_osmotic(n_series: np.ndarray, n_blocks: int = 20):
    """chi = Var(N)/<N> at fixed volume (Eq. 1 with rho = N/V), with a block-average SE."""
    s = np.asarray(n_series, np.float64)
    mean = s.mean()
    chi = s.var() / mean if mean > 0 else float("nan")
    nb = max(2, min(n_blocks, s.size))
    m = s.size // nb
    vals = []
    for k in range(nb):
        b = s[k * m:(k + 1) * m]
        vals.append(((b - mean) ** 2).mean() / mean if mean > 0 else float("nan"))
    return float(chi), float(np.std(vals, ddof=1) / math.sqrt(nb))


def efficiency(pacc: float, n_f: int, n_eq: int = 0):
    return pacc / max(n_f, 1), pacc / max(n_eq + n_f, 1)


def ideal_pair_gas(lam: float, n_max: int = 4000):
    """Exact <N>, Var N of the ideal 1:1 pair gas, P(N) = lam^N/(N!)^2 / I_0(2 sqrt(lam))."""
    n = np.arange(n_max)
    logp = n * math.log(lam) - 2.0 * special.gammaln(n + 1)
    logp -= logp.max()
    p = np.exp(logp)
    p /= p.sum()
    mean = float((n * p).sum())
    var = float(((n - mean) ** 2 * p).sum())
    return mean, var


def jackknife(groups: list, stat):
    """stat(groups) and its delete-one-group jackknife standard error; groups are the
    independent units (chains), stat maps a list of groups to a number."""
    g = list(groups)
    k = len(g)
    full = float(stat(g))
    if k < 2:
        return full, float("nan")
    loo = np.array([stat(g[:i] + g[i + 1:]) for i in range(k)], np.float64)
    se = math.sqrt((k - 1) / k * ((loo - loo.mean()) ** 2).sum())
    return full, float(se)


def pooled_n_stats(chains: list):
    """chains: per-chain sufficient statistics dicts with keys count (samples of N),
    sum_n, sum_n2, trials, accepted.  Returns {mean_n, chi, acc} each as (value, se): the
    pooled <N>, chi = Var(N)/<N> (Eq. 1 at fixed V, variance of the pooled series), and
    the fraction of trials accepted, with jackknife errors over chains."""
    def mean_n(g):
        return sum(c["sum_n"] for c in g) / sum(c["count"] for c in g)

    def chi(g):
        n = sum(c["count"] for c in g)
        m = sum(c["sum_n"] for c in g) / n
        return (sum(c["sum_n2"] for c in g) / n - m * m) / m

    def acc(g):
        return sum(c["accepted"] for c in g) / max(sum(c["trials"] for c in g), 1)

    return {"mean_n": jackknife(chains, mean_n), "chi": jackknife(chains, chi), "acc": jackknife(chains, acc)}


def chain_sums(move, accepted, status, n_after, beta_dM, beta_mu: float, burn: int = 0) -> dict:
    """Sufficient statistics of one chain's trials after the first `burn`: the N series
    (count, sum_n, sum_n2), the accepted fraction (trials, accepted) and the sums of the
    Eq. 21 acceptance estimate min(1, e^x) per move type at beta_mu (x = -beta dM + beta mu
    for insertions, beta dM - beta mu for deletions; trials with status != 0 count as 0)."""
    mv = np.asarray(move)[burn:]
    ac = np.asarray(accepted)[burn:]
    stt = np.asarray(status)[burn:]
    n = np.asarray(n_after, np.float64)[burn:]
    bdm = np.asarray(beta_dM, np.float64)[burn:]
    ok = stt == 0
    x = np.where(mv == 1, -(bdm - beta_mu), bdm - beta_mu)
    p = np.where(ok & np.isfinite(x), np.exp(np.minimum(np.where(np.isfinite(x), x, 0.0), 0.0)), 0.0)
    ins = mv == 1
    return {"count": int(n.size), "sum_n": float(n.sum()), "sum_n2": float((n * n).sum()),
            "trials": int(ac.size), "accepted": int(ac.sum()),
            "n_ins": int(ins.sum()), "p21_ins": float(p[ins].sum()),
            "n_del": int((~ins).sum()), "p21_del": float(p[~ins].sum()),
            "bdm_ins": float(bdm[ins & ok].sum()), "bdm_del": float(bdm[~ins & ok].sum()),
            "ok_ins": int((ins & ok).sum()), "ok_del": int((~ins & ok).sum())}


def eq21_acceptance(chains: list):
    """Eq. 21 acceptance of a trial (insertions and deletions equally likely) pooled over
    chains' sums, with its jackknife error"""
    def f(g):
        pi = sum(c["p21_ins"] for c in g) / max(sum(c["n_ins"] for c in g), 1)
        pd = sum(c["p21_del"] for c in g) / max(sum(c["n_del"] for c in g), 1)
        return 0.5 * (pi + pd)

    return jackknife(chains, f)


def mean_work(chains: list, insertion: bool):
    """mean beta Delta M of the insertions (or deletions) with status 0, jackknife error"""
    k, n = ("bdm_ins", "ok_ins") if insertion else ("bdm_del", "ok_del")
    return jackknife(chains, lambda g: sum(c[k] for c in g) / max(sum(c[n] for c in g), 1))


def time_to_se(se: float, seconds: float, target_se: float) -> float:
    """seconds a run needs to bring the standard error of <N> from se (measured after
    `seconds`) to target_se, with SE falling as 1/sqrt(time)"""
    return float(seconds * (se / target_se) ** 2)
