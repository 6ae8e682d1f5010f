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
