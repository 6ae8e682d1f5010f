"""Statistical parity of the GPU engine with the FP64 oracle on the configurations.

For each configuration the GPU runs the sampling protocol of ``tests/config_protocols.py``
on its own seeded chains; the oracle ran the same protocol offline on other seeds
(``tests/golden/make_config_stats.py``, stored in ``tests/golden/config_stats.json``).
Compared, each within two combined standard errors (jackknife over independent chains on
both sides; the z-scores are printed):

* grand-canonical runs (250- and 4000-ion electrolytes at their BAR beta mu, a subset of
  the batched replicas): <N>, chi_osmotic = Var(N)/<N> of the pooled N series (Eq. 1 at
  fixed V), the fraction of trials accepted (Eqs. 6, 8), and the acceptance estimated from
  the same trials' work (Eq. 21);
* fixed-N runs (aqueous NaCl, where exchanges are rare at N_f = 1000): the mean beta
  Delta M of insertions and of deletions (Sec. II.E).  The two work distributions do not
  overlap, so the Eq. 21 acceptance at the working beta mu only counts moves (insertion
  exponents far above zero, deletion exponents far below); it is printed, not compared.

The chains of both sides are exact samples of the same Markov process, so each z-score
is a standard normal draw when the two implementations agree; the seeds are fixed, so a
run is reproducible.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2307_11447_gb300 import analysis as an
from paper_2307_11447_gb300 import lib as h4d

from .config_protocols import STATS, chain_inputs, config_of

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "config_stats.json")
Z_MAX = 2.0


def _golden(name):
    d = json.load(open(GOLDEN)) if os.path.exists(GOLDEN) else {}
    if name not in d.get("stats", {}):
        pytest.skip(f"no oracle statistics for {name} in {os.path.basename(GOLDEN)}")
    g = d["stats"][name]
    assert g["protocol"] == json.loads(json.dumps(STATS[name])), "oracle statistics are stale for this protocol"
    assert g["beta_mu"] == config_of(name)["beta_mu"]
    return g["chains"]


def _gpu_chains(name):
    prot = STATS[name]
    cfg = config_of(name)
    n_chains = prot["chains_gpu"] * len(prot.get("replicas", (0,)))
    inputs = [chain_inputs(name, k, prot["seed_gpu"] + k) for k in range(n_chains)]
    reps = [dict(L=i["L"], n_pairs=i["n_pairs"], cap_pairs=i["cap_pairs"], x=i["x"], n_water=i["n_water"])
            for i in inputs]
    ctx = h4d.Context(h4d.make_params(cfg), reps, seed=prot["seed_gpu"])
    ctx.h4d_run_md(prot["equil"])
    if prot["kind"] == "fixed_n":
        ctx.h4d_set_no_accept(1)
    recs = [[] for _ in range(n_chains)]
    done = 0
    while done < prot["trials"]:
        k = min(1000, prot["trials"] - done)
        ctx.h4d_run_trials(k, prot["n_eq"])
        for r in range(n_chains):
            recs[r].append(ctx.h4d_get_work(r, k))
        done += k
    out = []
    for r in range(n_chains):
        rec = np.concatenate(recs[r])
        assert rec.size == prot["trials"]
        out.append({"k": r, "rep": inputs[r].get("rep", 0), "n0": inputs[r]["n_pairs"],
                    "sums": an.chain_sums(rec["move"], rec["accepted"], rec["status"], rec["n_after"],
                                          rec["beta_dM"], cfg["beta_mu"], prot.get("burn", 0))})
    ctx.close()
    return out


def _z(a, b):
    (va, sa), (vb, sb) = a, b
    se = math.sqrt(sa * sa + sb * sb)
    return abs(va - vb) / se if se > 0 else (0.0 if va == vb else float("inf"))


def _compare(name, stats):
    orc_chains = _golden(name)
    gpu_chains = _gpu_chains(name)
    lines, worst = [], 0.0
    for label, f in stats.items():
        g, o = f(gpu_chains), f(orc_chains)
        z = _z(g, o)
        worst = max(worst, z)
        lines.append(f"{label}: gpu {g[0]:.5g} +- {g[1]:.2g}, oracle {o[0]:.5g} +- {o[1]:.2g}, z = {z:.2f}")
    print(f"\n[{name}] " + "; ".join(lines))
    return worst, gpu_chains, orc_chains


def _gc_stats(shifted=False):
    def sums(g):
        return [c["sums"] for c in g]

    def mean_n(g):
        return an.pooled_n_stats(sums(g))["mean_n"]

    def chi(g):
        return an.pooled_n_stats(sums(g))["chi"]

    def acc(g):
        return an.pooled_n_stats(sums(g))["acc"]

    def eq21(g):
        return an.eq21_acceptance(sums(g))

    if shifted:
        # replicas of different sizes: <N - N0> pooled, chi averaged over replicas
        def mean_n(g):  # noqa: F811
            def f(gg):
                return sum(c["sums"]["sum_n"] - c["n0"] * c["sums"]["count"] for c in gg) / sum(c["sums"]["count"] for c in gg)
            return an.jackknife(g, f)

        def chi(g):  # noqa: F811
            def f(gg):
                by = {}
                for c in gg:
                    by.setdefault(c["rep"], []).append(c["sums"])
                vals = []
                for s in by.values():
                    n = sum(x["count"] for x in s)
                    m = sum(x["sum_n"] for x in s) / n
                    vals.append((sum(x["sum_n2"] for x in s) / n - m * m) / m)
                return float(np.mean(vals))
            return an.jackknife(g, f)

    return {"<N>" if not shifted else "<N - N0>": mean_n, "chi": chi, "acceptance": acc, "acceptance (Eq. 21)": eq21}


def test_config_stats_lj250():
    worst, _, _ = _compare("lj250", _gc_stats())
    assert worst < Z_MAX


def test_config_stats_lj4000():
    worst, _, _ = _compare("lj4000", _gc_stats())
    assert worst < Z_MAX


def test_config_stats_batched_subset():
    worst, _, _ = _compare("batched_subset", _gc_stats(shifted=True))
    assert worst < Z_MAX


def test_config_stats_nacl_aq():
    def eq21(g):
        return an.eq21_acceptance([c["sums"] for c in g])

    stats = {"mean beta dM ins": lambda g: an.mean_work([c["sums"] for c in g], True),
             "mean beta dM del": lambda g: an.mean_work([c["sums"] for c in g], False)}
    worst, gpu_chains, orc_chains = _compare("nacl_aq", stats)
    # at the working beta mu (-60) the Eq. 21 estimate is saturated: insertion exponents lie
    # far above zero and deletion exponents far below, so it counts moves, not physics
    print(f"acceptance (Eq. 21) at beta mu {config_of('nacl_aq')['beta_mu']}: gpu {eq21(gpu_chains)[0]:.4f}, "
          f"oracle {eq21(orc_chains)[0]:.4f}")
    assert worst < Z_MAX
