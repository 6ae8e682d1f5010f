"""Writes tests/golden/config_stats.json from the FP64 oracle alone (test infrastructure).

Stages (each adds its section to the JSON, keeping the others):

* ``calibrate`` -- fixed-N insertion and deletion work of the 250- and 4000-ion
  electrolytes at their N (Sec. II.E), and the BAR estimate of beta mu from it (SI Sec. S1,
  Eq. S2).  The grand-canonical statistics run at these values (copied into
  ``workloads.CONFIGS``).
* ``stats <name>`` -- the oracle side of the per-configuration statistics of
  ``tests/config_protocols.py``: per-chain sufficient statistics of the N series and the
  acceptances (``analysis.chain_sums``), and for fixed-N runs every trial's beta Delta M
  and move.

Each chain runs in its own spawned process; nothing here touches the GPU library.
Usage: python tests/golden/make_config_stats.py calibrate | stats lj250 [workers]
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "config_stats.json")


def _run_chain(job):
    name, kind, k, prot, beta_mu = job
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from config_protocols import chain_inputs, config_of

    from oracle import oracle as orc

    seed = prot["seed_oracle"] + k
    inp = chain_inputs(name, k, seed)
    cfg = config_of(name)
    cfg.update(L=inp["L"], n_pairs=inp["n_pairs"], cap_pairs=inp["cap_pairs"], n_water=inp["n_water"],
               seed=seed, replica=0, use_cells=1, beta_mu=beta_mu, no_accept=int(kind == "fixed_n"))
    p = orc.make_params(cfg)
    st = orc.State(p, inp["x"], None, inp["n_pairs"], inp["cap_pairs"])
    orc.init_velocities(p, st)
    t0 = time.time()
    orc.md(p, st, prot["equil"])
    rec = orc.run_cycles(p, st, prot["trials"], prot["n_eq"])
    from paper_2307_11447_gb300 import analysis as an

    out = {"k": k, "rep": inp.get("rep", 0), "n0": inp["n_pairs"], "seconds": time.time() - t0,
           "sums": an.chain_sums(rec["move"], rec["accepted"], rec["status"], rec["n_after"], rec["beta_dM"],
                                 beta_mu, prot.get("burn", 0))}
    if kind == "fixed_n":
        out.update(move=rec["move"].tolist(), status=rec["status"].tolist(),
                   beta_dM=[float(v) for v in rec["beta_dM"]])
    return out


def _pool_map(jobs, workers):
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_run_chain, jobs, chunksize=1)


def _load():
    return json.load(open(OUT)) if os.path.exists(OUT) else {}


def _save(d):
    tmp = OUT + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, OUT)


def calibrate(workers):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from config_protocols import CALIBRATE

    from paper_2307_11447_gb300 import analysis as an

    d = _load()
    d.setdefault("calibrate", {})
    for name, prot in CALIBRATE.items():
        res = _pool_map([(name, "fixed_n", k, prot, 0.0) for k in range(prot["chains_oracle"])], workers)
        ins = [np.array(r["beta_dM"])[(np.array(r["move"]) == 1) & (np.array(r["status"]) == 0)] for r in res]
        dele = [np.array(r["beta_dM"])[(np.array(r["move"]) == 0) & (np.array(r["status"]) == 0)] for r in res]
        groups = list(zip(ins, dele))
        mu, se = an.jackknife(groups, lambda g: an.bar_mu(np.concatenate([a for a, _ in g]),
                                                          np.concatenate([b for _, b in g])))
        d["calibrate"][name] = {"protocol": prot, "bar_beta_mu": mu, "bar_beta_mu_se": se,
                                "n_ins": int(sum(map(len, ins))), "n_del": int(sum(map(len, dele))),
                                "chains": [{k: r[k] for k in ("k", "move", "status", "beta_dM")} for r in res]}
        print(f"{name}: BAR beta mu {mu:.3f} +- {se:.3f} ({d['calibrate'][name]['n_ins']} ins, "
              f"{d['calibrate'][name]['n_del']} del)", flush=True)
        _save(d)


def stats(name, workers):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from config_protocols import STATS, config_of

    prot = STATS[name]
    beta_mu = config_of(name)["beta_mu"]
    n_chains = prot["chains_oracle"] * len(prot.get("replicas", (0,)))
    t0 = time.time()
    res = _pool_map([(name, prot["kind"], k, prot, beta_mu) for k in range(n_chains)], workers)
    d = _load()
    d.setdefault("stats", {})
    d["stats"][name] = {"protocol": prot, "beta_mu": beta_mu, "chains": res, "wall_s": time.time() - t0}
    _save(d)
    print(f"{name}: {n_chains} oracle chains in {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    if sys.argv[1] == "calibrate":
        calibrate(int(sys.argv[2]) if len(sys.argv) > 2 else os.cpu_count())
    else:
        stats(sys.argv[2], int(sys.argv[3]) if len(sys.argv) > 3 else os.cpu_count())
