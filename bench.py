"""Benchmark of the H4D grand-canonical hot path on one or more GB300s.

Workload (default): the 4000-ion LJ electrolyte at density 0.3 (L = 23.71 sigma), NEMD
protocol of 500 steps, 1000 equilibrium MD steps between trials, split into independent
Markov chains (one per replica; 304 chains = 2 per SM).  One benchmark step is one
grand-canonical cycle of every chain: 1000 equilibrium MD steps, trial setup, 500 NEMD
steps with the 4D pair forces, FP64 work, Metropolis and commit -- all in one persistent
launch.  Inputs are generated from fixed seeds and equilibrated for 1000 MD steps before
timing.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "accepted salt-pair exchanges/s & 4D atom-steps/s, plain vs batched/learned"
FLOPS_PER_PAIR = 55  # FP32 operations per unordered pair inside the cut-off (FMA = 2, MUFU = 1)
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="h4d", choices=["h4d", "reference"])
    ap.add_argument("--chains", type=int, default=None, help="chains per GPU (default: 304 LJ, 152 aqueous)")
    ap.add_argument("--sequential", type=int, default=0,
                    help="batched workload: also time this many replicas run one at a time (alone on the GPU)")
    ap.add_argument("--workload", default="lj4000")
    ap.add_argument("--cpu-cores", type=int, default=None,
                    help="host processes for the oracle legs (default: every host core)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--equil", type=int, default=1000)
    ap.add_argument("--n-eq", type=int, default=None, help="override equilibrium steps per cycle (profiling)")
    ap.add_argument("--n-f", type=int, default=None, help="override NEMD steps per trial (profiling)")
    ap.add_argument("--tune-iters", type=int, default=20, help="force passes per autotuner candidate")
    ap.add_argument("--skin", type=float, default=None, help="Verlet skin (default: the workload's)")
    ap.add_argument("--skin-outer", type=float, default=None, help="outer-list skin (default: the workload's)")
    # learned-proposal workload (nacl_learned): records, training and calibration before timing
    ap.add_argument("--records", type=int, default=100000, help="training records to generate (nacl_learned)")
    ap.add_argument("--record-nf", type=int, default=50, help="NEMD steps of the record-generating trials")
    ap.add_argument("--cell-len", type=float, default=1.4, help="proposal grid cell edge (A)")
    ap.add_argument("--train-steps", type=int, default=2000)
    ap.add_argument("--calib-cycles", type=int, default=2, help="fixed-N production cycles per proposal")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_over_ranks(t, units, dist=None, device="cuda"):
    """Whole-job figures of a timed region: the MAX of the ranks' times and the SUM of
    their units (rank-local values when there is one rank)."""
    units = np.asarray(units, np.float64)
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(t), units
    import torch

    tt = torch.tensor([float(t)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    tv = torch.tensor(units, dtype=torch.float64, device=device)
    dist.all_reduce(tv)
    return float(tt.item()), tv.cpu().numpy()


def workload(name, chains, rank):
    from paper_2307_11447_gb300 import workloads as wl

    if name == "batched256":
        cfg, reps = wl.batched_system(256, seed=7 + rank)
        if ARGS.n_eq is not None:
            cfg["n_eq"] = ARGS.n_eq
        if ARGS.n_f is not None:
            cfg["n_f"] = ARGS.n_f
        return cfg, reps
    cfg = dict(wl.CONFIGS["nacl_aq" if name in ("nacl_learned", "nacl_water") else name])
    if name == "nacl_water":
        cfg["exchange"] = "water"  # one rigid water per trial; the NaCl pairs stay
    if ARGS.skin is not None:
        cfg["skin"] = ARGS.skin
    if ARGS.skin_outer is not None:
        cfg["skin_outer"] = ARGS.skin_outer
    if ARGS.n_eq is not None:
        cfg["n_eq"] = ARGS.n_eq
    if ARGS.n_f is not None:
        cfg["n_f"] = ARGS.n_f
    if name in ("nacl_aq", "nacl_learned", "nacl_water"):
        reps = []
        for c in range(chains):
            x = wl.aqueous_positions(cfg["n_water"], cfg["n_pairs"], cfg["L"], 2000 * (rank + 1) + c)
            reps.append(dict(L=cfg["L"], n_pairs=cfg["n_pairs"], cap_pairs=cfg["cap_pairs"], x=x,
                             n_water=cfg["n_water"],
                             cap_water=cfg["n_water"] + (32 if name == "nacl_water" else 0)))
        return cfg, reps
    reps = []
    for c in range(chains):
        seed = 1000 * (rank + 1) + c
        x = wl.lj_positions(cfg["n_pairs"], cfg["L"], seed)
        reps.append(dict(L=cfg["L"], n_pairs=cfg["n_pairs"], cap_pairs=cfg["cap_pairs"], x=x))
    return cfg, reps


def src_hash():
    """Hash of the engine kernel sources (the traffic figure is tied to them)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2307_11447_gb300", "csrc")
    for f in ("h4d_engine.cu", "h4d_engine.cuh"):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def pair_pass_roofline(pairs, tune, tpa_hist, phase, achieved, peak):
    """The force pass by itself: (1) launched alone by the autotuner (every chain's pass at
    once, each timed by its group's device global timer; the pass time of the lane count
    most chains use), (2) inside the persistent kernel (its share of the launch time from
    the phase timers).  Same algorithmic count as the kernel roofline: 55 flop per pair
    inside the cut-off, each unordered pair once."""
    t_most = max(tpa_hist.items(), key=lambda kv: kv[1])[0]
    us = tune[t_most][0] / 1e3
    alone = pairs * FLOPS_PER_PAIR / (us * 1e-6) / 1e12
    inside = achieved / phase["force"] if phase.get("force") else None
    return {"alone": {"threads_per_atom": int(t_most), "us_per_pass": us, "achieved": alone, "frac": alone / peak},
            "inside_engine": {"achieved": inside, "frac": inside / peak if inside else None},
            "unit": "TFLOP/s"}


def default_launch(args, cfg):
    """True for the launch the committed traffic figure was scaled to: the 4000-ion
    workload with its own chain count, protocol and skins"""
    from paper_2307_11447_gb300 import workloads as wl

    ref = wl.CONFIGS["lj4000"]
    return (args.workload == "lj4000" and args.chains == ref["chains"] and cfg["n_eq"] == ref["n_eq"]
            and cfg["n_f"] == ref["n_f"] and cfg["skin"] == ref["skin"] and cfg["skin_outer"] == ref["skin_outer"])


def traffic_from_profile(cfg):
    """DRAM bytes per launch of the engine kernel from the committed ncu summary, or None
    when the kernel source or the list skins changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        t = json.load(open(p))
    except Exception:
        return None
    if t.get("src_sha") != src_hash() or t.get("skins") != [cfg["skin"], cfg["skin_outer"]]:
        return None
    return t.get("dram_bytes_per_launch")


class ClockSampler:
    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [l.strip().split(",") for l in open(self.f.name) if l.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for k, n in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2307_11447_gb300 import analysis as an
    from paper_2307_11447_gb300 import lib as h4d

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    cfg, reps = workload(args.workload, args.chains, rank)
    params = h4d.make_params(cfg)
    with torch.cuda.stream(stream):
        ctx = h4d.Context(params, reps, seed=12345 + rank, stream=stream.cuda_stream)
    n_eq, n_f = cfg["n_eq"], cfg["n_f"]
    sm_count, _, _ = h4d.h4d_device_info()
    fp32_probe_tflops, _ = h4d.h4d_measure_fp32_peak()
    # equilibrate the random starts (untimed), autotune the force pass, then warm up
    ctx.h4d_run_md(args.equil)
    learned = None
    if args.workload == "nacl_learned":
        learned = learned_setup(ctx, cfg, args, stream)
    water_cal = None
    if args.workload == "nacl_water":
        water_cal = water_calibration(ctx, cfg, args)
    tune = ctx.h4d_autotune(args.tune_iters)
    tpa_hist = {}
    for r in range(ctx.R):
        t = ctx.h4d_get_counts(r)["threads_per_atom"]
        tpa_hist[t] = tpa_hist.get(t, 0) + 1
    for _ in range(args.warmup):
        ctx.h4d_run_trials(1, n_eq)
    torch.cuda.synchronize()
    c0 = [ctx.h4d_get_counts(r) for r in range(ctx.R)]
    pairs0 = ctx.h4d_count_pairs()

    def barrier():
        if world > 1:
            dist.barrier()

    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for k in range(args.steps):
        ctx.h4d_run_trials(1, n_eq)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    per_launch_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    t_ms = sum(per_launch_ms)
    c1 = [ctx.h4d_get_counts(r) for r in range(ctx.R)]
    pairs1 = ctx.h4d_count_pairs()
    # units this rank processed
    atom_steps = 0.0
    nemd_atom_steps = 0.0
    accepted = 0
    for r, (a, b) in enumerate(zip(c0, c1)):
        mean_n = (b["sum_n"] - a["sum_n"]) / max(b["cycles"] - a["cycles"], 1)  # exchanged units
        if args.workload == "nacl_water":  # the waters vary, the ion pairs stay
            n_atoms = 3.0 * mean_n + 2.0 * reps[r]["n_pairs"]
        else:
            n_atoms = 2.0 * mean_n + 3.0 * reps[r].get("n_water", 0)
        atom_steps += n_atoms * (n_eq + n_f) * args.steps
        nemd_atom_steps += n_atoms * n_f * args.steps
        accepted += (b["accepted_ins"] + b["accepted_del"]) - (a["accepted_ins"] + a["accepted_del"])
    builds = sum(b["nbr_builds"] - a["nbr_builds"] for a, b in zip(c0, c1))
    t_nemd = sum(b["t_nemd_ns"] - a["t_nemd_ns"] for a, b in zip(c0, c1)) / 1e9
    t_md = sum(b["t_md_ns"] - a["t_md_ns"] for a, b in zip(c0, c1)) / 1e9
    nemd_frac = t_nemd / max(t_nemd + t_md, 1e-30)
    t_all = max(t_nemd + t_md, 1e-30)
    # "build" is every list pass; "verlet_filter" is the part of it that filters the Verlet
    # rows from the outer rows (each full build ends with one, refreshes are only that)
    phase = {k: sum(b[f"t_{k}_ns"] - a[f"t_{k}_ns"] for a, b in zip(c0, c1)) / 1e9 / t_all
             for k in ("build", "filter", "force", "energy")}
    phase["verlet_filter"] = phase.pop("filter")
    refreshes = sum(b["nbr_refreshes"] - a["nbr_refreshes"] for a, b in zip(c0, c1))
    # each chain's own device time (its thread 0's timers) against the launch time: the
    # launch ends with its slowest chain
    chain_ms = np.array([(b["t_nemd_ns"] - a["t_nemd_ns"] + b["t_md_ns"] - a["t_md_ns"]) / 1e6
                         for a, b in zip(c0, c1)])
    tmax, tot = reduce_over_ranks(t_ms, [atom_steps, nemd_atom_steps, accepted], dist if world > 1 else None)
    secs = tmax / 1e3
    value = tot[0] / secs
    # roofline of the engine kernel: algorithmic FP32 work of the pair term
    pairs = 0.5 * (pairs0 + pairs1)
    force_evals = n_eq + n_f + 2
    flops_per_launch = pairs * force_evals * FLOPS_PER_PAIR
    avg_launch_s = (t_ms / args.steps) / 1e3
    achieved = flops_per_launch / avg_launch_s / 1e12
    sm_mhz = clk.get("sm_max_mhz") or 2070.0
    nominal = sm_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    # the roofline denominator is the FP32 throughput measured on this GPU (FMA chains on
    # every SM, timed with CUDA events); the nominal lanes x clock figure is kept beside it
    peak = fp32_probe_tflops
    # grand-canonical statistics of the timed cycles (jackknife over chains) and trials
    # that ended with non-finite work or an overflowing neighbour row (status 3)
    status3 = 0
    sums = []
    for r in range(ctx.R):
        rec = ctx.h4d_get_work(r, args.steps)
        status3 += int((rec["status"] == 3).sum())
        sums.append(an.chain_sums(rec["move"], rec["accepted"], rec["status"], rec["n_after"], rec["beta_dM"],
                                  cfg["beta_mu"]))
    gc = an.pooled_n_stats(sums)
    eq21 = an.eq21_acceptance(sums)

    if learned is not None:
        learned["uniform_arm"] = uniform_arm(ctx, reps, args, n_eq, n_f, stream)
        ctx.h4d_proposal(h4d.H4D_PROPOSAL_LEARNED, args.cell_len, 0.1, 0)
    seq = None
    if args.sequential and args.workload == "batched256":
        seq = sequential_baseline(reps, cfg, args.sequential, n_eq)
    equal_se = None
    # (no accepted exchange: <N> has no spread, so there is no common error to reach)
    if rank == 0 and args.workload in ("lj4000", "nacl_aq") and gc["mean_n"][1] > 0:
        equal_se = plain_at_equal_se(reps[0], cfg, n_eq, stream, secs, gc["mean_n"][1],
                                     int(sum(x["trials"] for x in sums)), accepted)
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(ctx, reps, args, n_eq, n_f, stream, world, dist if world > 1 else None)

    if rank == 0:
        out = {
            "metric": METRIC,
            "value": value,
            "unit": "atom-steps/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": tmax / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32 pair forces, f64 work/energies",
            "data": "synthetic (seeded uniform positions, equilibrated 1000 MD steps)",
            "config": workload_config(args, cfg, reps, n_f, n_eq, world),
            "nemd_4d_atom_steps_per_s": tot[1] / (secs * nemd_frac) if nemd_frac > 0 else None,
            "accepted_exchanges_per_s": tot[2] / secs,
            "accepted": int(tot[2]),
            "md_steps_per_nbr_build": (n_eq + n_f) * args.steps * len(c0) / max(builds, 1),
            "md_steps_per_verlet_refresh": (n_eq + n_f) * args.steps * len(c0) / max(builds + refreshes, 1),
            "nemd_time_fraction": nemd_frac,
            "phase_time_fraction": phase,
            "chain_time_ms": {"min": float(chain_ms.min()), "mean": float(chain_ms.mean()),
                              "max": float(chain_ms.max()), "cv": float(chain_ms.std() / chain_ms.mean()),
                              "launch_over_mean_chain": float(t_ms / chain_ms.mean())},
            "autotuned_threads_per_atom": {str(k): v for k, v in sorted(tpa_hist.items())},
            "autotune_us_per_force_pass_and_build": {str(k): [round(a / 1e3, 1), round(b / 1e3, 1)] for k, (a, b) in tune.items()},
            "trials": int(args.chains * world * args.steps),
            "gpu_launches": args.steps,
            "clocks": clk,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         # the ncu figure belongs to the default workload's launch (and source)
                         "traffic": traffic_from_profile(cfg) if default_launch(args, cfg) else None,
                         "kernel": "cycles_kernel (persistent: list build, 4D pair forces, VV, FP64 work, Metropolis)",
                         "peak_basis": f"measured FP32 FMA-chain throughput on this GPU ({sm_count} SMs); "
                                       f"nominal {sm_count} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_mhz:.0f} MHz = "
                                       f"{nominal:.1f} TFLOP/s",
                         "frac_of_nominal": achieved / nominal,
                         "pairs_in_cutoff": pairs, "flops_per_pair": FLOPS_PER_PAIR,
                         "pair_pass": pair_pass_roofline(pairs, tune, tpa_hist, phase, achieved, peak)},
            "grand_canonical": {
                "beta_mu": cfg["beta_mu"], "trials": int(sum(x["trials"] for x in sums)),
                "mean_n": gc["mean_n"], "chi_osmotic": gc["chi"], "acceptance": gc["acc"],
                "acceptance_eq21": eq21, "se_method": "jackknife over chains ([value, se])",
                "status3_trials": status3},
            "e2e": e2e,
        }
        if learned is not None:
            out["learned_proposal"] = learned
        if water_cal is not None:
            out["water_exchange_calibration"] = water_cal
        if equal_se is not None:
            out["grand_canonical"]["equal_se_plain_vs_batched"] = equal_se
        out["long_range_coulomb"] = ewald_timing()
        if seq is not None:
            out["sequential_one_replica_at_a_time"] = seq
            out["batched_over_sequential"] = value / seq["value"]
        if rank == 0 and os.environ.get("H4D_BENCH_CPU", "1") == "1":
            out["cpu_baseline"] = cpu_baseline(args.workload, sample_steps=60, cores=args.cpu_cores)
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def workload_config(args, cfg, reps, n_f, n_eq, world):
    if args.workload == "nacl_learned":
        return {"workload": f"learned proposal on aqueous NaCl: {cfg['n_water']} rigid waters + {cfg['n_pairs']} NaCl, "
                            f"L={cfg['L']} A, N_f={n_f}, N_eq={n_eq}, {len(reps)} chains/GPU, "
                            f"{args.cell_len} A proposal cells", "chains_per_gpu": len(reps),
                "n_f": n_f, "n_eq": n_eq, "parallelism": f"replicas x{world}",
                "l2": "state > L2; no flush needed"}
    if args.workload == "nacl_water":
        return {"workload": f"water exchange in aqueous NaCl: {cfg['n_water']} rigid waters (capacity +32) + "
                            f"{cfg['n_pairs']} NaCl, L={cfg['L']} A, N_f={n_f}, N_eq={n_eq}, {len(reps)} chains/GPU, "
                            f"beta mu of the water by BAR", "chains_per_gpu": len(reps),
                "n_f": n_f, "n_eq": n_eq, "parallelism": f"replicas x{world}",
                "l2": "state > L2; no flush needed"}
    if args.workload == "nacl_aq":
        return {"workload": f"aqueous NaCl: {cfg['n_water']} rigid waters + {cfg['n_pairs']} NaCl, L={cfg['L']} A, "
                            f"N_f={n_f}, N_eq={n_eq}, {len(reps)} chains/GPU", "chains_per_gpu": len(reps),
                "n_f": n_f, "n_eq": n_eq, "parallelism": f"replicas x{world}",
                "l2": "state > L2; no flush needed"}
    if args.workload == "batched256":
        ns = [2 * r["n_pairs"] for r in reps]
        return {"workload": f"batched: {len(reps)} LJ-electrolyte replicas, ions {min(ns)}-{max(ns)}, "
                            f"rho 0.1-0.4, N_f={n_f}, N_eq={n_eq}", "replicas_per_gpu": len(reps),
                "n_f": n_f, "n_eq": n_eq, "parallelism": f"replicas x{world}",
                "l2": "state smaller than L2 after warm-up; every step re-reads it (persistent launch)"}
    rho = cfg["n_ions"] / cfg["L"] ** 3
    # per atom: position, velocity pair, force, two reference positions, save copies, and
    # the Verlet and outer rows
    state_gb = args.chains * cfg["n_ions"] * 1.0e-9 * (16 * 6 + 2 * 256)
    l2 = (f"state > L2 (about {state_gb:.1f} GB per GPU); no flush needed" if state_gb > 0.129 else
          f"state about {state_gb * 1e3:.0f} MB per GPU, inside L2 after warm-up; every step re-reads it "
          f"(persistent launch)")
    return {"workload": f"LJ electrolyte {cfg['n_ions']} ions rho={rho:.1f} (L={cfg['L']:.3f}), N_f={n_f}, N_eq={n_eq}, "
                        f"{args.chains} chains/GPU", "chains_per_gpu": args.chains, "ions": cfg["n_ions"],
            "n_f": n_f, "n_eq": n_eq, "parallelism": f"replicas x{world}", "l2": l2}


# ---------------------------------------------------------------------------------------
# learned insertion-site proposal on aqueous NaCl
# ---------------------------------------------------------------------------------------
def _balanced_mu(x_ins, x_del):
    """beta mu at which insertions and deletions of a fixed-N sample (taken at beta mu = 0)
    are accepted equally often: the equilibrium condition of Eqs. 3-8 at that N"""
    f = lambda m: np.exp(np.minimum(x_ins + m, 0)).mean() - np.exp(np.minimum(x_del - m, 0)).mean()
    lo, hi = -1000.0, 1000.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if f(mid) < 0 else (lo, mid)
    return 0.5 * (lo + hi)


def _initial_weights(seed):
    """seeded Gaussian start of the 96-64-64-2 network (std 1/sqrt(fan-in), zero biases),
    flat layout W1, b1, W2, b2, W3, b3"""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, 96 ** -0.5, 96 * 64), np.zeros(64), rng.normal(0, 64 ** -0.5, 64 * 64), np.zeros(64),
             rng.normal(0, 64 ** -0.5, 64 * 2), np.zeros(2)]
    return np.concatenate(parts)


def _fixed_n_sample(ctx, cycles):
    """insertion and deletion exponents of every chain's fixed-N trials, per chain"""
    groups = []
    ctx.h4d_run_trials(cycles, 10)
    for r in range(ctx.R):
        w = ctx.h4d_get_work(r, cycles)
        w = w[w["status"] == 0]
        ins = w["move"] == 1
        groups.append((w["x_acc"][ins], w["x_acc"][~ins]))
    return groups


def _flat(groups):
    return np.concatenate([a for a, _ in groups]), np.concatenate([b for _, b in groups])


def learned_setup(ctx, cfg, args, stream):
    """Untimed preparation of the learned proposal: fixed-N uniform trials with a short
    protocol generate the training records, the network trains on the GPU, and a fixed-N
    sample of production trials of each proposal gives the balancing beta mu and the
    insertion and deletion exponents of both (taken at beta mu = 0)."""
    import torch

    from paper_2307_11447_gb300 import lib as h4d

    R = ctx.R
    n_f = cfg["n_f"]
    per_rep = int(math.ceil(args.records / R)) + 4  # a few trials end with non-finite work
    ctx.h4d_set_no_accept(1)
    ctx.h4d_set_mu(0.0)
    ctx.h4d_set_protocol(args.record_nf, cfg["w_max"], cfg["dt"], cfg.get("kappa_sr", 0.0), 0)
    ctx.h4d_proposal(h4d.H4D_PROPOSAL_UNIFORM, args.cell_len, 0.1, per_rep)
    t0 = time.perf_counter()
    done = 0
    while done < per_rep:
        k = min(50, per_rep - done)
        ctx.h4d_run_trials(k, 10)
        done += k
    torch.cuda.synchronize()
    t_rec = time.perf_counter() - t0
    ys, sts = [], []
    for r in range(R):
        _, y, _, s = ctx.h4d_proposal_records(r)
        ys.append(y)
        sts.append(s)
    ys, sts = np.concatenate(ys), np.concatenate(sts)
    ok = (sts == 0) & np.isfinite(ys)  # training uses the same records
    if not ok.any():
        raise RuntimeError("no usable training records")
    y0 = float(np.median(ys[ok]))
    ctx.h4d_proposal_set_weights(_initial_weights(1))
    t0 = time.perf_counter()
    loss0 = ctx.h4d_train_proposal(1, 4096, 0.0, y0, seed=1)
    loss = ctx.h4d_train_proposal(args.train_steps, 4096, 2e-3, y0, seed=2)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    # production protocol, fixed N: both proposals from the same ensemble
    ctx.h4d_set_protocol(n_f, cfg["w_max"], cfg["dt"], cfg.get("kappa_sr", 0.0), 0)
    from paper_2307_11447_gb300 import analysis as an

    ctx.h4d_proposal(h4d.H4D_PROPOSAL_UNIFORM, args.cell_len, 0.1, 0)
    ug = _fixed_n_sample(ctx, args.calib_cycles)
    ctx.h4d_proposal(h4d.H4D_PROPOSAL_LEARNED, args.cell_len, 0.1, 0)
    lg = _fixed_n_sample(ctx, args.calib_cycles)
    ui, ud = _flat(ug)
    li, ld = _flat(lg)
    mu = _balanced_mu(ui, ud)
    acc = lambda xi, xd: 0.5 * (np.exp(np.minimum(xi + mu, 0)).mean() + np.exp(np.minimum(xd - mu, 0)).mean())
    # standard errors by a jackknife over chains (Eq. 21 estimates at the balancing beta mu)
    acc_se = lambda g: an.jackknife(g, lambda gg: acc(*_flat(gg)))[1]
    ctx.h4d_set_no_accept(0)
    ctx.h4d_set_mu(mu)
    cfg["beta_mu"] = mu  # the timed cycles run at the balancing beta mu
    return {
        "records": int(ok.sum()), "record_n_f": args.record_nf, "cell_len_A": args.cell_len,
        "grid_cells_per_edge": int(max(3, min(32, math.floor(cfg["L"] / args.cell_len)))),
        "record_generation_s": t_rec, "train_steps": args.train_steps, "train_batch": 4096, "train_s": t_train,
        "train_loss_first_last": [loss0, loss], "target_shift_y0": y0,
        "beta_mu_balanced": mu,
        "fixed_n_production": {
            "trials_per_proposal": int(len(ui) + len(ud)),
            "uniform": {"median_x_ins": float(np.median(ui)), "median_x_del": float(np.median(ud)),
                        "mean_acceptance_at_balanced_mu": float(acc(ui, ud)),
                        "mean_acceptance_se": float(acc_se(ug))},
            "learned": {"median_x_ins": float(np.median(li)), "median_x_del": float(np.median(ld)),
                        "mean_acceptance_at_balanced_mu": float(acc(li, ld)),
                        "mean_acceptance_se": float(acc_se(lg))},
        },
    }


def uniform_arm(ctx, reps, args, n_eq, n_f, stream):
    """The same grand-canonical cycles with uniform placement (the plain method), timed
    like the learned ones."""
    import torch

    from paper_2307_11447_gb300 import lib as h4d

    ctx.h4d_proposal(h4d.H4D_PROPOSAL_UNIFORM, args.cell_len, 0.1, 0)
    c0 = [ctx.h4d_get_counts(r) for r in range(ctx.R)]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(args.steps):
        ctx.h4d_run_trials(1, n_eq)
    ev[1].record(stream)
    torch.cuda.synchronize()
    secs = ev[0].elapsed_time(ev[1]) / 1e3
    c1 = [ctx.h4d_get_counts(r) for r in range(ctx.R)]
    acc = sum((b["accepted_ins"] + b["accepted_del"]) - (a["accepted_ins"] + a["accepted_del"]) for a, b in zip(c0, c1))
    units = 0.0
    for r, (a, b) in enumerate(zip(c0, c1)):
        mean_pairs = (b["sum_n"] - a["sum_n"]) / max(b["cycles"] - a["cycles"], 1)
        units += (2.0 * mean_pairs + 3.0 * reps[r].get("n_water", 0)) * (n_eq + n_f) * args.steps
    return {"atom_steps_per_s": units / secs, "accepted_exchanges_per_s": acc / secs, "accepted": int(acc),
            "ms_per_step": 1e3 * secs / args.steps}


def sequential_baseline(reps, cfg, count, n_eq):
    """The same cycle run replica by replica, each alone in its own context (the GPU idle
    but for one replica), on `count` replicas spread over the size range; the rate is
    their atom-steps over their summed time."""
    import torch

    from paper_2307_11447_gb300 import lib as h4d

    idx = np.linspace(0, len(reps) - 1, count).astype(int)
    t_sum, units = 0.0, 0.0
    for k in idx:
        ctx = h4d.Context(h4d.make_params(cfg), [reps[k]], seed=5)
        ctx.h4d_run_md(200)
        ctx.h4d_autotune(10)
        ctx.h4d_run_trials(1, n_eq)
        torch.cuda.synchronize()
        c0 = ctx.h4d_get_counts(0)
        t0 = time.perf_counter()
        ctx.h4d_run_trials(1, n_eq)
        torch.cuda.synchronize()
        t_sum += time.perf_counter() - t0
        c1 = ctx.h4d_get_counts(0)
        units += 2.0 * c1["n_pairs"] * (n_eq + cfg["n_f"])
        ctx.close()
    return {"value": units / t_sum, "unit": "atom-steps/s", "replicas_timed": int(count),
            "seconds_for_256_estimate": t_sum * len(reps) / count}


def water_calibration(ctx, cfg, args):
    """Untimed: beta mu of the rigid water by BAR (SI Eq. S2) on fixed-N water trials of
    every chain at the configuration's protocol, then set for the timed cycles."""
    from paper_2307_11447_gb300 import analysis as an

    ctx.h4d_set_no_accept(1)
    ins, dele = [], []
    ctx.h4d_run_trials(args.calib_cycles, 100)
    for r in range(ctx.R):
        w = ctx.h4d_get_work(r, args.calib_cycles)
        ok = w["status"] == 0
        ins.append(w["beta_dM"][ok & (w["move"] == 1)])
        dele.append(w["beta_dM"][ok & (w["move"] == 0)])
    groups = list(zip(ins, dele))
    mu, se = an.jackknife(groups, lambda g: an.bar_mu(np.concatenate([a for a, _ in g]),
                                                      np.concatenate([b for _, b in g])))
    a, b = np.concatenate(ins), np.concatenate(dele)
    acc = 0.5 * (an.p_acc(a, mu, True) + an.p_acc(b, mu, False))
    ctx.h4d_set_no_accept(0)
    ctx.h4d_set_mu(mu)
    cfg["beta_mu"] = mu
    return {"beta_mu_bar": mu, "beta_mu_se": se, "fixed_n_trials": int(a.size + b.size),
            "mean_beta_dM_ins": float(a.mean()), "mean_beta_dM_del": float(b.mean()),
            "acceptance_eq21_at_bar_mu": float(acc), "cycles": args.calib_cycles, "n_eq": 100}


def ewald_timing(kmax=14, alpha=0.25):
    """The long-range Coulomb term (Eqs. 9-10, reciprocal-space Ewald sum with forces) of
    one configuration of the aqueous NaCl system (9110 atoms, L = 45 A), evaluated once to
    warm up and once timed: the two kernels' device time from CUDA events inside the call.
    A term is one (k-vector, atom) phase, its sine and cosine and their accumulation; each
    kernel evaluates every term of the half space of k-vectors once."""
    from paper_2307_11447_gb300 import lib as h4d
    from paper_2307_11447_gb300 import workloads as wl

    cfg = dict(wl.CONFIGS["nacl_aq"])
    x = wl.aqueous_positions(cfg["n_water"], cfg["n_pairs"], cfg["L"], 5)
    p = h4d.make_params(cfg)
    h4d.h4d_ewald_lr(p, cfg["L"], x, alpha, kmax, n_water=cfg["n_water"])
    ur, us, _, ms = h4d.h4d_ewald_lr(p, cfg["L"], x, alpha, kmax, n_water=cfg["n_water"], kernel_ms=True)
    n_k = ((2 * kmax + 1) ** 3 - 1) // 2  # half space of 0 < max_d |n_d| <= kmax
    n = len(x)
    return {"atoms": n, "kmax": kmax, "alpha_per_A": alpha, "k_vectors_half_space": n_k, "kernel_ms": ms,
            "terms_per_s": 2.0 * n_k * n / (ms * 1e-3), "U_recip_kJ_mol": ur, "U_self_kJ_mol": us}


def plain_at_equal_se(rep, cfg, n_eq, stream, batched_s, se_batched, trials_batched, accepted_batched):
    """The plain arm of the equal-error comparison: one chain alone on the GPU (its own
    context, the same cycle), timed with CUDA events over one cycle after a warm-up.  The
    batched run reached SE(<N>) = se_batched with trials_batched independent-chain trials
    in batched_s seconds; a single chain needs at least as many trials for the same error
    (its consecutive trials are correlated), so its time to that error is at least
    trials_batched x its time per cycle."""
    import torch

    from paper_2307_11447_gb300 import lib as h4d

    with torch.cuda.stream(stream):
        ctx = h4d.Context(h4d.make_params(cfg), [rep], seed=777, stream=stream.cuda_stream)
    ctx.h4d_run_md(200)
    ctx.h4d_autotune(5)
    ctx.h4d_run_trials(1, n_eq)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.h4d_run_trials(1, n_eq)
    e1.record(stream)
    torch.cuda.synchronize()
    t1 = e0.elapsed_time(e1) / 1e3
    ctx.close()
    plain_s = t1 * trials_batched
    return {"se_mean_n": se_batched, "trials": trials_batched, "batched_s": batched_s,
            "plain_s_per_cycle": t1, "plain_s_to_same_se_lower_bound": plain_s,
            "speedup_at_equal_se": plain_s / batched_s,
            "accepted_exchanges_per_s": {"batched": accepted_batched / batched_s,
                                         "plain": accepted_batched / plain_s}}


def run_e2e(ctx, reps, args, n_eq, n_f, stream, world, dist):
    """Same metric through the public API with host buffers: every step uploads each
    chain's positions and velocities from pinned host memory, runs one cycle and reads the
    counters and trial records back."""
    import ctypes

    import torch

    from paper_2307_11447_gb300.lib import h4d_counts as h4d_counts_t

    xs, vs, counts = [], [], []
    for r in range(ctx.R):
        x, v = ctx.h4d_get_state(r)
        c = ctx.h4d_get_counts(r)
        counts.append((int(c["n_water"]), int(c["n_pairs"])))  # the layout of the snapshot
        xs.append(torch.from_numpy(x).pin_memory())
        vs.append(torch.from_numpy(v).pin_memory())
    torch.cuda.synchronize()
    h2d = sum(x.numel() * 8 + v.numel() * 8 for x, v in zip(xs, vs))
    d2h = 0
    t0 = time.perf_counter()
    atom_steps = 0.0
    for k in range(args.steps):
        for r in range(ctx.R):
            ctx.h4d_set_water_state(r, counts[r][0], counts[r][1], xs[r].numpy(), vs[r].numpy())
        ctx.h4d_run_trials(1, n_eq)
        d2h = 0
        for r in range(ctx.R):
            c = ctx.h4d_get_counts(r)
            rec = ctx.h4d_get_work(r, 1)
            d2h += ctypes.sizeof(h4d_counts_t) + rec.nbytes
            atom_steps += (2.0 * c["n_pairs"] + 3.0 * c["n_water"]) * (n_eq + n_f)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    secs, tot = reduce_over_ranks(secs, [atom_steps], dist)
    atom_steps = float(tot[0])
    return {"value": atom_steps / secs, "unit": "atom-steps/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h)}


# ---------------------------------------------------------------------------------------
# CPU oracle timing (test infrastructure, used only for the baseline legs)
# ---------------------------------------------------------------------------------------
def _oracle_chain(job):
    name, seed, n_steps = job
    sys.path.insert(0, ROOT)
    from oracle import oracle as orc
    from paper_2307_11447_gb300 import workloads as wl

    if name == "batched256":
        # one replica of the batched workload (sizes 100-1000 ions, rho 0.1-0.4) per process
        cfg, reps = wl.batched_system(256, seed=7)
        rep = reps[(seed * 37) % len(reps)]
        cfg = dict(cfg, L=rep["L"], n_pairs=rep["n_pairs"], cap_pairs=rep["cap_pairs"])
    else:
        cfg = dict(wl.CONFIGS["nacl_aq" if name in ("nacl_learned", "nacl_water") else name])
    p = orc.make_params(cfg, use_cells=1, seed=seed)
    if cfg.get("n_water", 0):
        x = wl.aqueous_positions(cfg["n_water"], cfg["n_pairs"], cfg["L"], seed)
    else:
        x = wl.lj_positions(cfg["n_pairs"], cfg["L"], seed)
    st = orc.State(p, x, None, cfg["n_pairs"], cfg["cap_pairs"])
    orc.init_velocities(p, st)
    t0 = time.perf_counter()
    orc.md(p, st, n_steps)
    dt = time.perf_counter() - t0
    return (3 * cfg.get("n_water", 0) + 2 * cfg["n_pairs"]) * n_steps, dt


def cpu_baseline(name, sample_steps=8, cores=None, one_core=True):
    """The oracle as it stands, one chain per host process (spawned), each running
    sample_steps MD steps of the 4000-ion system (every MD step costs one 4D force
    evaluation like a NEMD step)."""
    import multiprocessing as mp

    cores = cores or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_chain, [(name, 77 + k, sample_steps) for k in range(cores)])
    wall = time.perf_counter() - t0
    units = sum(r[0] for r in res)
    busy = max(r[1] for r in res)
    system = {"nacl_aq": "aqueous NaCl system", "nacl_learned": "aqueous NaCl system",
              "nacl_water": "aqueous NaCl system", "batched256": "batched workload (one replica each)",
              "lj250": "250-ion system"}.get(name, "4000-ion system")
    out = {"value": units / busy, "unit": "atom-steps/s", "cores": cores, "kind": "oracle",
           "sample": f"{cores} chains x {sample_steps} MD steps of the {system}, cell list, FP64 "
                     f"(wall {wall:.1f} s incl. process start)"}
    if one_core and cores > 1:
        with ctx.Pool(1) as pool:
            u1, t1 = pool.map(_oracle_chain, [(name, 77, sample_steps)])[0]
        out["one_core"] = {"value": u1 / t1, "unit": "atom-steps/s", "seconds": t1}
    return out


def reference_config(args, world):
    """The GPU arm's `config` for the same flags (positions are not needed for it)."""
    if args.workload == "batched256":
        cfg, reps = workload(args.workload, args.chains, 0)
    else:
        cfg, _ = workload(args.workload, 0, 0)
        reps = [{}] * args.chains
    return workload_config(args, cfg, reps, cfg["n_f"], cfg["n_eq"], world)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cores = args.cpu_cores or os.cpu_count() or 1
    # the same sample size as the GPU line's cpu_baseline (60 MD steps per chain), so the
    # process start-up does not weigh on the rate
    for _ in range(args.warmup):
        cpu_baseline(args.workload, sample_steps=2, cores=cores, one_core=False)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(args.workload, sample_steps=60, cores=cores, one_core=False))
    secs = time.perf_counter() - t0
    value = float(np.mean([v["value"] for v in vals]))
    out = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "atom-steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": reference_config(args, world),
        "cpu_baseline": {"value": value, "unit": "atom-steps/s", "cores": cores, "kind": "oracle",
                         "sample": vals[-1]["sample"]},
        "e2e": {"value": value, "unit": "atom-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


ARGS = None


def main():
    global ARGS
    args = parse()
    if args.chains is None:
        args.chains = 152 if args.workload in ("nacl_aq", "nacl_learned", "nacl_water") else 304
    ARGS = args
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
