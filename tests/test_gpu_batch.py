"""Batching of uneven replicas in one persistent launch.

* A batch of 320 LJ-electrolyte replicas with ion counts in [100, 1000] and densities in
  [0.1, 0.4] runs in one launch; the planner packs the smaller replicas as groups of warps
  into shared CTAs.  Sixteen of them, chosen across the size range, are run again each
  alone in a context of its own (a whole CTA, another thread count) with the same seed
  and replica key: positions, velocities, trial records (byte for byte) and counters must be
  bit-identical,
  because every sum of the engine is independent of the launch plan.
* The lanes per neighbour row (threads_per_atom, the autotuner's choice) change only the
  FP32 summation order of the forces: single trials from the same states under each of
  1, 2, 4, 8, 16 lanes agree with the single-lane trials within the trial-work tolerance
  of the oracle comparisons (1e-3 kT within 20 kT of the acceptance boundary, at least
  half of those within 2e-5 kT, 1e-3 relative beyond), with identical decisions away from
  ties; the autotuned context lies within the same bounds.
* Replicas packed with others match the FP64 oracle trial by trial when the oracle uses
  the same (seed, replica key).
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2307_11447_gb300 import lib as h4d
from paper_2307_11447_gb300 import workloads as wl

from .parity_util import trial_work_bound

pytestmark = pytest.mark.gpu

TWO32 = 4294967296.0
N_BATCH = 320
SUBSET = tuple(range(0, N_BATCH, N_BATCH // 16))


def quantize(x, L):
    return np.mod(np.rint(np.mod(x, L) / L * TWO32), TWO32) * (L / TWO32)


def _batch():
    cfg = dict(wl.lj_config(250, 0.2, 60, n_eq=30, beta_mu=-8.7))
    reps = []
    for k, (n, _rho, L) in enumerate(wl.batched_replicas(N_BATCH, seed=11)):
        cap = n // 2 + max(16, (3 * n) // 20)
        reps.append(dict(L=L, n_pairs=n // 2, cap_pairs=cap, x=wl.lj_positions(n // 2, L, 40000 + k), key=k))
    return cfg, reps


@pytest.fixture(scope="module")
def batch_run():
    cfg, reps = _batch()
    ctx = h4d.Context(h4d.make_params(cfg), reps, seed=2024)
    ctx.h4d_run_md(100)
    ctx.h4d_run_trials(5, cfg["n_eq"])
    out = {r: dict(state=ctx.h4d_get_state(r), work=ctx.h4d_get_work(r, 5), counts=ctx.h4d_get_counts(r))
           for r in range(N_BATCH)}
    ctx.close()
    return cfg, reps, out


def test_batched_replicas_are_bit_identical_to_each_replica_alone(batch_run):
    cfg, reps, out = batch_run
    shared = [r for r in SUBSET if out[r]["counts"]["plan_cta_groups"] > 1]
    warps = sorted({out[r]["counts"]["plan_warps"] for r in SUBSET})
    sizes = [2 * reps[r]["n_pairs"] for r in SUBSET]
    print(f"\nsubset ions {min(sizes)}-{max(sizes)}; group warps in the batch {warps}; "
          f"{len(shared)} of {len(SUBSET)} share a CTA with other replicas")
    assert len(shared) >= 3  # the multi-group CTAs of the planner are exercised
    accepted = 0
    for r in SUBSET:
        ctx = h4d.Context(h4d.make_params(cfg), [reps[r]], seed=2024)
        ctx.h4d_run_md(100)
        ctx.h4d_run_trials(5, cfg["n_eq"])
        c1 = ctx.h4d_get_counts(0)
        assert c1["plan_cta_groups"] == 1 and c1["plan_warps"] == 16  # a whole CTA of its own
        xa, va = out[r]["state"]
        xb, vb = ctx.h4d_get_state(0)
        assert np.array_equal(xa, xb) and np.array_equal(va, vb), r
        wa, wb = out[r]["work"], ctx.h4d_get_work(0, 5)
        assert wa.tobytes() == wb.tobytes(), r  # every bit, non-finite work of status-3 trials included
        for k in ("n_pairs", "cycles", "accepted_ins", "accepted_del", "md_steps", "nbr_builds", "nbr_refreshes"):
            assert c1[k] == out[r]["counts"][k], (r, k)
        assert c1["sum_n"] == out[r]["counts"]["sum_n"] and c1["sum_n2"] == out[r]["counts"]["sum_n2"]
        accepted += int(wa["accepted"].sum())
        ctx.close()
    print(f"{accepted} accepted exchanges among the compared trials")


def _trial_close(a, b):
    """trial-work tolerance of the oracle comparisons"""
    err = abs(a["beta_dM"] - b["beta_dM"])
    near = abs(b["x_acc"]) < 20
    return err <= trial_work_bound(b["beta_dM"], b["x_acc"]), near, err


def _single_trials(cfg, reps, out, tpa):
    starts = []
    for r in SUBSET:
        x, v = out[r]["state"]
        n_pairs = out[r]["counts"]["n_pairs"]
        starts.append(dict(L=reps[r]["L"], n_pairs=n_pairs, cap_pairs=reps[r]["cap_pairs"],
                           x=quantize(x, reps[r]["L"]), v=v, key=r))
    ctx = h4d.Context(h4d.make_params(cfg, threads_per_atom=tpa), starts, seed=77)
    if tpa == 0:
        ctx.h4d_autotune(5)
    ctx.h4d_run_trials(1, 0)
    recs = [ctx.h4d_get_work(k, 1)[0] for k in range(len(starts))]
    ctx.close()
    return recs


def test_threads_per_atom_leave_trials_within_the_work_tolerance(batch_run):
    cfg, reps, out = batch_run
    ref = _single_trials(cfg, reps, out, 1)
    near_errs = []
    for tpa in (2, 4, 8, 16, 0):
        recs = _single_trials(cfg, reps, out, tpa)
        for a, b in zip(recs, ref):
            assert a["move"] == b["move"] and a["status"] == b["status"]
            ok, near, err = _trial_close(a, b)
            assert ok, (tpa, a["beta_dM"], b["beta_dM"])
            if near:
                near_errs.append(err)
            if abs(b["ln_u"] - b["x_acc"]) > 1e-3:
                assert a["accepted"] == b["accepted"]
    print(f"\n{len(near_errs)} trials near the boundary: max |d beta dM| {max(near_errs, default=0):.2e}")
    assert np.mean(np.array(near_errs) <= 2e-5) >= 0.5


def test_packed_replicas_match_oracle_trials(batch_run):
    """single trials of replicas inside a packed batch against the oracle keyed by the
    same (seed, replica key)"""
    cfg, reps, out = batch_run
    starts = []
    for r in range(N_BATCH):
        x, v = out[r]["state"]
        starts.append(dict(L=reps[r]["L"], n_pairs=out[r]["counts"]["n_pairs"], cap_pairs=reps[r]["cap_pairs"],
                           x=quantize(x, reps[r]["L"]), v=v, key=r))
    ctx = h4d.Context(h4d.make_params(cfg), starts, seed=91)
    ctx.h4d_run_trials(1, 0)
    checked = 0
    for r in SUBSET[::2]:
        rg = ctx.h4d_get_work(r, 1)[0]
        s = starts[r]
        po = orc.make_params(dict(cfg, L=s["L"], seed=91, replica=r, use_cells=1))
        st = orc.State(po, s["x"], s["v"], s["n_pairs"], s["cap_pairs"])
        ro = orc.trial(po, st)
        assert rg["move"] == ro["move"] and rg["status"] == ro["status"]
        ok, _, _ = _trial_close(rg, ro)
        assert ok, (r, rg["beta_dM"], ro["beta_dM"])
        if abs(ro["ln_u"] - ro["x_acc"]) > 1e-3:
            assert rg["accepted"] == ro["accepted"]
        checked += 1
    assert ctx.h4d_get_counts(SUBSET[0])["plan_cta_groups"] >= 1
    ctx.close()
    assert checked == len(SUBSET[::2])
