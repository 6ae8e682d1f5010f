"""Sampling protocols of the per-configuration statistics.

The oracle (tests/golden/make_config_stats.py, offline) and the GPU (tests/test_gpu_config_stats.py)
run the same protocol on independent chains; the tests compare the resulting statistics
at two combined standard errors.  A chain starts from seeded uniform positions
(``workloads.lj_positions`` / ``aqueous_positions``), Maxwell-Boltzmann velocities, and
``equil`` thermostatted MD steps, then runs ``trials`` cycles of ``n_eq`` MD steps plus one
pair-exchange trial.  Grand-canonical runs ("gc") accept trials by Eqs. 6 and 8; fixed-N
runs ("fixed_n", Sec. II.E) record the work of every trial and accept none.  Statistics
use the trials after the first ``burn``.

The number of equilibrium MD steps between trials is not part of the configurations
(their 1000 steps are the initial equilibration); the grand-canonical runs of the
250-ion electrolyte use 100 so that a chain sees tens of accepted exchanges.
"""
from paper_2307_11447_gb300 import workloads as wl

# beta mu estimation: fixed-N insertion and deletion work at the configuration's N (BAR)
CALIBRATE = {
    "lj250": dict(kind="fixed_n", chains_oracle=32, equil=1000, trials=20, n_eq=1000, seed_oracle=20000),
    "lj4000": dict(kind="fixed_n", chains_oracle=24, equil=1000, trials=6, n_eq=1000, seed_oracle=21000),
}

STATS = {
    "lj250": dict(kind="gc", chains_oracle=32, chains_gpu=256, equil=1000, trials=600, n_eq=100, burn=100,
                  seed_oracle=22000, seed_gpu=32000),
    "lj4000": dict(kind="gc", chains_oracle=24, chains_gpu=304, equil=1000, trials=6, n_eq=1000, burn=0,
                   seed_oracle=23000, seed_gpu=33000),
    # eight replicas of the batched workload spanning its size range, several chains each
    "batched_subset": dict(kind="gc", replicas=(0, 37, 74, 111, 148, 185, 222, 255), chains_oracle=4, chains_gpu=16,
                           equil=500, trials=40, n_eq=100, burn=0, seed_oracle=24000, seed_gpu=34000),
    # fixed N: the works do not depend on beta mu; the run (and the BAR estimate of the
    # configuration's beta mu drawn from it) took the exponents at -60
    "nacl_aq": dict(kind="fixed_n", chains_oracle=8, chains_gpu=152, equil=200, trials=3, n_eq=100, burn=0,
                    seed_oracle=25000, seed_gpu=35000, beta_mu=-60.0),
}


def config_of(name: str) -> dict:
    """workload dictionary of a statistics configuration (the batched subset uses the
    batched workload's physics)"""
    if name == "batched_subset":
        cfg, _ = wl.batched_system(256, seed=7)
        return dict(cfg)
    cfg = dict(wl.CONFIGS[name])
    if "beta_mu" in STATS.get(name, {}):
        cfg["beta_mu"] = STATS[name]["beta_mu"]
    return cfg


def chain_inputs(name: str, k: int, seed: int) -> dict:
    """box, ion pairs, capacity, waters and seeded positions of chain k of a configuration"""
    prot = STATS.get(name) or CALIBRATE[name]
    if name == "batched_subset":
        reps = wl.batched_replicas(256, seed=7)
        ridx = prot["replicas"][k % len(prot["replicas"])]
        n, _rho, L = reps[ridx]
        cap = n // 2 + max(16, (3 * n) // 20)
        return dict(L=L, n_pairs=n // 2, cap_pairs=cap, x=wl.lj_positions(n // 2, L, seed), n_water=0, rep=ridx)
    cfg = wl.CONFIGS[name]
    if cfg.get("n_water", 0):
        x = wl.aqueous_positions(cfg["n_water"], cfg["n_pairs"], cfg["L"], seed)
        return dict(L=cfg["L"], n_pairs=cfg["n_pairs"], cap_pairs=cfg["cap_pairs"], x=x, n_water=cfg["n_water"])
    return dict(L=cfg["L"], n_pairs=cfg["n_pairs"], cap_pairs=cfg["cap_pairs"],
                x=wl.lj_positions(cfg["n_pairs"], cfg["L"], seed), n_water=0)
