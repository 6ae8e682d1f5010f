"""Workload definitions and seeded synthetic inputs.

This module holds parameter values and random initial configurations only; none of the
method's arithmetic lives here.  Both the CUDA path and the CPU oracle take their inputs
from it.

Systems (units: LJ reduced units with k_B T = 1 for the LJ electrolyte; Angstrom, fs,
amu, kJ/mol and e for aqueous NaCl):

* ``lj250``  -- 250 ions (125 +1 / 125 -1), sigma = eps = m = 1, LJ cut-off 2.5,
  Bjerrum length 2 (Coulomb prefactor 2 at k_B T = 1), erfc(0.3 r)/r Coulomb cut at 4,
  density 0.2, dt 0.005, w_max 4, linear altitude protocol over 100 steps.
* ``lj4000`` -- the same electrolyte with 4000 ions at density 0.3, 500 NEMD steps.
* ``batched256`` -- 256 independent LJ-electrolyte replicas, ion counts uniform in
  [100, 1000] (even), densities uniform in [0.1, 0.4].
* ``nacl_aq`` -- 3000 rigid SPC/E-geometry waters + 55 Na+ + 55 Cl- at L = 45 A.

Initial positions are uniform random with overlap rejection (minimum distance 0.8 sigma,
or 2.0 A between atoms of different molecules); the configurations are then equilibrated
by the method's own MD.
"""
from __future__ import annotations

import math

import numpy as np

# --------------------------------------------------------------------------------------
# LJ electrolyte (RPM-like): type 0 cation (+1), type 1 anion (-1)
# --------------------------------------------------------------------------------------
LJ_PHYSICS = dict(
    system="lj",
    beta=1.0,
    rc_lj=2.5,
    rc_coul=4.0,
    alpha=0.3,
    kcoul=2.0,  # Bjerrum length 2 sigma at k_B T = 1
    kappa_sr=0.0,
    q=[1.0, -1.0],
    sig=[1.0, 1.0],
    eps=[1.0, 1.0],
    mass=[1.0, 1.0],
    mvv2e=1.0,
    dt=0.005,
    w_max=4.0,
    tau_t=0.1,
    schedule="linear",
    sched_n=1.0,
    n_water=0,
    d_oh=0.0,
    d_hh=0.0,
    skin=0.3,
    min_dist=0.8,
)

# --------------------------------------------------------------------------------------
# Aqueous NaCl: type 0 Na+, 1 Cl-, 2 O (SPC/E), 3 H
# --------------------------------------------------------------------------------------
KT_298 = 2.47772  # kJ/mol at 298 K
AQ_PHYSICS = dict(
    system="aq",
    beta=1.0 / KT_298,
    rc_lj=10.0,
    rc_coul=10.0,
    alpha=0.25,
    kcoul=1389.35458,  # kJ A / (mol e^2)
    kappa_sr=1.0,
    q=[1.0, -1.0, -0.8476, 0.4238],
    sig=[2.16, 4.83, 3.166, 0.0],
    eps=[1.475, 0.0535, 0.650, 0.0],
    mass=[22.99, 35.45, 15.9994, 1.008],
    mvv2e=1.0e4,  # amu A^2 / fs^2 -> kJ/mol
    dt=1.0,
    w_max=3.0,
    tau_t=100.0,
    schedule="linear",
    sched_n=1.0,
    d_oh=1.0,
    d_hh=2.0 * math.sin(math.radians(109.47) / 2.0),
    skin=1.0,
    min_dist=2.0,
)


def box_for(n_ions: int, rho: float) -> float:
    return (n_ions / rho) ** (1.0 / 3.0)


def lj_config(n_ions: int, rho: float, n_f: int, **extra) -> dict:
    cfg = dict(LJ_PHYSICS)
    cfg.update(n_ions=n_ions, n_pairs=n_ions // 2, rho=rho, L=box_for(n_ions, rho), n_f=n_f)
    cfg.update(extra)
    return cfg


# The five workloads.  beta_mu of the 250- and 4000-ion electrolytes is the BAR estimate
# (SI Eq. S2) from fixed-N insertion and deletion work of the FP64 oracle at the
# configuration's N (tests/golden/make_config_stats.py, stage "calibrate"): -8.694 +- 0.150
# for 250 ions, -8.818 +- 0.524 for 4000 ions.
CONFIGS = {
    "lj250": lj_config(250, 0.2, 100, trials=200, n_eq=1000, cap_pairs=256, beta_mu=-8.694),
    # Verlet skin 0.4, outer-list skin 1.8: the best of two skin sweeps on two GPUs (+2%
    # over 0.3 / 1.8; larger Verlet skins cost more in the force pass than they save in
    # list passes, larger outer skins more in the outer rows)
    "lj4000": lj_config(4000, 0.3, 500, trials=10000, n_eq=1000, cap_pairs=2304, chains=304,
                        beta_mu=-8.818, skin=0.4, skin_outer=1.8),
}


def _pick_far(rng, L, placed, n_new, min_dist, max_tries=200000):
    """Random sequential placement with a minimum-image overlap check on a cell grid."""
    pos = np.zeros((n_new, 3))
    nc = max(1, int(L // min_dist))
    cell = {}
    for p in placed:
        key = tuple((np.floor(p / L * nc).astype(int)) % nc)
        cell.setdefault(key, []).append(p)
    k = 0
    tries = 0
    while k < n_new:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place atoms without overlap")
        r = rng.random(3) * L
        c = np.floor(r / L * nc).astype(int) % nc
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for q in cell.get(((c[0] + dx) % nc, (c[1] + dy) % nc, (c[2] + dz) % nc), ()):
                        d = r - q
                        d -= L * np.round(d / L)
                        if d @ d < min_dist * min_dist:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            pos[k] = r
            cell.setdefault(tuple(c), []).append(r)
            k += 1
    return pos


def lj_positions(n_pairs: int, L: float, seed: int, min_dist: float = 0.8) -> np.ndarray:
    """Uniform random ion positions (interleaved cation/anion) with overlap rejection:
    every atom closer than min_dist (minimum image) to another is redrawn until none is."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    n = 2 * n_pairs
    x = rng.random((n, 3)) * L
    for _ in range(10000):
        if n < 2:
            break
        pairs = cKDTree(np.mod(x, L), boxsize=L).query_pairs(min_dist, output_type="ndarray")
        if len(pairs) == 0:
            break
        bad = np.unique(pairs[:, 1])
        x[bad] = rng.random((bad.size, 3)) * L
    else:
        raise RuntimeError("could not place atoms without overlap")
    return np.mod(x, L)


def aqueous_positions(n_water: int, n_pairs: int, L: float, seed: int, d_oh: float = 1.0,
                      hoh_deg: float = 109.47) -> np.ndarray:
    """Rigid waters (O,H,H) and interleaved Na/Cl on randomly chosen sites of a cubic
    lattice filling the box, each water with a uniformly random orientation."""
    rng = np.random.default_rng(seed)
    n_sites = n_water + 2 * n_pairs
    m = int(math.ceil(n_sites ** (1.0 / 3.0)))
    a = L / m
    g = (np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), -1).reshape(-1, 3) + 0.5) * a
    sites = g[rng.permutation(len(g))[:n_sites]]
    th = math.radians(hoh_deg)
    ref = np.array([[0.0, 0.0, 0.0], [d_oh, 0.0, 0.0], [d_oh * math.cos(th), d_oh * math.sin(th), 0.0]])
    q = rng.normal(size=(n_water, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    a0, b, c, d = q.T
    rot = np.stack([
        np.stack([a0 * a0 + b * b - c * c - d * d, 2 * (b * c - a0 * d), 2 * (b * d + a0 * c)], -1),
        np.stack([2 * (b * c + a0 * d), a0 * a0 - b * b + c * c - d * d, 2 * (c * d - a0 * b)], -1),
        np.stack([2 * (b * d - a0 * c), 2 * (c * d + a0 * b), a0 * a0 - b * b - c * c + d * d], -1)], 1)
    out = np.zeros((3 * n_water + 2 * n_pairs, 3))
    out[: 3 * n_water] = (sites[:n_water, None, :] + np.einsum("kj,wij->wki", ref, rot)).reshape(-1, 3)
    out[3 * n_water:] = sites[n_water:]
    return np.mod(out, L)


def aq_config(n_water: int, n_pairs: int, L: float, n_f: int, **extra) -> dict:
    cfg = dict(AQ_PHYSICS)
    cfg.update(n_water=n_water, n_pairs=n_pairs, L=L, n_f=n_f)
    cfg.update(extra)
    return cfg


def batched_replicas(n_rep: int = 256, seed: int = 7, n_min: int = 100, n_max: int = 1000,
                     rho_min: float = 0.1, rho_max: float = 0.4, min_box: float = 8.6):
    """Ion counts uniform in [n_min, n_max] (even) and densities uniform in
    [rho_min, rho_max], one (n_ions, rho, L) triple per replica.  Draws whose box is
    smaller than min_box (twice the largest cut-off plus skin, so that every pair has a
    single minimum image) are redrawn."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n_rep:
        n = int(rng.integers(n_min // 2, n_max // 2 + 1)) * 2
        rho = float(rng.uniform(rho_min, rho_max))
        L = box_for(n, rho)
        if L >= min_box:
            out.append((n, rho, L))
    return out


def batched_system(n_rep: int = 256, seed: int = 7):
    """The batched workload: LJ-electrolyte physics of the 250-ion system, one replica per
    (n, rho, L) draw, seeded positions per replica."""
    cfg = lj_config(250, 0.2, 100, n_eq=1000, beta_mu=-6.0)
    reps = []
    for k, (n, rho, L) in enumerate(batched_replicas(n_rep, seed)):
        cap = n // 2 + max(16, (3 * n) // 20)
        reps.append(dict(L=L, n_pairs=n // 2, cap_pairs=cap, x=lj_positions(n // 2, L, 10000 + k), rho=rho))
    return cfg, reps


# aqueous NaCl (~1 m): 3000 rigid waters + 55 Na+ + 55 Cl-, L = 45 A, NaCl-pair NEMD over
# 1000 steps of 1 fs, 2000 equilibrium steps between trials.  beta mu of the pair: BAR (SI
# Eq. S2) on the oracle's fixed-N works of this configuration (24 trials from 8 chains,
# insertion and deletion works barely overlap): -139.4 +- 12.6
def _aq_main():
    return aq_config(3000, 55, 45.0, 1000, n_eq=2000, cap_pairs=80, beta_mu=-139.4)


CONFIGS["nacl_aq"] = _aq_main()
