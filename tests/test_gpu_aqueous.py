"""Aqueous NaCl on the GPU against the oracle: 4-type pair terms with Lorentz-Berthelot
mixing and intramolecular exclusions, rigid waters kept rigid by SHAKE/RATTLE, and
single insertion/deletion trials (Sec. II.D.2 model, Sec. II.A trial).  A reduced box
(400 waters + 10 ion pairs, L = 24 A) keeps the brute-force oracle fast."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2307_11447_gb300 import lib as h4d
from paper_2307_11447_gb300 import workloads as wl

from .parity_util import force_bounds

pytestmark = pytest.mark.gpu

TWO32 = 4294967296.0
NW, NP, L = 400, 10, 24.0


def quantize(x, L):
    return np.mod(np.rint(np.mod(x, L) / L * TWO32), TWO32) * (L / TWO32)


def small_cfg(**kw):
    cfg = wl.aq_config(NW, NP, L, 20, n_eq=0, cap_pairs=16, beta_mu=-40.0, seed=4, replica=0)
    cfg.update(kw)
    return cfg


def _relaxed_state(steps=60):
    cfg = small_cfg()
    p = orc.make_params(cfg)
    x = wl.aqueous_positions(NW, NP, L, 2)
    st = orc.State(p, x, None, NP, cfg["cap_pairs"])
    orc.init_velocities(p, st)
    orc.md(p, st, steps)
    return cfg, quantize(st.positions(), L), st.velocities()


def _bonds(x):
    o, h1, h2 = x[0:3 * NW:3], x[1:3 * NW:3], x[2:3 * NW:3]
    d = lambda a, b: np.linalg.norm((a - b) - L * np.round((a - b) / L), axis=1)
    return d(o, h1), d(o, h2), d(h1, h2)


def test_aqueous_forces_match_oracle():
    cfg, x, _ = _relaxed_state(20)
    Uo, Fo = orc.energy_forces(orc.make_params(cfg), x)
    Ug, Fg = h4d.h4d_eval_forces(h4d.make_params(cfg), L, x, None, n_water=NW)
    err = np.linalg.norm(Fg - Fo, axis=1)
    bound = force_bounds(cfg, x, Fo)
    assert np.all(err <= bound), (err / bound).max()
    assert Ug == pytest.approx(Uo, rel=1e-10)


def test_aqueous_flyers_screened_forces_match_oracle():
    cfg, x, _ = _relaxed_state(20)
    w = np.zeros(len(x))
    fly = np.zeros(len(x), np.uint8)
    a, b = 3 * NW + 4, 3 * NW + 7  # a cation and an anion
    w[[a, b]] = float(np.float32(1.75))
    fly[[a, b]] = 1
    Uo, Fo = orc.energy_forces(orc.make_params(cfg), x, w, fly)
    Ug, Fg = h4d.h4d_eval_forces(h4d.make_params(cfg), L, x, w, n_water=NW)
    keep = fly == 0
    err = np.linalg.norm(Fg - Fo, axis=1)[keep]
    bound = force_bounds(cfg, x, Fo, w)[keep]
    assert np.all(err <= bound), (err / bound).max()
    assert Ug == pytest.approx(Uo, rel=1e-10)


def test_gpu_md_keeps_water_rigid_and_conserves_energy():
    cfg, x, v = _relaxed_state(20)
    cfg = dict(cfg, tau_t=0.0)  # plain NVE
    ctx = h4d.Context(h4d.make_params(cfg), [dict(L=L, n_pairs=NP, cap_pairs=16, x=x, v=v, n_water=NW)], seed=1)
    U0, K0 = ctx.h4d_get_energies(0)
    ctx.h4d_run_md(300)
    U1, K1 = ctx.h4d_get_energies(0)
    xg, vg = ctx.h4d_get_state(0)
    for d, ref in zip(_bonds(xg), (1.0, 1.0, cfg["d_hh"])):
        assert np.abs(d - ref).max() < 2e-5
    # rigid-body velocities: no bond-parallel relative velocity
    o, h1 = slice(0, 3 * NW, 3), slice(1, 3 * NW, 3)
    rab = xg[o] - xg[h1]
    rab -= L * np.round(rab / L)
    assert np.abs((rab * (vg[o] - vg[h1])).sum(1)).max() < 1e-6
    # the oracle's FP64 NVE over the same 300 fs sets the scale of the integration error
    po = orc.make_params(cfg)
    st = orc.State(po, x, v, NP, 16)
    E0o = orc.energy_forces(po, st.positions())[0] + orc.kinetic(po, st.velocities())
    orc.nve(po, st, 300)
    E1o = orc.energy_forces(po, st.positions())[0] + orc.kinetic(po, st.velocities())
    n = 3 * NW + 2 * NP
    drift_g, drift_o = abs((U1 + K1) - (U0 + K0)) / n, abs(E1o - E0o) / n
    print(f"NVE drift per atom over 300 fs: gpu {drift_g:.2e}, oracle {drift_o:.2e} kJ/mol")
    assert drift_g < 3 * drift_o + 1e-3


def test_aqueous_single_trials_match_oracle():
    cfg, x0, v0 = _relaxed_state(60)
    po = orc.make_params(cfg)
    ctx = h4d.Context(h4d.make_params(cfg), [dict(L=L, n_pairs=NP, cap_pairs=16, x=x0, v=v0, n_water=NW)],
                      seed=cfg["seed"])
    moves = set()
    for k in range(4):
        ctx.h4d_set_state(0, NP, x0, v0)
        ctx.h4d_run_trials(1, 0)
        rg = ctx.h4d_get_work(0, 1)[0]
        st = orc.State(po, x0, v0, NP, cfg["cap_pairs"])
        st.s.trial_ctr = k
        ro = orc.trial(po, st)
        moves.add(int(ro["move"]))
        assert rg["move"] == ro["move"] and rg["cation"] == ro["cation"] and rg["anion"] == ro["anion"]
        # Aqueous tolerance: the truncated (energy-shifted) potentials make the force jump at
        # the cut-offs, and FP32 distances classify pairs crossing a cut-off a step apart
        # from FP64; over a trial of 1220 atoms this moves beta dM by ~1e-3.
        err = abs(rg["beta_dM"] - ro["beta_dM"])
        print(f"trial {k}: beta dM gpu {rg['beta_dM']:.6f} oracle {ro['beta_dM']:.6f} |diff| {err:.2e}")
        assert err <= 1e-2 + 1e-5 * abs(ro["beta_dM"]), (k, rg["beta_dM"], ro["beta_dM"])
        if abs(ro["ln_u"] - ro["x_acc"]) > 0.05:
            assert rg["accepted"] == ro["accepted"]
