"""Rigid-water exchange on the GPU (Sec. II.A with one flying particle; Sec. II.C: the
flying water's velocities drawn in its molecular frame; the flyer frozen in 3D) against
the oracle's pinned statement of the same move.

* Inserted waters from an empty box: the GPU places the same three atoms (the H atoms
  within one 32-bit grid step: the rotation's sines may round differently) with the same
  velocities (float-float storage, 1e-12 relative).
* Single trials from a relaxed aqueous state (400 waters + 10 NaCl): move, deleted water,
  status and beta Delta M within the aqueous trial tolerance (1e-2 + 1e-5 |beta dM| kT, the
  cut-off events of 1220 atoms); decisions away from ties; and, for trials every one of
  which is accepted (beta mu = +-1e8), the whole end state: the layout after an accepted
  insertion (new water last, ions up by three) or deletion (last water into the slot,
  ions down by three) and the positions and velocities of every atom.
* Ideal gas of rigid waters in 64 replicas: Poisson law, <N> = zV and Var N/<N> = 1.
"""
import math

import numpy as np
import pytest
from scipy import special

from oracle import oracle as orc
from paper_2307_11447_gb300 import lib as h4d
from paper_2307_11447_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TWO32 = 4294967296.0
NW, NP, L = 400, 10, 24.0


def quantize(x, L):
    return np.mod(np.rint(np.mod(x, L) / L * TWO32), TWO32) * (L / TWO32)


def _mi(d, L):
    return d - L * np.round(d / L)


def test_inserted_waters_match_oracle():
    Lb = 12.0
    cfg = wl.aq_config(0, 0, Lb, 2, exchange="water", q=[0.0] * 4, eps=[0.0] * 4, rc_lj=4.5, rc_coul=4.5,
                       beta_mu=math.log(1e6), seed=21, replica=0, tau_t=0.0)
    po = orc.make_params(dict(cfg, n_water=0))
    st = orc.State(po, np.zeros((0, 3)), None, 0, 0, cap_water=1)
    ctx = h4d.Context(h4d.make_params(cfg), [dict(L=Lb, n_pairs=0, cap_pairs=0, x=np.zeros((0, 3)), v=np.zeros((0, 3)),
                                                  n_water=0, cap_water=1)], seed=21)
    q = Lb / TWO32
    n_ins = 0
    for k in range(60):
        st.s.n_water = 0
        st.s.trial_ctr = k
        ro = orc.trial(po, st)
        ctx.h4d_set_water_state(0, 0, 0, np.zeros((0, 3)), np.zeros((0, 3)))
        ctx.h4d_run_trials(1, 0)
        rg = ctx.h4d_get_work(0, 1)[0]
        assert rg["move"] == ro["move"] and rg["accepted"] == ro["accepted"] and rg["status"] == ro["status"]
        if ro["move"] != 1:
            continue
        n_ins += 1
        xg, vg = ctx.h4d_get_state(0)
        xo, vo = st.positions(), st.velocities()
        assert xg.shape == xo.shape == (3, 3)
        assert np.abs(_mi(xg - xo, Lb)).max() <= 1.01 * q
        assert np.array_equal(xg[0], xo[0])  # the O sits exactly on its drawn grid point
        assert np.abs(vg - vo).max() <= 1e-12 * np.abs(vo).max()
    assert n_ins > 15


def _relaxed(cfg, steps=60):
    p = orc.make_params(cfg)
    x = wl.aqueous_positions(NW, NP, L, 2)
    st = orc.State(p, x, None, NP, cfg["cap_pairs"], cap_water=NW + 4)
    orc.init_velocities(p, st)
    orc.md(p, st, steps)
    return quantize(st.positions(), L), st.velocities()


def _cfg(**kw):
    cfg = wl.aq_config(NW, NP, L, 20, n_eq=0, cap_pairs=NP, beta_mu=-10.0, seed=4, replica=0, exchange="water")
    cfg.update(kw)
    return cfg


def _trials(cfg, x0, v0, n_trials, compare_state):
    po = orc.make_params(cfg)
    ctx = h4d.Context(h4d.make_params(cfg), [dict(L=L, n_pairs=NP, cap_pairs=NP, x=x0, v=v0, n_water=NW,
                                                  cap_water=NW + 4)], seed=cfg["seed"])
    moves = set()
    for k in range(n_trials):
        ctx.h4d_set_water_state(0, NW, NP, x0, v0)
        ctx.h4d_run_trials(1, 0)
        rg = ctx.h4d_get_work(0, 1)[0]
        st = orc.State(po, x0, v0, NP, NP, cap_water=NW + 4)
        st.s.trial_ctr = k
        ro = orc.trial(po, st)
        moves.add(int(ro["move"]))
        assert rg["move"] == ro["move"] and rg["cation"] == ro["cation"] and rg["status"] == ro["status"] == 0
        assert rg["n_before"] == ro["n_before"] == NW
        err = abs(rg["beta_dM"] - ro["beta_dM"])
        print(f"water trial {k}: move {ro['move']} beta dM gpu {rg['beta_dM']:.6f} oracle {ro['beta_dM']:.6f} "
              f"|diff| {err:.2e}, accepted {ro['accepted']}")
        big = abs(ro["beta_dM"]) >= 1e4  # an insertion onto an overlap: forces beyond 1e6
        assert err <= (1e-2 * abs(ro["beta_dM"]) if big else 1e-2 + 1e-5 * abs(ro["beta_dM"])), \
            (k, rg["beta_dM"], ro["beta_dM"])
        if abs(ro["ln_u"] - ro["x_acc"]) > 0.05:
            assert rg["accepted"] == ro["accepted"] and rg["n_after"] == ro["n_after"]
        if compare_state:
            assert ctx.h4d_get_counts(0)["n_water"] == st.n_water
            xg, vg = ctx.h4d_get_state(0)
            xo, vo = st.positions(), st.velocities()
            assert xg.shape == xo.shape
            dx = np.abs(_mi(xg - xo, L)).max()
            dv = np.abs(vg - vo).max()
            print(f"   end state: {len(xg)} atoms, max |dx| {dx:.2e} A, max |dv| {dv:.2e} A/fs")
            # an atom in the wrong slot would be Angstroms off; trajectories that pushed
            # neighbours off an overlap (beta dM above 1e3) amplify the FP32 rounding
            tight = abs(ro["beta_dM"]) < 1e3
            assert dx < (1e-3 if tight else 2e-2) and dv < (1e-4 if tight else 1e-2)
    ctx.close()
    return moves


def test_water_trials_match_oracle():
    cfg = _cfg()
    x0, v0 = _relaxed(cfg)
    moves = _trials(cfg, x0, v0, 6, compare_state=True)
    assert moves == {0, 1}


def test_accepted_water_exchanges_match_oracle_end_states():
    cfg = _cfg()
    x0, v0 = _relaxed(cfg)
    # every insertion accepted, then every deletion accepted
    m_ins = _trials(dict(cfg, beta_mu=1.0e8), x0, v0, 6, compare_state=True)
    m_del = _trials(dict(cfg, beta_mu=-1.0e8), x0, v0, 6, compare_state=True)
    assert 1 in m_ins and 0 in m_del


def test_ideal_water_gas_is_poisson_on_gpu():
    Lb, lam, n_rep, n_trials = 12.0, 3.0, 64, 4000
    cfg = wl.aq_config(3, 0, Lb, 2, exchange="water", q=[0.0] * 4, eps=[0.0] * 4, rc_lj=4.5, rc_coul=4.5,
                       beta_mu=math.log(lam / Lb**3), tau_t=0.0)
    reps = [dict(L=Lb, n_pairs=0, cap_pairs=0, x=wl.aqueous_positions(3, 0, Lb, 100 + r), v=np.zeros((9, 3)),
                 n_water=3, cap_water=24) for r in range(n_rep)]
    ctx = h4d.Context(h4d.make_params(cfg), reps, seed=17)
    series = [[] for _ in range(n_rep)]
    done = 0
    while done < n_trials:
        k = min(1000, n_trials - done)
        ctx.h4d_run_trials(k, 0)
        for r in range(n_rep):
            series[r].append(ctx.h4d_get_work(r, k)["n_after"])
        done += k
    ctx.close()
    n = np.concatenate([np.concatenate(s)[200:] for s in series]).astype(float)
    means = np.array([np.concatenate(s)[200:].mean() for s in series])
    se = means.std(ddof=1) / math.sqrt(n_rep)
    print(f"\n<N> {n.mean():.4f} +- {se:.4f} (zV {lam}), Var/<N> {n.var() / n.mean():.4f}")
    assert abs(n.mean() - lam) < 4 * se + 1e-3
    assert abs(n.var() / n.mean() - 1.0) < 0.05
    kk = np.arange(15)
    pk = np.exp(kk * math.log(lam) - lam - special.gammaln(kk + 1))
    hist = np.bincount(n.astype(int), minlength=25)[:15] / n.size
    assert np.abs(hist - pk).max() < 0.01


def test_packed_water_replicas_are_bit_identical_to_each_alone():
    """Water exchange in a packed launch: twelve aqueous replicas of 40-300 waters (+ 0-2
    NaCl pairs, short cut-offs so that the small boxes are legal) share CTAs; three trials
    with every insertion accepted, then three with every deletion accepted, so the ions
    of every replica move up and down inside its packed slice.  Each replica run alone in
    a context of its own with the same seed and replica key gives the same records, end
    state and water count bit for bit."""
    sizes = [40, 60, 80, 100, 120, 150, 180, 200, 220, 240, 270, 300]
    cfg = wl.aq_config(0, 0, 12.0, 20, rc_lj=4.0, rc_coul=4.0, exchange="water", n_eq=5, beta_mu=1.0e8)
    reps = []
    for k, nw in enumerate(sizes):
        npair = k % 3
        Lk = ((nw + 2 * npair) / 0.025) ** (1.0 / 3.0)  # a dilute liquid: lattice spacing near 3 A
        reps.append(dict(L=Lk, n_pairs=npair, cap_pairs=npair, n_water=nw, cap_water=nw + 8, key=100 + k,
                         x=wl.aqueous_positions(nw, npair, Lk, 500 + k)))

    def run(rs):
        ctx = h4d.Context(h4d.make_params(cfg), rs, seed=99)
        ctx.h4d_run_md(40)
        ctx.h4d_run_trials(3, cfg["n_eq"])
        ctx.h4d_set_mu(-1.0e8)
        ctx.h4d_run_trials(3, cfg["n_eq"])
        out = [(ctx.h4d_get_work(r, 6), ctx.h4d_get_state(r), ctx.h4d_get_counts(r)["n_water"]) for r in range(len(rs))]
        ctx.close()
        return out

    packed = run(reps)
    moved = 0
    for k in range(0, len(reps), 3):
        alone = run([reps[k]])[0]
        wp, (xp, vp), nwp = packed[k]
        wa, (xa, va), nwa = alone
        assert wp.tobytes() == wa.tobytes(), k
        assert nwp == nwa and np.array_equal(xp, xa) and np.array_equal(vp, va), k
        moved += int(wp["accepted"].sum())
    assert moved > 0  # layouts did change
