"""Early rejection (SI, "Simple, early rejection scheme") on the GPU against the oracle.

Single trials from one equilibrated state of the 250-ion electrolyte with an excluded cube
of edge 0.6 L, so that both kinds of move occur in both directions.  Tolerances: the move,
its classification (the cube is judged on identical fixed-point coordinates) and the pair
identical; an instantaneous move has no protocol work and its beta dM is a difference of
FP64 energies of identical fixed-point states on both sides (1e-9 relative); NEMD trials as
in the other trial tests (1e-3 kT within 20 kT of the acceptance boundary, 1e-3 relative
beyond it); decisions identical away from ties.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2307_11447_gb300 import lib as h4d

from .test_gpu_proposal import _lj_state, work_close

pytestmark = pytest.mark.gpu


def test_early_rejection_trials_match_oracle():
    cfg, _, x0, v0 = _lj_state(2)
    L, n_pairs = cfg["L"], cfg["n_pairs"]
    cfg.update(v_ex=(0.6 * L) ** 3)
    po = orc.make_params(cfg, use_cells=0)
    ctx = h4d.Context(h4d.make_params(cfg), [dict(L=L, n_pairs=n_pairs, cap_pairs=cfg["cap_pairs"], x=x0, v=v0)],
                      seed=cfg["seed"])
    ctx.h4d_set_early_rejection(cfg["v_ex"])
    kinds = set()
    for k in range(24):
        ctx.h4d_set_state(0, n_pairs, x0, v0)
        ctx.h4d_run_trials(1, 0)
        rg = ctx.h4d_get_work(0, 1)[0]
        st = orc.State(po, x0, v0, n_pairs, cfg["cap_pairs"])
        st.s.trial_ctr = k
        ro = orc.trial(po, st)
        print(f"trial {k}: move {ro['move']} instant gpu {rg['instant']} oracle {ro['instant']} "
              f"beta dM gpu {rg['beta_dM']:.9g} oracle {ro['beta_dM']:.9g}")
        assert rg["move"] == ro["move"] and rg["status"] == ro["status"] == 0
        assert rg["instant"] == ro["instant"]
        assert rg["cation"] == ro["cation"] and rg["anion"] == ro["anion"]
        kinds.add((int(ro["move"]), int(ro["instant"])))
        if ro["instant"]:
            assert rg["w_prot"] == 0.0
            assert abs(rg["beta_dM"] - ro["beta_dM"]) <= 1e-9 * (1.0 + abs(ro["beta_dM"]))
        else:
            assert work_close(rg["beta_dM"], ro["beta_dM"], ro["x_acc"]), (k, rg["beta_dM"], ro["beta_dM"])
        if abs(ro["ln_u"] - ro["x_acc"]) > 1e-3:
            assert rg["accepted"] == ro["accepted"]
    assert kinds == {(0, 0), (0, 1), (1, 0), (1, 1)}, kinds


def test_early_rejection_off_by_default_and_rejects_bad_volumes():
    cfg, _, x0, v0 = _lj_state(2)
    L, n_pairs = cfg["L"], cfg["n_pairs"]
    ctx = h4d.Context(h4d.make_params(cfg), [dict(L=L, n_pairs=n_pairs, cap_pairs=cfg["cap_pairs"], x=x0, v=v0)],
                      seed=cfg["seed"])
    ctx.h4d_run_trials(8, 0)
    assert np.all(ctx.h4d_get_work(0, 8)["instant"] == 0)
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(h4d.H4DError):
            ctx.h4d_set_early_rejection(bad)
    ctx.h4d_set_early_rejection(0.0)
