"""Failure reporting of the engine, provoked from the host with inputs that stay in bounds
(no GPU fault, trap or hang is involved: every device loop is bounded and every index is
clamped or checked).

* Neighbour rows too short for the density (max_nbr 128, the smallest capacity the row
  layout allows, for an electrolyte at density 0.9 with some 300 atoms inside r_list):
  equilibrium MD raises error bit 0 and the getters return H4D_ECAPACITY; inside NEMD the
  same overflow rejects the trial with status 3 instead.
* Two atoms placed almost on top of each other: the equilibrium-MD state becomes
  non-finite (bit 1, H4D_ENAN).
* Rigid waters driven so fast that SHAKE cannot restore the bonds in its 100 iterations:
  bit 2, H4D_ETIMEOUT (a bounded loop gave up).
* A fresh state (h4d_set_state) clears the flags.
"""
import numpy as np
import pytest

from paper_2307_11447_gb300 import lib as h4d
from paper_2307_11447_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _lj(max_nbr=0, dense=False, **kw):
    cfg = dict(wl.lj_config(1000, 0.9, 20, cap_pairs=520) if dense else wl.CONFIGS["lj250"])
    cfg.update(max_nbr=max_nbr, **kw)
    x = wl.lj_positions(cfg["n_pairs"], cfg["L"], 5)
    return cfg, h4d.Context(h4d.make_params(cfg), [dict(L=cfg["L"], n_pairs=cfg["n_pairs"], cap_pairs=cfg["cap_pairs"], x=x)],
                            seed=3), x


def test_row_overflow_reports_capacity_and_rejects_nemd_trials():
    cfg, ctx, x = _lj(max_nbr=128, dense=True)
    ctx.h4d_run_md(5)
    with pytest.raises(h4d.H4DError) as e:
        ctx.h4d_get_energies(0)
    assert e.value.code == h4d.H4D_ECAPACITY
    assert ctx.h4d_get_counts(0)["error_flags"] & 1
    # a trial whose rows overflow is rejected with status 3 (no error flag of its own)
    ctx.h4d_set_state(0, cfg["n_pairs"], x, None)
    assert ctx.h4d_get_counts(0)["error_flags"] == 0
    ctx.h4d_run_trials(4, 0)
    rec = ctx.h4d_get_work(0, 4)
    assert np.all(rec["status"] == 3) and rec["accepted"].sum() == 0
    assert ctx.h4d_get_counts(0)["rejected_status"] >= 4
    ctx.close()


def test_overlapping_atoms_report_non_finite_state():
    cfg, ctx, x = _lj()
    y = x.copy()
    y[1] = y[0] + np.array([0.02, 0.0, 0.0])  # 0.02 sigma apart
    ctx.h4d_set_state(0, cfg["n_pairs"], y, None)
    ctx.h4d_run_md(5)
    with pytest.raises(h4d.H4DError) as e:
        ctx.h4d_get_energies(0)
    assert e.value.code == h4d.H4D_ENAN
    assert ctx.h4d_get_counts(0)["error_flags"] & 2
    ctx.h4d_set_state(0, cfg["n_pairs"], x, None)  # a good state clears the flags
    ctx.h4d_run_md(5)
    U, K = ctx.h4d_get_energies(0)
    assert np.isfinite(U) and np.isfinite(K)
    ctx.close()


def test_unconverged_shake_reports_timeout():
    cfg = wl.aq_config(300, 2, 22.5, 50, tau_t=0.0)
    x = wl.aqueous_positions(300, 2, 22.5, 8)
    rng = np.random.default_rng(2)
    v = rng.normal(size=x.shape) * 0.004
    h = np.zeros(len(x), bool)
    h[: 900] = np.arange(900) % 3 != 0
    v[h] = rng.normal(size=(h.sum(), 3)) * 3.0  # 3 A/fs hydrogens: bonds cannot be restored
    ctx = h4d.Context(h4d.make_params(cfg), [dict(L=22.5, n_pairs=2, cap_pairs=4, x=x, v=v, n_water=300)], seed=4)
    ctx.h4d_run_md(1)
    with pytest.raises(h4d.H4DError) as e:
        ctx.h4d_get_energies(0)
    assert e.value.code == h4d.H4D_ETIMEOUT
    assert ctx.h4d_get_counts(0)["error_flags"] & 4
    ctx.close()
