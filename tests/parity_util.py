"""Helpers for GPU-vs-oracle force parity.

The pair potential is shifted in energy but not in force at each cut-off (reading of
Eqs. 19-20), so the force jumps by |u'(r_c)| there.  A pair whose distance lies within a
relative 1e-6 of a cut-off can be classified differently by the FP32 kernel and the FP64
oracle; for such pairs the per-atom allowance adds that jump.  Everything else must agree
to 1e-5 (|F| + F_rms).
"""
import math

import numpy as np

from oracle import oracle as orc


def _jumps(cfg):
    p = orc.make_params(cfg)
    nt = len(cfg["q"])
    out = {}
    for rc, lj in ((cfg["rc_lj"], True), (cfg["rc_coul"], False)):
        for ti in range(nt):
            for tj in range(nt):
                over = dict(q=[0.0] * nt) if lj else dict(eps=[0.0] * nt)
                pp = orc.make_params(dict(cfg, **over))
                _, du = orc.pair(pp, ti, tj, rc * (1.0 - 1e-12))
                out[(rc, ti, tj)] = abs(du)
    return out


def force_bounds(cfg, x, Fo, w=None, rel=1e-5, band=1e-6):
    """per-atom bound |dF_i| <= rel (|F_i| + F_rms) + sum of cut-off jumps of boundary pairs"""
    x = np.asarray(x)
    n = len(x)
    L = cfg["L"]
    p = orc.make_params(cfg)
    types = np.array([orc.atom_type(p, a) for a in range(n)])
    frms = math.sqrt((Fo**2).sum(1).mean())
    bound = rel * (np.linalg.norm(Fo, axis=1) + frms)
    jumps = _jumps(cfg)
    ww = np.zeros(n) if w is None else np.asarray(w)
    for rc in {cfg["rc_lj"], cfg["rc_coul"]}:
        for i in range(n):
            d = x - x[i]
            d -= L * np.round(d / L)
            r = np.sqrt((d * d).sum(1) + (ww - ww[i]) ** 2)
            near = np.nonzero(np.abs(r - rc) < band * rc)[0]
            for j in near:
                if j != i:
                    bound[i] += jumps.get((rc, types[i], types[j]), 0.0)
    return bound


def trial_work_bound(beta_dM, x_acc):
    """Allowed |beta dM_gpu - beta dM_oracle| of one trial (kT).  Near the acceptance
    boundary (|x| < 20): 1e-3, the spread of the oracle's own binary32-force build
    (tests/test_oracle_tolerance.py).  Farther out: 1e-3 + 1e-3 |beta dM|.  Trials that
    exchange more than 1e4 kT are insertions onto overlaps, driven by forces beyond 1e10
    whose FP32 rounding the dynamics amplify: 1e-2 |beta dM| (the binary32-force oracle
    moves one such trial of the 250-ion electrolyte, beta dM = 4.2e6, by 5.2e-4 relative);
    their decision is certain either way."""
    if abs(x_acc) < 20:
        return 1e-3
    if abs(beta_dM) < 1e4:
        return 1e-3 + 1e-3 * abs(beta_dM)
    return 1e-2 * abs(beta_dM)
