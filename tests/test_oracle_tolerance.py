"""How far binary32 pair forces alone move the work of a trial.

The GPU integrates NEMD trajectories with FP32 pair forces (FP64 energies and work sums).
The oracle's tolerance-derivation build (liboracle_fp32.so, same source compiled with
ORC_FP32_FORCES) evaluates exactly those forces in binary32 and keeps everything else in
FP64.  Its trials against the FP64 build's show the spread that the per-trial work
tolerance of the GPU tests has to cover: the median trial moves by a few 1e-6 kT, but a
few per cent of trials jump by 2e-4 to 8e-4 kT (discrete events: a pair whose distance
sits within binary32 rounding of a cut-off, where the truncated forces jump, is counted
in a different step).  Hence the GPU criterion: every trial within 1e-3 kT of the oracle,
the median within 2e-5 kT.  CPU only."""
import numpy as np

from oracle import oracle as orc
from paper_2307_11447_gb300 import workloads as wl

TWO32 = 4294967296.0


def quantize(x, L):
    y = np.mod(x, L)
    return np.mod(np.rint(y / L * TWO32), TWO32) * (L / TWO32)


def _state(seed):
    cfg = dict(wl.CONFIGS["lj250"])
    cfg.update(seed=seed, replica=0, beta_mu=-8.0, n_f=30)
    L = cfg["L"]
    po = orc.make_params(cfg, use_cells=0)
    st = orc.State(po, quantize(wl.lj_positions(cfg["n_pairs"], L, seed), L), None, cfg["n_pairs"], cfg["cap_pairs"])
    orc.init_velocities(po, st)
    orc.md(po, st, 200)
    return cfg, po, quantize(st.positions(), L), st.velocities()


def _trials(cfg, po, x0, v0, k):
    out = []
    for t in range(k):
        st = orc.State(po, x0, v0, cfg["n_pairs"], cfg["cap_pairs"])
        st.s.trial_ctr = t
        out.append(orc.trial(po, st))
    return out


def test_fp32_pair_forces_alone_move_trial_work_by_up_to_1e_3_kT():
    devs = []
    for seed in (1, 6):
        cfg, po, x0, v0 = _state(seed)
        a = _trials(cfg, po, x0, v0, 6)
        with orc.fp32_forces():
            b = _trials(cfg, po, x0, v0, 6)
        for ra, rb in zip(a, b):
            assert ra["move"] == rb["move"]
            if abs(ra["x_acc"]) < 20:
                devs.append(abs(ra["beta_dM"] - rb["beta_dM"]))
    devs = np.array(devs)
    print("FP32-force work deviations (kT):", np.array2string(devs, precision=2))
    assert np.median(devs) < 2e-5
    assert devs.max() > 1e-4  # FP32 forces alone exceed 1e-4 kT on some trials ...
    assert devs.max() < 1e-3  # ... and stay inside the 1e-3 kT GPU tolerance
