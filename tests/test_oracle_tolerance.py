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


def test_fp64_trajectory_can_put_a_pair_within_binary32_rounding_of_the_cutoff():
    """the mechanism behind the jumps: 11 NVE steps from the seed-6 state bring ions 24 and
    54 to 1.1e-7 sigma inside the Coulomb cut-off (4 sigma) -- closer than binary32 resolves
    r^2 = 16 (one ulp is 9.5e-7 below 16) -- so an FP32 force pass may count the pair a step
    later than FP64 does; the missed force jump, 0.05 kT/sigma, costs about 2.9e-4 kT"""
    cfg, po, x0, v0 = _state(6)
    L = cfg["L"]
    p0 = orc.make_params(dict(cfg, tau_t=0.0), use_cells=0)
    st = orc.State(p0, x0, v0, cfg["n_pairs"], cfg["cap_pairs"])
    orc.nve(p0, st, 11)
    x = st.positions()
    d = x[54] - x[24]
    d -= L * np.round(d / L)
    r = float(np.sqrt(d @ d))
    print(f"r(24, 54) after 11 steps = 4 - {4.0 - r:.3e}")
    assert 0.0 < 4.0 - r < 2e-7
    assert np.float32(r * r) >= np.float32(16.0) - np.spacing(np.float32(16.0))


def _c1_pair(args):
    x0, v0, cfg, k = args
    out = []
    for fp32 in (False, True):
        if fp32:
            with orc.fp32_forces():
                po = orc.make_params(cfg, use_cells=1)
                st = orc.State(po, x0, v0, cfg["n_pairs"], cfg["cap_pairs"])
                st.s.trial_ctr = k
                out.append(float(orc.trial(po, st)["beta_dM"]))
        else:
            po = orc.make_params(cfg, use_cells=1)
            st = orc.State(po, x0, v0, cfg["n_pairs"], cfg["cap_pairs"])
            st.s.trial_ctr = k
            out.append(float(orc.trial(po, st)["beta_dM"]))
    return out


def test_fp32_forces_move_long_protocol_work_by_hundredths_of_kT():
    """The 4000-ion, 500-step configuration: binary32 pair forces alone move the work of a
    trial by 1e-3 to a few 1e-2 kT (chaotic divergence over 2.5 tau plus cut-off events
    among 4000 ions), which is why that configuration's per-trial work is reported and
    held only to 0.1 kT on the GPU"""
    import multiprocessing as mp

    cfg = dict(wl.CONFIGS["lj4000"])
    cfg.update(seed=9, replica=0, beta_mu=-6.0)
    L = cfg["L"]
    po = orc.make_params(cfg, use_cells=1)
    st = orc.State(po, quantize(wl.lj_positions(cfg["n_pairs"], L, 9), L), None, cfg["n_pairs"], cfg["cap_pairs"])
    orc.init_velocities(po, st)
    orc.md(po, st, 200)
    x0, v0 = quantize(st.positions(), L), st.velocities()
    with mp.get_context("spawn").Pool(4) as pool:
        res = pool.map(_c1_pair, [(x0, v0, cfg, k) for k in range(4)])
    devs = np.array([abs(b - a) for a, b in res])
    print("C1 FP32-force work deviations (kT):", np.array2string(devs, precision=4))
    assert devs.max() > 1e-3
    assert devs.max() < 0.05
