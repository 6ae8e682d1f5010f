"""ctypes binding of the FP64 CPU oracle (h4d_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()`` and by the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The GPU library never
imports this module and this module never imports the GPU library.

Every function takes plain numpy arrays; configurations are the parameter dictionaries
of ``paper_2307_11447_gb300.workloads`` (parameter values and seeded inputs only).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "h4d_oracle.c")
_HDR = os.path.join(_HERE, "h4d_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

MAXT = 4
SCHED = {"linear": 0, "wv": 1, "wx": 2}


_LIB32 = os.path.join(_HERE, "liboracle_fp32.so")


def build(force: bool = False, fp32_forces: bool = False) -> str:
    """Compile the oracle with the host C compiler (no GPU, no CUDA).  fp32_forces builds
    the tolerance-derivation variant whose dynamics use binary32 pair forces."""
    out = _LIB32 if fp32_forces else _LIB
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
        tmp = out + f".tmp{os.getpid()}"
        defs = ["-DORC_FP32_FORCES"] if fp32_forces else []
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", *defs, "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, out)
    return out


class fp32_forces:
    """context manager: oracle calls inside use the binary32-pair-force build"""

    def __enter__(self):
        global _lib, _lib_path
        self._saved = (_lib, _lib_path)
        _lib, _lib_path = None, build(fp32_forces=True)
        return self

    def __exit__(self, *exc):
        global _lib, _lib_path
        _lib, _lib_path = self._saved
        return False


class Params(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("beta_mu", ctypes.c_double),
        ("rc_lj", ctypes.c_double),
        ("rc_coul", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("kcoul", ctypes.c_double),
        ("kappa_sr", ctypes.c_double),
        ("ntypes", ctypes.c_int32),
        ("pad0", ctypes.c_int32),
        ("q", ctypes.c_double * MAXT),
        ("sig", ctypes.c_double * MAXT),
        ("eps", ctypes.c_double * MAXT),
        ("mass", ctypes.c_double * MAXT),
        ("mvv2e", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("w_max", ctypes.c_double),
        ("tau_t", ctypes.c_double),
        ("n_f", ctypes.c_int32),
        ("schedule", ctypes.c_int32),
        ("sched_n", ctypes.c_double),
        ("d_oh", ctypes.c_double),
        ("d_hh", ctypes.c_double),
        ("n_water", ctypes.c_int32),
        ("use_cells", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("replica", ctypes.c_uint64),
        ("bias_alpha", ctypes.c_double),
        ("bias_xb", ctypes.c_double),
        ("fw", ctypes.c_double),
        ("v_ex", ctypes.c_double),
        ("no_accept", ctypes.c_int32),
        ("single", ctypes.c_int32),
        ("water_ex", ctypes.c_int32),
        ("pad_w", ctypes.c_int32),
    ]


class _State(ctypes.Structure):
    _fields_ = [
        ("n_pairs", ctypes.c_int32),
        ("cap_pairs", ctypes.c_int32),
        ("x", ctypes.POINTER(ctypes.c_double)),
        ("v", ctypes.POINTER(ctypes.c_double)),
        ("trial_ctr", ctypes.c_uint64),
        ("step_ctr", ctypes.c_uint64),
        ("n_water", ctypes.c_int32),
        ("cap_water", ctypes.c_int32),
    ]


RECORD_DTYPE = np.dtype(
    [
        ("move", np.int32),
        ("accepted", np.int32),
        ("n_before", np.int32),
        ("n_after", np.int32),
        ("status", np.int32),
        ("cation", np.int32),
        ("anion", np.int32),
        ("cell_c", np.int32),
        ("cell_a", np.int32),
        ("instant", np.int32),
        ("dH", np.float64),
        ("beta_dM", np.float64),
        ("w_prot", np.float64),
        ("ln_u", np.float64),
        ("x_acc", np.float64),
        ("ln_q", np.float64),
    ]
)
PROP_NW = 96 * 64 + 64 + 64 * 64 + 64 + 64 * 2 + 2


class Proposal(ctypes.Structure):
    """learned insertion-site proposal (mode 0 uniform, 1 learned); keeps its weights alive"""
    _fields_ = [
        ("mode", ctypes.c_int32),
        ("G", ctypes.c_int32),
        ("bf16", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("eps", ctypes.c_double),
        ("w", ctypes.POINTER(ctypes.c_double)),
    ]


def make_proposal(G: int, weights=None, eps: float = 0.1, bf16: bool = True) -> Proposal:
    q = Proposal()
    q.G = int(G)
    q.eps = float(eps)
    q.bf16 = int(bf16)
    if weights is None:
        q.mode = 0
        q._w = np.zeros(PROP_NW)
    else:
        q.mode = 1
        q._w = np.ascontiguousarray(weights, np.float64)
        assert q._w.size == PROP_NW
    q.w = _ptr(q._w)
    return q

_lib = None
_lib_path = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_lib_path or build())
        d = ctypes.c_double
        pd = ctypes.POINTER(ctypes.c_double)
        pu8 = ctypes.POINTER(ctypes.c_uint8)
        pi32 = ctypes.POINTER(ctypes.c_int32)
        pu64 = ctypes.POINTER(ctypes.c_uint64)
        P = ctypes.POINTER(Params)
        S = ctypes.POINTER(_State)
        _lib.orc_philox4x64_10.argtypes = [pu64, pu64, pu64]
        _lib.orc_pair.argtypes = [P, ctypes.c_int, ctypes.c_int, d, d, pd, pd]
        _lib.orc_energy_forces.argtypes = [P, ctypes.c_int, pd, pd, pu8, pd]
        _lib.orc_energy_forces.restype = d
        _lib.orc_neighbor_pairs.argtypes = [ctypes.c_int, pd, d, d, pi32, pi32, ctypes.c_int64]
        _lib.orc_neighbor_pairs.restype = ctypes.c_int64
        _lib.orc_altitude.argtypes = [P, ctypes.c_int, ctypes.c_int]
        _lib.orc_altitude.restype = d
        _lib.orc_kinetic.argtypes = [P, ctypes.c_int, pd, pu8]
        _lib.orc_kinetic.restype = d
        _lib.orc_nve.argtypes = [P, S, ctypes.c_int64, pd]
        _lib.orc_nve.restype = d
        _lib.orc_md.argtypes = [P, S, ctypes.c_int64]
        _lib.orc_nemd_path.argtypes = [P, S, pi32, ctypes.c_int, ctypes.c_int, pd]
        _lib.orc_nemd_path.restype = d
        _lib.orc_trial.argtypes = [P, S, ctypes.c_void_p]
        _lib.orc_run_cycles.argtypes = [P, S, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
        _lib.orc_init_velocities.argtypes = [P, S]
        _lib.orc_atom_type.argtypes = [P, ctypes.c_int]
        _lib.orc_bias_density.argtypes = [d, d, d, d]
        _lib.orc_bias_density.restype = d
        _lib.orc_erfinv.argtypes = [d]
        _lib.orc_erfinv.restype = d
        _lib.orc_bias_offset.argtypes = [d, d, d, ctypes.c_uint64, ctypes.c_uint64]
        _lib.orc_bias_offset.restype = d
        Q = ctypes.POINTER(Proposal)
        _lib.orc_proposal_features.argtypes = [P, ctypes.c_int, ctypes.c_int, pd, ctypes.c_int, ctypes.c_int, pd]
        _lib.orc_proposal_logits.argtypes = [P, Q, ctypes.c_int, pd, ctypes.c_int, ctypes.c_int, pd]
        _lib.orc_trial_prop.argtypes = [P, Q, S, ctypes.c_void_p, pd, pd]
        _lib.orc_in_excluded_volume.argtypes = [P, pd, pd]
        _lib.orc_in_excluded_volume.restype = ctypes.c_int
        _lib.orc_run_cycles_prop.argtypes = [P, Q, S, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
        _lib.orc_ewald.argtypes = [P, ctypes.c_int, pd, d, ctypes.c_int, d, pd, pd, pd, pd, pd]
        _lib.orc_ewald.restype = d
    return _lib


def _ptr(a, ct=ctypes.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ct))


def make_params(cfg: dict, **override) -> Params:
    """Build the oracle's parameter block from a workload dictionary."""
    c = dict(cfg)
    c.update(override)
    p = Params()
    p.L = float(c["L"])
    p.beta = float(c["beta"])
    p.beta_mu = float(c.get("beta_mu", 0.0))
    p.rc_lj = float(c["rc_lj"])
    p.rc_coul = float(c["rc_coul"])
    p.alpha = float(c["alpha"])
    p.kcoul = float(c["kcoul"])
    p.kappa_sr = float(c.get("kappa_sr", 0.0))
    p.ntypes = len(c["q"])
    for k in range(len(c["q"])):
        p.q[k] = c["q"][k]
        p.sig[k] = c["sig"][k]
        p.eps[k] = c["eps"][k]
        p.mass[k] = c["mass"][k]
    p.mvv2e = float(c.get("mvv2e", 1.0))
    p.dt = float(c["dt"])
    p.w_max = float(c["w_max"])
    p.tau_t = float(c.get("tau_t", 0.0))
    p.n_f = int(c["n_f"])
    p.schedule = SCHED[c.get("schedule", "linear")] if isinstance(c.get("schedule", "linear"), str) else int(c["schedule"])
    p.sched_n = float(c.get("sched_n", 1.0))
    p.d_oh = float(c.get("d_oh", 0.0))
    p.d_hh = float(c.get("d_hh", 0.0))
    p.n_water = int(c.get("n_water", 0))
    p.use_cells = int(c.get("use_cells", 0))
    p.seed = int(c.get("seed", 0))
    p.replica = int(c.get("replica", 0))
    p.bias_alpha = float(c.get("bias_alpha", 0.0))
    p.bias_xb = float(c.get("bias_xb", 0.0))
    p.fw = float(c.get("fw", 0.0))
    p.v_ex = float(c.get("v_ex", 0.0))
    p.no_accept = int(bool(c.get("no_accept", 0)))
    p.single = int(c.get("exchange", "pair") == "single")
    p.water_ex = int(c.get("exchange", "pair") == "water")
    return p


class State:
    """A chain's state: positions and velocities of 3*n_water + 2*cap_pairs atoms (one atom
    per unit instead of two with single-particle exchange).  With water exchange the
    number of waters starts at p.n_water and varies up to cap_water."""

    def __init__(self, p: Params, x: np.ndarray, v: np.ndarray | None, n_pairs: int, cap_pairs: int,
                 cap_water: int | None = None):
        self.unit = 1 if p.single else 2
        self.water_ex = bool(p.water_ex)
        cap_w = p.n_water if cap_water is None else int(cap_water)
        if cap_w < p.n_water:
            raise ValueError("cap_water below the number of waters")
        n_cap = 3 * cap_w + self.unit * cap_pairs
        self.x = np.zeros((n_cap, 3), np.float64)
        self.v = np.zeros((n_cap, 3), np.float64)
        n = 3 * p.n_water + self.unit * n_pairs
        self.x[:n] = np.asarray(x, np.float64).reshape(-1, 3)[:n]
        if v is not None:
            self.v[:n] = np.asarray(v, np.float64).reshape(-1, 3)[:n]
        self.s = _State()
        self.s.n_pairs = n_pairs
        self.s.cap_pairs = cap_pairs
        self.s.x = _ptr(self.x)
        self.s.v = _ptr(self.v)
        self.s.trial_ctr = 0
        self.s.step_ctr = 0
        self.s.n_water = p.n_water
        self.s.cap_water = cap_w
        self._n_water = p.n_water

    @property
    def n_water(self) -> int:
        return self.s.n_water if self.water_ex else self._n_water

    @property
    def n_pairs(self) -> int:
        return self.s.n_pairs

    @property
    def n_atoms(self) -> int:
        return 3 * self.n_water + self.unit * self.s.n_pairs

    def positions(self) -> np.ndarray:
        return self.x[: self.n_atoms].copy()

    def velocities(self) -> np.ndarray:
        return self.v[: self.n_atoms].copy()


def philox(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, np.uint64)
    k = np.asarray(key, np.uint64)
    out = np.zeros(4, np.uint64)
    lib().orc_philox4x64_10(_ptr(c, ctypes.c_uint64), _ptr(k, ctypes.c_uint64), _ptr(out, ctypes.c_uint64))
    return out


def pair(p: Params, ti: int, tj: int, r4: float, g: float = 1.0):
    u = ctypes.c_double()
    du = ctypes.c_double()
    lib().orc_pair(ctypes.byref(p), ti, tj, r4, g, ctypes.byref(u), ctypes.byref(du))
    return u.value, du.value


def energy_forces(p: Params, x: np.ndarray, w: np.ndarray | None = None, fly: np.ndarray | None = None):
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    n = x.shape[0]
    F = np.zeros((n, 3), np.float64)
    wa = None if w is None else np.ascontiguousarray(w, np.float64)
    fa = None if fly is None else np.ascontiguousarray(fly, np.uint8)
    U = lib().orc_energy_forces(ctypes.byref(p), n, _ptr(x), _ptr(wa), _ptr(fa, ctypes.c_uint8), _ptr(F))
    return U, F


def neighbor_pairs(x: np.ndarray, L: float, r_list: float):
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    n = x.shape[0]
    m = lib().orc_neighbor_pairs(n, _ptr(x), L, r_list, None, None, 0)
    oi = np.zeros(max(m, 1), np.int32)
    oj = np.zeros(max(m, 1), np.int32)
    lib().orc_neighbor_pairs(n, _ptr(x), L, r_list, _ptr(oi, ctypes.c_int32), _ptr(oj, ctypes.c_int32), m)
    return oi[:m], oj[:m]


def in_excluded_volume(p: Params, xc, xa) -> bool:
    """early rejection: whether the anion at xa lies in the excluded cube on the cation at xc"""
    xc = np.ascontiguousarray(xc, np.float64)
    xa = np.ascontiguousarray(xa, np.float64)
    return bool(lib().orc_in_excluded_volume(ctypes.byref(p), _ptr(xc), _ptr(xa)))


def altitude(p: Params, insertion: bool, k: int) -> float:
    return lib().orc_altitude(ctypes.byref(p), int(insertion), int(k))


def kinetic(p: Params, v: np.ndarray, fly: np.ndarray | None = None) -> float:
    v = np.ascontiguousarray(v, np.float64).reshape(-1, 3)
    fa = None if fly is None else np.ascontiguousarray(fly, np.uint8)
    return lib().orc_kinetic(ctypes.byref(p), v.shape[0], _ptr(v), _ptr(fa, ctypes.c_uint8))


def nve(p: Params, st: State, n_steps: int, trace: bool = False):
    tr = np.zeros(n_steps, np.float64) if trace else None
    U = lib().orc_nve(ctypes.byref(p), ctypes.byref(st.s), n_steps, _ptr(tr))
    return (U, tr) if trace else U


def md(p: Params, st: State, n_steps: int) -> None:
    lib().orc_md(ctypes.byref(p), ctypes.byref(st.s), n_steps)


def nemd_path(p: Params, st: State, flyers, insertion: bool):
    f = np.ascontiguousarray(flyers, np.int32)
    U = ctypes.c_double()
    w = lib().orc_nemd_path(ctypes.byref(p), ctypes.byref(st.s), _ptr(f, ctypes.c_int32), f.size, int(insertion), ctypes.byref(U))
    return w, U.value


def trial(p: Params, st: State) -> np.ndarray:
    rec = np.zeros(1, RECORD_DTYPE)
    lib().orc_trial(ctypes.byref(p), ctypes.byref(st.s), rec.ctypes.data)
    return rec[0]


def run_cycles(p: Params, st: State, n_cycles: int, n_eq: int) -> np.ndarray:
    recs = np.zeros(n_cycles, RECORD_DTYPE)
    lib().orc_run_cycles(ctypes.byref(p), ctypes.byref(st.s), n_cycles, n_eq, recs.ctypes.data)
    return recs


def init_velocities(p: Params, st: State) -> None:
    lib().orc_init_velocities(ctypes.byref(p), ctypes.byref(st.s))


def atom_type(p: Params, a: int) -> int:
    return lib().orc_atom_type(ctypes.byref(p), a)


def proposal_features(p: Params, G: int, x: np.ndarray, exclude=(-1, -1)) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    out = np.zeros((G**3, 96), np.float64)
    lib().orc_proposal_features(ctypes.byref(p), G, x.shape[0], _ptr(x), int(exclude[0]), int(exclude[1]), _ptr(out))
    return out


def proposal_logits(p: Params, q: Proposal, x: np.ndarray, exclude=(-1, -1)) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    out = np.zeros((q.G**3, 2), np.float64)
    lib().orc_proposal_logits(ctypes.byref(p), ctypes.byref(q), x.shape[0], _ptr(x), int(exclude[0]),
                              int(exclude[1]), _ptr(out))
    return out


def trial_prop(p: Params, q: Proposal | None, st: State, want_site: bool = False):
    """one trial with the proposal q; with want_site also the move's training record
    (features [2, 96] of the cation and anion cells, insertion-direction exponent)"""
    rec = np.zeros(1, RECORD_DTYPE)
    feat = np.zeros((2, 96), np.float64) if want_site else None
    y = np.zeros(1, np.float64) if want_site else None
    lib().orc_trial_prop(ctypes.byref(p), None if q is None else ctypes.byref(q), ctypes.byref(st.s),
                         rec.ctypes.data, _ptr(feat), _ptr(y))
    return (rec[0], feat, float(y[0])) if want_site else rec[0]


def run_cycles_prop(p: Params, q: Proposal | None, st: State, n_cycles: int, n_eq: int) -> np.ndarray:
    recs = np.zeros(n_cycles, RECORD_DTYPE)
    lib().orc_run_cycles_prop(ctypes.byref(p), None if q is None else ctypes.byref(q), ctypes.byref(st.s),
                              n_cycles, n_eq, recs.ctypes.data)
    return recs


def bias_density(alpha, xb, L, x):
    return lib().orc_bias_density(alpha, xb, L, x)


def erfinv(y):
    return lib().orc_erfinv(y)


def bias_offset(alpha, xb, L, r_mode, r_u):
    return lib().orc_bias_offset(alpha, xb, L, int(r_mode), int(r_u))


def ewald(p: Params, x: np.ndarray, alpha: float, kmax: int, rcut: float, forces: bool = False):
    """Ewald sum of the periodic Coulomb energy: dict with U (total), real, recip, self,
    excl and, when asked, the reciprocal-space forces [n, 3]"""
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    n = x.shape[0]
    parts = [ctypes.c_double() for _ in range(4)]
    F = np.zeros((n, 3)) if forces else None
    U = lib().orc_ewald(ctypes.byref(p), n, _ptr(x), alpha, int(kmax), rcut, *[ctypes.byref(v) for v in parts], _ptr(F))
    out = {"U": U, "real": parts[0].value, "recip": parts[1].value, "self": parts[2].value, "excl": parts[3].value}
    if forces:
        out["F_recip"] = F
    return out
