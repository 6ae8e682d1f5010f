"""Thin ctypes binding of libh4d (include/h4d.h).  Argument marshalling only: every step
of the method runs in the library's CUDA kernels.  The functions keep the C names.

The library is built in-tree (``paper_2307_11447_gb300/build.py``); loading fails loudly
when it is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

H4D_OK = 0
H4D_EINVAL = -1
H4D_ECAPACITY = -2
H4D_ETIMEOUT = -3
H4D_ENAN = -4
H4D_ECUDA = -5
H4D_ENODEV = -6
H4D_SYS_LJ = 0
H4D_SYS_AQ = 1
SCHED = {"linear": 0, "wv": 1, "wx": 2}


class H4DError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {strerror(code)} ({code})")
        self.code = code


class h4d_params(ctypes.Structure):
    _fields_ = [
        ("system", ctypes.c_int32),
        ("ntypes", ctypes.c_int32),
        ("beta", ctypes.c_double),
        ("beta_mu", ctypes.c_double),
        ("rc_lj", ctypes.c_double),
        ("rc_coul", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("kcoul", ctypes.c_double),
        ("kappa_sr", ctypes.c_double),
        ("q", ctypes.c_double * 4),
        ("sig", ctypes.c_double * 4),
        ("eps", ctypes.c_double * 4),
        ("mass", ctypes.c_double * 4),
        ("mvv2e", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("w_max", ctypes.c_double),
        ("tau_t", ctypes.c_double),
        ("sched_n", ctypes.c_double),
        ("n_f", ctypes.c_int32),
        ("schedule", ctypes.c_int32),
        ("d_oh", ctypes.c_double),
        ("d_hh", ctypes.c_double),
        ("skin", ctypes.c_double),
        ("skin_outer", ctypes.c_double),
        ("max_nbr", ctypes.c_int32),
        ("threads_per_atom", ctypes.c_int32),
        ("exchange", ctypes.c_int32),
        ("pad_exchange", ctypes.c_int32),
    ]


class h4d_system(ctypes.Structure):
    _fields_ = [
        ("n_replicas", ctypes.c_int32),
        ("L", ctypes.POINTER(ctypes.c_double)),
        ("n_water", ctypes.POINTER(ctypes.c_int32)),
        ("n_pairs", ctypes.POINTER(ctypes.c_int32)),
        ("cap_pairs", ctypes.POINTER(ctypes.c_int32)),
        ("host_x", ctypes.POINTER(ctypes.c_double)),
        ("host_v", ctypes.POINTER(ctypes.c_double)),
        ("replica_key", ctypes.POINTER(ctypes.c_uint64)),
        ("cap_water", ctypes.POINTER(ctypes.c_int32)),
    ]


class h4d_counts(ctypes.Structure):
    _fields_ = [
        ("n_pairs", ctypes.c_int64),
        ("cycles", ctypes.c_int64),
        ("trials_ins", ctypes.c_int64),
        ("trials_del", ctypes.c_int64),
        ("accepted_ins", ctypes.c_int64),
        ("accepted_del", ctypes.c_int64),
        ("rejected_status", ctypes.c_int64),
        ("md_steps", ctypes.c_int64),
        ("sum_n", ctypes.c_double),
        ("sum_n2", ctypes.c_double),
        ("nbr_builds", ctypes.c_int64),
        ("error_flags", ctypes.c_int64),
        ("t_nemd_ns", ctypes.c_double),
        ("t_md_ns", ctypes.c_double),
        ("t_build_ns", ctypes.c_double),
        ("t_force_ns", ctypes.c_double),
        ("t_energy_ns", ctypes.c_double),
        ("threads_per_atom", ctypes.c_int64),
        ("nbr_refreshes", ctypes.c_int64),
        ("t_filter_ns", ctypes.c_double),
        ("last_smid", ctypes.c_int64),
        ("t_last_begin_ns", ctypes.c_double),
        ("t_last_end_ns", ctypes.c_double),
        ("plan_warps", ctypes.c_int64),
        ("plan_cta_groups", ctypes.c_int64),
        ("n_water", ctypes.c_int64),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


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
H4D_PROPOSAL_UNIFORM = 0
H4D_PROPOSAL_LEARNED = 1
H4D_PROP_NW = 96 * 64 + 64 + 64 * 64 + 64 + 64 * 2 + 2

_lib = None


def library_path() -> str:
    return _build.OUT


def lib():
    """Load libh4d (building it first when the sources are newer)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libh4d.so is missing; the CUDA library is required")
        L = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        pd = ctypes.POINTER(ctypes.c_double)
        pi32 = ctypes.POINTER(ctypes.c_int32)
        i32, i64, d = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sig = {
            "h4d_create": ([ctypes.POINTER(h4d_params), ctypes.POINTER(h4d_system), ctypes.c_uint64, vp, ctypes.POINTER(vp)], i32),
            "h4d_destroy": ([vp], None),
            "h4d_strerror": ([ctypes.c_int], ctypes.c_char_p),
            "h4d_set_mu": ([vp, d], i32),
            "h4d_set_protocol": ([vp, i32, d, d, d, i32], i32),
            "h4d_set_no_accept": ([vp, i32], i32),
            "h4d_set_bias": ([vp, d, d], i32),
            "h4d_set_early_rejection": ([vp, d], i32),
            "h4d_set_species_wmax": ([vp, d], i32),
            "h4d_run_md": ([vp, i64], i32),
            "h4d_run_trials": ([vp, i64, i32], i32),
            "h4d_get_counts": ([vp, i32, ctypes.POINTER(h4d_counts)], i32),
            "h4d_get_energies": ([vp, i32, pd, pd], i32),
            "h4d_get_work": ([vp, i32, vp, i64, ctypes.POINTER(i64)], i32),
            "h4d_get_state": ([vp, i32, pd, pd, i64, ctypes.POINTER(i64)], i32),
            "h4d_set_state": ([vp, i32, i32, pd, pd], i32),
            "h4d_set_water_state": ([vp, i32, i32, i32, pd, pd], i32),
            "h4d_num_replicas": ([vp], i32),
            "h4d_device_info": ([pi32, pi32, pi32], i32),
            "h4d_measure_fp32_peak": ([pd, pd], i32),
            "h4d_autotune": ([vp, i32, pd, pd], i32),
            "h4d_count_pairs": ([vp, ctypes.POINTER(i64)], i32),
            "h4d_save": ([vp, ctypes.c_char_p], i32),
            "h4d_load": ([vp, ctypes.c_char_p], i32),
            "h4d_eval_forces": ([ctypes.POINTER(h4d_params), d, i32, i32, pd, pd, pd, pd], i32),
            "h4d_eval_forces_static": ([ctypes.POINTER(h4d_params), d, i32, i32, pd, pd, pd, pd], i32),
            "h4d_neighbor_pairs": ([d, i32, pd, d, pi32, pi32, i64, ctypes.POINTER(i64)], i32),
            "h4d_ewald_lr": ([ctypes.POINTER(h4d_params), d, i32, i32, pd, d, i32, d, d, pd, pd, pd, pd], i32),
            "h4d_proposal": ([vp, i32, d, d, i32], i32),
            "h4d_proposal_set_weights": ([vp, pd, i64], i32),
            "h4d_proposal_get_weights": ([vp, pd, i64], i32),
            "h4d_proposal_records": ([vp, i32, vp, pd, pi32, pi32, i64, ctypes.POINTER(i64)], i32),
            "h4d_proposal_logits": ([vp, i32, vp, vp, i64, ctypes.POINTER(i64)], i32),
            "h4d_train_proposal": ([vp, i64, i32, d, d, ctypes.c_uint64, pd], i32),
            "h4d_proposal_grad": ([pd, i64, vp, vp, pd, pd], i32),
            "h4d_coulomb_poly": ([d, d, vp, pi32], i32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().h4d_strerror(code).decode()


def _ck(code: int, where: str):
    if code != H4D_OK:
        raise H4DError(code, where)


def _pd(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_params(cfg: dict, **override) -> h4d_params:
    c = dict(cfg)
    c.update(override)
    p = h4d_params()
    p.system = H4D_SYS_LJ if c.get("system", "lj") == "lj" else H4D_SYS_AQ
    p.ntypes = len(c["q"])
    p.beta = c["beta"]
    p.beta_mu = c.get("beta_mu", 0.0)
    p.rc_lj = c["rc_lj"]
    p.rc_coul = c["rc_coul"]
    p.alpha = c["alpha"]
    p.kcoul = c["kcoul"]
    p.kappa_sr = c.get("kappa_sr", 0.0)
    for k in range(p.ntypes):
        p.q[k] = c["q"][k]
        p.sig[k] = c["sig"][k]
        p.eps[k] = c["eps"][k]
        p.mass[k] = c["mass"][k]
    p.mvv2e = c.get("mvv2e", 1.0)
    p.dt = c["dt"]
    p.w_max = c["w_max"]
    p.tau_t = c.get("tau_t", 0.0)
    p.sched_n = c.get("sched_n", 1.0)
    p.n_f = c["n_f"]
    s = c.get("schedule", "linear")
    p.schedule = SCHED[s] if isinstance(s, str) else int(s)
    p.d_oh = c.get("d_oh", 0.0)
    p.d_hh = c.get("d_hh", 0.0)
    p.skin = c.get("skin", 0.3)
    p.skin_outer = c.get("skin_outer", 0.0)
    p.max_nbr = c.get("max_nbr", 0)
    p.threads_per_atom = c.get("threads_per_atom", 0)
    p.exchange = {"pair": 0, "single": 1, "water": 2}[c.get("exchange", "pair")]
    return p


class Context:
    """Owns an h4d_ctx.  Replicas: list of dicts with keys L, n_pairs, cap_pairs, x, v
    (optional), n_water (optional), cap_water (optional, water exchange: the most waters
    the replica may hold), key (optional: the replica's random-stream key, by default its
    index)."""

    def __init__(self, params: h4d_params, replicas: list, seed: int, stream: int | None = None):
        R = len(replicas)
        self.params = params
        L = np.array([r["L"] for r in replicas], np.float64)
        nw = np.array([r.get("n_water", 0) for r in replicas], np.int32)
        npair = np.array([r["n_pairs"] for r in replicas], np.int32)
        cap = np.array([r["cap_pairs"] for r in replicas], np.int32)
        capw = np.array([r.get("cap_water", r.get("n_water", 0)) for r in replicas], np.int32)
        xs = np.ascontiguousarray(np.concatenate([np.asarray(r["x"], np.float64).reshape(-1, 3) for r in replicas]))
        have_v = all(r.get("v") is not None for r in replicas)
        vs = np.ascontiguousarray(np.concatenate([np.asarray(r["v"], np.float64).reshape(-1, 3) for r in replicas])) if have_v else None
        s = h4d_system()
        s.n_replicas = R
        s.L = _pd(L)
        s.n_water = nw.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        s.n_pairs = npair.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        s.cap_pairs = cap.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        s.host_x = _pd(xs)
        s.host_v = _pd(vs)
        have_key = all(r.get("key") is not None for r in replicas)
        keys = np.array([int(r["key"]) for r in replicas], np.uint64) if have_key else None
        s.replica_key = keys.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)) if have_key else None
        s.cap_water = capw.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        h = ctypes.c_void_p()
        _ck(lib().h4d_create(ctypes.byref(params), ctypes.byref(s), seed, ctypes.c_void_p(stream or 0), ctypes.byref(h)), "h4d_create")
        self.h = h
        self.R = R
        unit = 1 if params.exchange == 1 else 2  # atoms per exchange unit
        self.cap_atoms = [3 * int(capw[i]) + unit * int(cap[i]) for i in range(R)]

    def close(self):
        if self.h:
            lib().h4d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def h4d_set_mu(self, beta_mu):
        _ck(lib().h4d_set_mu(self.h, beta_mu), "h4d_set_mu")

    def h4d_set_protocol(self, n_f, w_max, dt, kappa_sr, schedule=0):
        _ck(lib().h4d_set_protocol(self.h, n_f, w_max, dt, kappa_sr, schedule), "h4d_set_protocol")

    def h4d_set_species_wmax(self, f_w):
        _ck(lib().h4d_set_species_wmax(self.h, f_w), "h4d_set_species_wmax")

    def h4d_set_bias(self, alpha_b, x_b):
        _ck(lib().h4d_set_bias(self.h, alpha_b, x_b), "h4d_set_bias")

    def h4d_set_early_rejection(self, v_ex):
        _ck(lib().h4d_set_early_rejection(self.h, v_ex), "h4d_set_early_rejection")

    def h4d_set_no_accept(self, on):
        _ck(lib().h4d_set_no_accept(self.h, int(on)), "h4d_set_no_accept")

    def h4d_run_md(self, n_steps):
        _ck(lib().h4d_run_md(self.h, n_steps), "h4d_run_md")

    def h4d_run_trials(self, k_cycles, n_eq):
        _ck(lib().h4d_run_trials(self.h, k_cycles, n_eq), "h4d_run_trials")

    def h4d_get_counts(self, r=0) -> dict:
        c = h4d_counts()
        _ck(lib().h4d_get_counts(self.h, r, ctypes.byref(c)), "h4d_get_counts")
        return c.as_dict()

    def h4d_get_energies(self, r=0):
        U = ctypes.c_double()
        K = ctypes.c_double()
        _ck(lib().h4d_get_energies(self.h, r, ctypes.byref(U), ctypes.byref(K)), "h4d_get_energies")
        return U.value, K.value

    def h4d_get_work(self, r=0, cap=1024) -> np.ndarray:
        out = np.zeros(cap, RECORD_DTYPE)
        n = ctypes.c_int64()
        _ck(lib().h4d_get_work(self.h, r, out.ctypes.data, cap, ctypes.byref(n)), "h4d_get_work")
        return out[: n.value]

    def h4d_get_state(self, r=0):
        cap = self.cap_atoms[r]
        x = np.zeros((cap, 3))
        v = np.zeros((cap, 3))
        n = ctypes.c_int64()
        _ck(lib().h4d_get_state(self.h, r, _pd(x), _pd(v), cap, ctypes.byref(n)), "h4d_get_state")
        return x[: n.value].copy(), v[: n.value].copy()

    def h4d_set_state(self, r, n_pairs, x, v):
        x = np.ascontiguousarray(x, np.float64)
        v = None if v is None else np.ascontiguousarray(v, np.float64)
        _ck(lib().h4d_set_state(self.h, r, n_pairs, _pd(x), _pd(v)), "h4d_set_state")

    def h4d_set_water_state(self, r, n_water, n_pairs, x, v):
        x = np.ascontiguousarray(x, np.float64)
        v = None if v is None else np.ascontiguousarray(v, np.float64)
        _ck(lib().h4d_set_water_state(self.h, r, n_water, n_pairs, _pd(x), _pd(v)), "h4d_set_water_state")

    def h4d_autotune(self, n_iter=20):
        """Returns {tpa: (mean ns per force pass, mean ns per build)} per candidate."""
        fp = np.zeros(5)
        bp = np.zeros(5)
        _ck(lib().h4d_autotune(self.h, n_iter, _pd(fp), _pd(bp)), "h4d_autotune")
        return {t: (float(fp[k]), float(bp[k])) for k, t in enumerate((1, 2, 4, 8, 16))}

    def h4d_count_pairs(self) -> int:
        n = ctypes.c_int64()
        _ck(lib().h4d_count_pairs(self.h, ctypes.byref(n)), "h4d_count_pairs")
        return n.value

    def h4d_save(self, path):
        _ck(lib().h4d_save(self.h, path.encode()), "h4d_save")

    def h4d_load(self, path):
        _ck(lib().h4d_load(self.h, path.encode()), "h4d_load")

    # ---- learned insertion-site proposal ----
    def h4d_proposal(self, mode, cell_len, eps=0.1, records_per_replica=0):
        _ck(lib().h4d_proposal(self.h, int(mode), cell_len, eps, int(records_per_replica)), "h4d_proposal")

    def h4d_proposal_set_weights(self, w):
        w = np.ascontiguousarray(w, np.float64)
        _ck(lib().h4d_proposal_set_weights(self.h, _pd(w), w.size), "h4d_proposal_set_weights")

    def h4d_proposal_get_weights(self) -> np.ndarray:
        w = np.zeros(H4D_PROP_NW)
        _ck(lib().h4d_proposal_get_weights(self.h, _pd(w), w.size), "h4d_proposal_get_weights")
        return w

    def h4d_proposal_records(self, r=0, cap=1 << 20):
        """(features [n, 2, 96] float32, y [n], move [n], status [n]) of replica r"""
        n = ctypes.c_int64()
        _ck(lib().h4d_proposal_records(self.h, r, None, None, None, None, cap, ctypes.byref(n)), "h4d_proposal_records")
        k = n.value
        f = np.zeros((max(k, 1), 2, 96), np.float32)
        y = np.zeros(max(k, 1))
        mv = np.zeros(max(k, 1), np.int32)
        st = np.zeros(max(k, 1), np.int32)
        pi = ctypes.POINTER(ctypes.c_int32)
        _ck(lib().h4d_proposal_records(self.h, r, f.ctypes.data, _pd(y), mv.ctypes.data_as(pi), st.ctypes.data_as(pi),
                                       k, ctypes.byref(n)), "h4d_proposal_records")
        return f[:k], y[:k], mv[:k], st[:k]

    def h4d_proposal_logits(self, r=0, features=False):
        n = ctypes.c_int64()
        rc = lib().h4d_proposal_logits(self.h, r, None, None, 0, ctypes.byref(n))
        if rc not in (H4D_OK, H4D_ECAPACITY):
            _ck(rc, "h4d_proposal_logits")
        nc = n.value
        lg = np.zeros((nc, 2), np.float32)
        ft = np.zeros((nc, 96), np.float32) if features else None
        _ck(lib().h4d_proposal_logits(self.h, r, lg.ctypes.data, None if ft is None else ft.ctypes.data, nc,
                                      ctypes.byref(n)), "h4d_proposal_logits")
        return (lg, ft) if features else lg

    def h4d_train_proposal(self, steps, batch, lr, y0, seed=0) -> float:
        loss = ctypes.c_double()
        _ck(lib().h4d_train_proposal(self.h, int(steps), int(batch), lr, y0, seed, ctypes.byref(loss)),
            "h4d_train_proposal")
        return loss.value


def h4d_eval_forces(params: h4d_params, L: float, x, w=None, n_water: int = 0):
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    n = x.shape[0]
    wa = None if w is None else np.ascontiguousarray(w, np.float64)
    F = np.zeros((n, 3))
    U = ctypes.c_double()
    _ck(lib().h4d_eval_forces(ctypes.byref(params), L, n_water, n, _pd(x), _pd(wa), _pd(F), ctypes.byref(U)), "h4d_eval_forces")
    return U.value, F


def h4d_eval_forces_static(params: h4d_params, L: float, x, w=None, n_water: int = 0):
    """h4d_eval_forces without any device allocation (static scratch in the library)."""
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    n = x.shape[0]
    wa = None if w is None else np.ascontiguousarray(w, np.float64)
    F = np.zeros((n, 3))
    U = ctypes.c_double()
    _ck(lib().h4d_eval_forces_static(ctypes.byref(params), L, n_water, n, _pd(x), _pd(wa), _pd(F), ctypes.byref(U)),
        "h4d_eval_forces_static")
    return U.value, F


def h4d_neighbor_pairs(L: float, x, r_list: float):
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    n = x.shape[0]
    m = ctypes.c_int64()
    _ck(lib().h4d_neighbor_pairs(L, n, _pd(x), r_list, None, None, 0, ctypes.byref(m)), "h4d_neighbor_pairs")
    oi = np.zeros(max(m.value, 1), np.int32)
    oj = np.zeros(max(m.value, 1), np.int32)
    _ck(
        lib().h4d_neighbor_pairs(L, n, _pd(x), r_list, oi.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 oj.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), m.value, ctypes.byref(m)),
        "h4d_neighbor_pairs",
    )
    return oi[: m.value], oj[: m.value]


def h4d_proposal_grad(w, feat, tgt):
    """loss and gradient of the proposal network on records feat [n, 2, 96] with targets
    tgt [n, 2], through the library's BF16 forward/backward kernels"""
    w = np.ascontiguousarray(w, np.float64)
    f = np.ascontiguousarray(feat, np.float32).reshape(-1, 2, 96)
    t = np.ascontiguousarray(tgt, np.float32).reshape(-1, 2)
    g = np.zeros(H4D_PROP_NW)
    loss = ctypes.c_double()
    _ck(lib().h4d_proposal_grad(_pd(w), f.shape[0], f.ctypes.data, t.ctypes.data, ctypes.byref(loss), _pd(g)),
        "h4d_proposal_grad")
    return loss.value, g


def h4d_coulomb_poly(alpha, rc_coul):
    """(coefficients of C(r^2), lowest first, float32; True when the engine uses the form)"""
    c = np.zeros(8, np.float32)
    used = ctypes.c_int32()
    _ck(lib().h4d_coulomb_poly(ctypes.c_double(alpha), ctypes.c_double(rc_coul), c.ctypes.data,
                               ctypes.byref(used)), "h4d_coulomb_poly")
    return c, bool(used.value)


def h4d_device_info():
    """(SM count, engine kernel binary version, PTX version) of the current device"""
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _ck(lib().h4d_device_info(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "h4d_device_info")
    return a.value, b.value, c.value


def h4d_measure_fp32_peak():
    """(TFLOP/s, seconds) of the FMA-chain probe"""
    t, s = ctypes.c_double(), ctypes.c_double()
    _ck(lib().h4d_measure_fp32_peak(ctypes.byref(t), ctypes.byref(s)), "h4d_measure_fp32_peak")
    return t.value, s.value


def h4d_ewald_lr(params: h4d_params, L: float, x, alpha: float, kmax: int, wbar: float = 0.0,
                 kappa_lr: float = 0.0, n_water: int = 0, forces: bool = True, kernel_ms: bool = False):
    """(U_recip, U_self, F_recip or None) of the long-range Coulomb term (Eqs. 9-10), plus
    the kernels' device time in ms when kernel_ms"""
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    n = x.shape[0]
    ur, us, tk = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    F = np.zeros((n, 3)) if forces else None
    _ck(lib().h4d_ewald_lr(ctypes.byref(params), L, n_water, n, _pd(x), alpha, int(kmax), wbar, kappa_lr,
                           ctypes.byref(ur), ctypes.byref(us), _pd(F), ctypes.byref(tk)), "h4d_ewald_lr")
    return (ur.value, us.value, F, tk.value) if kernel_ms else (ur.value, us.value, F)
