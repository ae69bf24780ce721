"""CPU oracle for population annealing of the 2D Ising ferromagnet (arXiv:2102.06611).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` leg may import this package.  The product path
(``paper_2102_06611_gb300``) never imports it and shares no code with it.

The arithmetic lives in plain C (``pa_oracle.c``, ``exact_ising.c``, ``pa_analysis.c``), built with gcc
and ``-ffp-contract=off`` so that every binary64 multiply and add is rounded on its own.
This module only marshals arguments through ctypes and adds nothing to the method.

Parity pins (``tests/test_oracle_*.py``):
  * Philox4x32-10: the published known-answer vectors of Salmon et al. (SC'11).
  * ``exp``: <= 1 ulp against libm and against a 60-digit decimal reference.
  * energies: ground state, antiferromagnetic state, stripes, single flips.
  * Metropolis sweep: level distribution at L=4 against brute-force Boltzmann weights.
  * Q_i / free energy: ln Z from enumeration, transfer matrix and Kaufman's closed form.
  * copy numbers: mean equals tau_hat (Sec. II), Poisson pmf chi-square.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborapa.so")
_SOURCES = ["pa_oracle.c", "exact_ising.c", "pa_analysis.c"]
_lock = threading.Lock()
_lib = None

STREAM_INIT, STREAM_SWEEP, STREAM_RESAMPLE, STREAM_POISSON, STREAM_REFINE = 0, 1, 2, 3, 4
NEAREST, POISSON, MULTINOMIAL = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (no FMA contraction, -O2)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Info(ctypes.Structure):
    _fields_ = [("lnQ", ctypes.c_double), ("S", ctypes.c_double),
                ("kmin", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("R_new", ctypes.c_int64)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.POINTER
            u32p, i32p, i64p, u64p, i8p, dp = (P(ctypes.c_uint32), P(ctypes.c_int32),
                                                P(ctypes.c_int64), P(ctypes.c_uint64),
                                                P(ctypes.c_int8), P(ctypes.c_double))
            vp = ctypes.c_void_p
            sig = {
                "orc_philox4x32_10": (None, [u32p, u32p, u32p]),
                "orc_exp": (ctypes.c_double, [ctypes.c_double]),
                "orc_metropolis_threshold": (ctypes.c_uint64, [ctypes.c_double]),
                "orc_energy_mag": (None, [ctypes.c_int, i8p, i32p, i32p]),
                "orc_hash": (ctypes.c_uint64, [ctypes.c_int, i8p]),
                "orc_pack": (None, [ctypes.c_int, i8p, u32p]),
                "orc_unpack": (None, [ctypes.c_int, u32p, i8p]),
                "orc_init_replica": (None, [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, i8p]),
                "orc_sweep_replica": (None, [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                             ctypes.c_uint32, ctypes.c_double, ctypes.c_int, i8p]),
                "orc_sweep_replica_t0": (None, [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                                ctypes.c_uint32, ctypes.c_double, ctypes.c_int,
                                                ctypes.c_int, i8p]),
                "orc_heatbath_threshold": (ctypes.c_uint64, [ctypes.c_double]),
                "orc_sweep_replica_u": (None, [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                               ctypes.c_uint32, ctypes.c_double, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_int, i8p]),
                "orc_pa_set_update": (None, [vp, ctypes.c_int]),
                "orc_sweep_uniform": (ctypes.c_uint32, [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                                        ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
                                                        ctypes.c_int]),
                "orc_poisson": (ctypes.c_int64, [ctypes.c_double, ctypes.c_uint64,
                                                 ctypes.c_uint32, ctypes.c_uint32]),
                "orc_resample_levels": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                                       i32p, ctypes.c_double, ctypes.c_double,
                                                       ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                                                       ctypes.c_int64, i32p, P(_Info)]),
                "orc_resample_shard": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, i64p, ctypes.c_int64,
                                                      ctypes.c_int64, i32p, ctypes.c_int64, ctypes.c_double,
                                                      ctypes.c_double, ctypes.c_uint32, ctypes.c_uint64,
                                                      ctypes.c_int, i64p, i32p, P(_Info)]),
                "orc_observables_from_sums": (None, [ctypes.c_int, ctypes.c_int64, i64p, ctypes.c_double,
                                                     ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                     ctypes.c_double, ctypes.c_uint32, ctypes.c_int, dp]),
                "orc_population_sums": (None, [ctypes.c_int64, i32p, i32p, i32p, i64p]),
                "orc_pa_create": (vp, [ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_uint64, ctypes.c_int]),
                "orc_pa_destroy": (None, [vp]),
                "orc_pa_init": (None, [vp]),
                "orc_pa_resample": (ctypes.c_int, [vp, ctypes.c_double]),
                "orc_pa_sweep": (None, [vp, ctypes.c_int]),
                "orc_pa_observables": (None, [vp, dp, i64p]),
                "orc_pa_R": (ctypes.c_int64, [vp]),
                "orc_pa_R_prev": (ctypes.c_int64, [vp]),
                "orc_pa_status": (ctypes.c_int, [vp]),
                "orc_pa_sum_lnQ": (ctypes.c_double, [vp]),
                "orc_pa_histogram": (None, [vp, i32p]),
                "orc_pa_hashes": (None, [vp, u64p]),
                "orc_pa_get": (None, [vp, i32p, i32p, i32p]),
                "orc_pa_counts": (None, [vp, i32p]),
                "orc_pa_spins": (None, [vp, ctypes.c_int64, ctypes.c_int64, i8p]),
                "orc_pa_set": (ctypes.c_int, [vp, ctypes.c_int64, i8p, i32p, ctypes.c_uint32,
                                              ctypes.c_double, ctypes.c_double]),
                "orc_overlap": (ctypes.c_double, [ctypes.c_int, i64p, ctypes.c_double]),
                "orc_bisect_next_beta": (ctypes.c_double, [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_double,
                                                           ctypes.c_double, ctypes.c_double, ctypes.c_int, dp]),
                "orc_pa_propose_bisect": (ctypes.c_double, [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                            ctypes.c_int, dp]),
                "orc_accept_or_bisect": (ctypes.c_double, [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_double,
                                                           ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                           ctypes.c_double, ctypes.c_int, dp,
                                                           ctypes.POINTER(ctypes.c_int)]),
                "orc_analysis": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int64, i32p, i32p,
                                                i32p, ctypes.c_int, dp]),
                "orc_pa_analysis": (ctypes.c_int, [vp, ctypes.c_int, dp]),
                "orc_weighted_average": (None, [ctypes.c_int, dp, dp, dp, dp, dp, ctypes.c_int, dp]),
                "orc_bruteforce": (ctypes.c_int, [ctypes.c_int, i64p, i64p, i64p]),
                "orc_transfer_lnZ": (ctypes.c_double, [ctypes.c_int, ctypes.c_double]),
                "orc_kaufman_lnZ": (ctypes.c_double, [ctypes.c_int, ctypes.c_double]),
                "orc_kaufman_thermo": (None, [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


# ----------------------------------------------------------------------------- primitives
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                            _ptr(out, ctypes.c_uint32))
    return out


def exp(x: float) -> float:
    return lib().orc_exp(float(x))


def metropolis_threshold(y: float) -> int:
    return int(lib().orc_metropolis_threshold(float(y)))


def energy_mag(L: int, s: np.ndarray):
    s = np.ascontiguousarray(s, dtype=np.int8).reshape(L * L)
    E, M = ctypes.c_int32(), ctypes.c_int32()
    lib().orc_energy_mag(L, _ptr(s, ctypes.c_int8), ctypes.byref(E), ctypes.byref(M))
    return E.value, M.value


def replica_hash(L: int, s: np.ndarray) -> int:
    s = np.ascontiguousarray(s, dtype=np.int8).reshape(L * L)
    return int(lib().orc_hash(L, _ptr(s, ctypes.c_int8)))


def pack(L: int, s: np.ndarray) -> np.ndarray:
    s = np.ascontiguousarray(s, dtype=np.int8).reshape(L * L)
    out = np.zeros(L * ((L + 31) // 32), dtype=np.uint32)
    lib().orc_pack(L, _ptr(s, ctypes.c_int8), _ptr(out, ctypes.c_uint32))
    return out


def unpack(L: int, words: np.ndarray) -> np.ndarray:
    w = np.ascontiguousarray(words, dtype=np.uint32)
    s = np.zeros(L * L, dtype=np.int8)
    lib().orc_unpack(L, _ptr(w, ctypes.c_uint32), _ptr(s, ctypes.c_int8))
    return s


def init_replica(L: int, seed: int, j: int) -> np.ndarray:
    s = np.zeros(L * L, dtype=np.int8)
    lib().orc_init_replica(L, seed, j, _ptr(s, ctypes.c_int8))
    return s


METROPOLIS, HEATBATH = 0, 1


def sweep_replica(L: int, seed: int, step: int, slot: int, beta: float, theta: int,
                  s: np.ndarray, t0: int = 0, update: int = METROPOLIS) -> np.ndarray:
    """theta sweeps numbered t0 .. t0 + theta - 1 within temperature step `step`."""
    out = np.array(s, dtype=np.int8, copy=True).reshape(L * L)
    if update == METROPOLIS:
        lib().orc_sweep_replica_t0(L, seed, step, slot, float(beta), int(t0), int(theta),
                                   _ptr(out, ctypes.c_int8))
    else:
        lib().orc_sweep_replica_u(L, seed, step, slot, float(beta), int(t0), int(theta), int(update),
                                  _ptr(out, ctypes.c_int8))
    return out


def heatbath_threshold(y: float) -> int:
    return int(lib().orc_heatbath_threshold(float(y)))


def sweep_uniform(L: int, seed: int, step: int, slot: int, tag: int, r: int, p: int) -> int:
    """The 32-bit uniform of colour-site p of row r in sweep-colour `tag` = 2t + q."""
    return int(lib().orc_sweep_uniform(L, seed, step, slot, tag, r, p))


def poisson(lam: float, seed: int, j: int, step: int) -> int:
    return int(lib().orc_poisson(float(lam), seed, j, step))


def resample_levels(L, R_target, levels, beta_prev, beta_new, step, seed, kind, capacity):
    """Step 2 of the method from given levels: returns (status, counts, lnQ, S, kmin, R_new)."""
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    counts = np.zeros(len(lv), dtype=np.int32)
    info = _Info()
    st = lib().orc_resample_levels(L, R_target, len(lv), _ptr(lv, ctypes.c_int32),
                                   float(beta_prev), float(beta_new), step, seed, kind,
                                   capacity, _ptr(counts, ctypes.c_int32), ctypes.byref(info))
    return st, counts, info.lnQ, info.S, info.kmin, info.R_new


def resample_shard(L, R_target, hist, R_prev, levels, parent_base, beta_prev, beta_new, step, seed, kind,
                   hist_before=None):
    """Step 2 for the parents of one shard of a population split by slot ranges: tables from
    the whole population's histogram `hist` (R_prev parents), copy numbers of the local parents
    keyed by their global index parent_base + j.  Multinomial resampling also needs
    `hist_before`, the level histogram of the parents below parent_base.  Returns (status,
    counts, lnQ, R_new_local)."""
    h = np.ascontiguousarray(hist, dtype=np.int64)
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    hb = None if hist_before is None else np.ascontiguousarray(hist_before, dtype=np.int64)
    counts = np.zeros(len(lv), dtype=np.int32)
    info = _Info()
    st = lib().orc_resample_shard(L, R_target, _ptr(h, ctypes.c_int64), R_prev, len(lv), _ptr(lv, ctypes.c_int32),
                                  parent_base, float(beta_prev), float(beta_new), step, seed, kind,
                                  None if hb is None else _ptr(hb, ctypes.c_int64),
                                  _ptr(counts, ctypes.c_int32), ctypes.byref(info))
    return st, counts, info.lnQ, info.R_new


def population_sums(E, M, fam) -> np.ndarray:
    """Exact integer sums of a population in slot order: sum E, E^2, |M|, M^2, families f,
    sum of family size^2."""
    E, M, F = (np.ascontiguousarray(a, np.int32) for a in (E, M, fam))
    out = np.zeros(6, np.int64)
    lib().orc_population_sums(len(E), _ptr(E, ctypes.c_int32), _ptr(M, ctypes.c_int32), _ptr(F, ctypes.c_int32),
                              _ptr(out, ctypes.c_int64))
    return out


def observables_from_sums(N, R, isums, beta, dbeta, lnQ, sum_lnQ, sum_lnR, step, theta) -> dict:
    """Step 4 (Sec. III, Sec. VII) of a population of R replicas from its exact integer sums
    (population_sums order)."""
    s = np.ascontiguousarray(isums, np.int64)
    out = np.zeros(15)
    lib().orc_observables_from_sums(int(N), int(R), _ptr(s, ctypes.c_int64), float(beta), float(dbeta), float(lnQ),
                                    float(sum_lnQ), float(sum_lnR), int(step), int(theta), _ptr(out, ctypes.c_double))
    return dict(zip(OBS_FIELDS, out.tolist()))


# ----------------------------------------------------------------------------- schedule
BISECT_ITERS = 48


def overlap(N: int, hist, dbeta: float) -> float:
    """Energy-histogram overlap alpha(dbeta) of a level histogram with its reweighting."""
    h = np.ascontiguousarray(hist, dtype=np.int64)
    return float(lib().orc_overlap(N, _ptr(h, ctypes.c_int64), float(dbeta)))


def bisect_next_beta(N, hist, beta, beta_final, dbeta_max, alpha_target, iters=BISECT_ITERS):
    h = np.ascontiguousarray(hist, dtype=np.int64)
    a = ctypes.c_double()
    b = lib().orc_bisect_next_beta(N, _ptr(h, ctypes.c_int64), float(beta), float(beta_final),
                                   float(dbeta_max), float(alpha_target), int(iters), ctypes.byref(a))
    return float(b), float(a.value)


def accept_or_bisect(N, hist, beta, beta_final, dbeta_max, dbeta_prop, alpha_floor, alpha_target,
                     iters=BISECT_ITERS):
    """Learned-schedule check: keep dbeta_prop if its overlap reaches alpha_floor, else bisect.
    Returns (beta_next, alpha, source) with source 2 = kept, 3 = fallback."""
    h = np.ascontiguousarray(hist, dtype=np.int64)
    a = ctypes.c_double()
    src = ctypes.c_int()
    b = lib().orc_accept_or_bisect(N, _ptr(h, ctypes.c_int64), float(beta), float(beta_final), float(dbeta_max),
                                   float(dbeta_prop), float(alpha_floor), float(alpha_target), int(iters),
                                   ctypes.byref(a), ctypes.byref(src))
    return float(b), float(a.value), int(src.value)


# ----------------------------------------------------------------------------- exact
def bruteforce(L: int):
    N = L * L
    g = np.zeros(N + 1, np.int64)
    sa = np.zeros(N + 1, np.int64)
    s2 = np.zeros(N + 1, np.int64)
    if lib().orc_bruteforce(L, _ptr(g, ctypes.c_int64), _ptr(sa, ctypes.c_int64),
                            _ptr(s2, ctypes.c_int64)):
        raise ValueError("lattice too large to enumerate")
    return g, sa, s2


def transfer_lnZ(L: int, beta: float) -> float:
    return lib().orc_transfer_lnZ(L, float(beta))


def kaufman_lnZ(L: int, beta: float) -> float:
    return lib().orc_kaufman_lnZ(L, float(beta))


def kaufman_thermo(L: int, beta: float, h: float = 2e-4):
    """(<E>, C per spin, ln Z) of the periodic L x L lattice from Kaufman's closed form."""
    out = np.zeros(3)
    lib().orc_kaufman_thermo(L, float(beta), float(h), _ptr(out, ctypes.c_double))
    return float(out[0]), float(out[1]), float(out[2])


# ----------------------------------------------------------------------------- full PA
OBS_FIELDS = ["beta", "dbeta", "R", "e", "C", "m", "m2", "chi", "lnQ", "minus_betaF",
              "families", "rho_t", "step", "theta", "sum_lnRratio"]


ANALYSIS_FIELDS = ["n_blocks", "mean_E", "var_E", "var_mean_E_jack", "var_mean_E_blocked", "R_eff_E",
                   "mean_absM", "var_absM", "var_mean_absM_jack", "var_mean_absM_blocked", "R_eff_M",
                   "C", "var_C_jack", "S_f", "rho_s", "families"]


def analysis(N: int, beta: float, E, M, fam, n_blocks: int = 100) -> dict:
    """Blocked / jackknife errors, R_eff(E), R_eff(|M|), family entropy of a population given
    as arrays in slot (tree) order (Sec. IV Eqs. neff, blocks, blocked_variance,
    jackknife-blocks, jackknife-variance; Sec. V Eq. rhos)."""
    E = np.ascontiguousarray(E, np.int32)
    M = np.ascontiguousarray(M, np.int32)
    fam = np.ascontiguousarray(fam, np.int32)
    out = np.zeros(16)
    st = lib().orc_analysis(int(N), float(beta), len(E), _ptr(E, ctypes.c_int32), _ptr(M, ctypes.c_int32),
                            _ptr(fam, ctypes.c_int32), int(n_blocks), _ptr(out, ctypes.c_double))
    if st != 0:
        raise ValueError("need 2 <= n_blocks <= R")
    return dict(zip(ANALYSIS_FIELDS, out.tolist()))


WEIGHTED_FIELDS = ["M_eff", "max_weight", "var_minus_betaF", "minus_betaF_combined", "e", "C", "m", "m2", "chi",
                   "e_plain", "C_plain", "m_plain", "m2_plain", "chi_plain"]


def weighted_average(R_i, R_target, minus_betaF, sum_lnRratio, obs, mode: int = 1) -> dict:
    """Weighted average over independent runs at one temperature (Sec. VIII, Eq.
    weighted-averages for mode 0, Eq. modified-weights2 for mode 1); obs is M x 5
    (e, C, m, m2, chi)."""
    arrs = [np.ascontiguousarray(a, np.float64) for a in (R_i, R_target, minus_betaF, sum_lnRratio)]
    o = np.ascontiguousarray(obs, np.float64).reshape(-1, 5)
    out = np.zeros(14)
    lib().orc_weighted_average(len(arrs[0]), *[_ptr(a, ctypes.c_double) for a in arrs], _ptr(o, ctypes.c_double),
                               int(mode), _ptr(out, ctypes.c_double))
    return dict(zip(WEIGHTED_FIELDS, out.tolist()))


class PA:
    """Plain single-threaded population annealing run (Sec. II steps 1-5)."""

    def __init__(self, L: int, R: int, seed: int, kind: int = NEAREST, capacity: int | None = None,
                 update: int = METROPOLIS):
        if capacity is None:
            capacity = default_capacity(R)
        self.L, self.N, self.R_target, self.capacity = L, L * L, R, capacity
        self._h = lib().orc_pa_create(L, R, capacity, seed, kind)
        if not self._h:
            raise ValueError("invalid oracle configuration")
        lib().orc_pa_set_update(self._h, int(update))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_pa_destroy(h)
            self._h = None

    def init(self):
        lib().orc_pa_init(self._h)

    def resample(self, beta_new: float) -> int:
        return lib().orc_pa_resample(self._h, float(beta_new))

    def sweep(self, theta: int):
        lib().orc_pa_sweep(self._h, int(theta))

    @property
    def R(self) -> int:
        return int(lib().orc_pa_R(self._h))

    @property
    def R_prev(self) -> int:
        return int(lib().orc_pa_R_prev(self._h))

    def observables(self) -> dict:
        out = np.zeros(15)
        isums = np.zeros(6, np.int64)
        lib().orc_pa_observables(self._h, _ptr(out, ctypes.c_double), _ptr(isums, ctypes.c_int64))
        d = dict(zip(OBS_FIELDS, out.tolist()))
        d["sums"] = isums
        return d

    def analysis(self, n_blocks: int = 100) -> dict:
        out = np.zeros(16)
        st = lib().orc_pa_analysis(self._h, int(n_blocks), _ptr(out, ctypes.c_double))
        if st != 0:
            raise ValueError("need 2 <= n_blocks <= R")
        return dict(zip(ANALYSIS_FIELDS, out.tolist()))

    def histogram(self) -> np.ndarray:
        h = np.zeros(self.N + 1, np.int32)
        lib().orc_pa_histogram(self._h, _ptr(h, ctypes.c_int32))
        return h

    def hashes(self) -> np.ndarray:
        out = np.zeros(self.R, np.uint64)
        lib().orc_pa_hashes(self._h, _ptr(out, ctypes.c_uint64))
        return out

    def state(self):
        R = self.R
        E, M, F = (np.zeros(R, np.int32) for _ in range(3))
        lib().orc_pa_get(self._h, _ptr(E, ctypes.c_int32), _ptr(M, ctypes.c_int32),
                         _ptr(F, ctypes.c_int32))
        return E, M, F

    def counts(self) -> np.ndarray:
        out = np.zeros(self.R_prev, np.int32)
        lib().orc_pa_counts(self._h, _ptr(out, ctypes.c_int32))
        return out

    def spins(self, first: int = 0, count: int | None = None) -> np.ndarray:
        if count is None:
            count = self.R - first
        out = np.zeros(count * self.N, np.int8)
        lib().orc_pa_spins(self._h, first, count, _ptr(out, ctypes.c_int8))
        return out.reshape(count, self.L, self.L)

    def propose_bisect(self, beta_final: float, dbeta_max: float, alpha_target: float,
                       iters: int = BISECT_ITERS):
        """Next beta of the adaptive schedule from the current population's histogram."""
        a = ctypes.c_double()
        b = lib().orc_pa_propose_bisect(self._h, float(beta_final), float(dbeta_max), float(alpha_target),
                                        int(iters), ctypes.byref(a))
        return float(b), float(a.value)

    def set_population(self, spins: np.ndarray, fam: np.ndarray, step: int, beta: float,
                       sum_lnQ: float = 0.0):
        s = np.ascontiguousarray(spins, dtype=np.int8)
        f = np.ascontiguousarray(fam, dtype=np.int32)
        R = len(f)
        if lib().orc_pa_set(self._h, R, _ptr(s, ctypes.c_int8), _ptr(f, ctypes.c_int32),
                            step, float(beta), float(sum_lnQ)):
            raise ValueError("population does not fit")


def default_capacity(R: int) -> int:
    """Buffer capacity for a fluctuating population: R + ceil(10 sqrt R) + 64."""
    import math
    return R + int(math.ceil(10.0 * math.sqrt(R))) + 64
