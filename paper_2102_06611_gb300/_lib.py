"""ctypes declarations of the C ABI in ``include/pa.h`` (argument marshalling only).

Loading fails loudly if the CUDA library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

(PA_OK, PA_ERR_INVALID_ARG, PA_ERR_STATE, PA_ERR_CAPACITY, PA_ERR_CUDA, PA_ERR_TIMEOUT, PA_ERR_NUMERIC,
 PA_ERR_TOO_LARGE) = range(8)
STATUS_NAMES = {0: "PA_OK", 1: "PA_ERR_INVALID_ARG", 2: "PA_ERR_STATE", 3: "PA_ERR_CAPACITY",
                4: "PA_ERR_CUDA", 5: "PA_ERR_TIMEOUT", 6: "PA_ERR_NUMERIC", 7: "PA_ERR_TOO_LARGE"}
PA_RESAMPLE_NEAREST, PA_RESAMPLE_POISSON, PA_RESAMPLE_MULTINOMIAL = 0, 1, 2
PA_UPDATE_METROPOLIS, PA_UPDATE_HEATBATH = 0, 1


class PAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class pa_config(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("resample", ctypes.c_int), ("R", ctypes.c_longlong),
                ("capacity", ctypes.c_longlong), ("seed", ctypes.c_ulonglong), ("update", ctypes.c_int),
                ("pad", ctypes.c_int)]


class pa_sizes(ctypes.Structure):
    _fields_ = [("spin_bytes", ctypes.c_size_t), ("int_bytes", ctypes.c_size_t),
                ("work_bytes", ctypes.c_size_t), ("bytes_per_replica", ctypes.c_size_t)]


class pa_buffers(ctypes.Structure):
    _fields_ = [("spins", ctypes.c_void_p * 2), ("level", ctypes.c_void_p * 2),
                ("mag", ctypes.c_void_p * 2), ("fam", ctypes.c_void_p * 2), ("work", ctypes.c_void_p)]


class pa_obs(ctypes.Structure):
    _fields_ = [("step", ctypes.c_longlong), ("R", ctypes.c_longlong), ("beta", ctypes.c_double),
                ("dbeta", ctypes.c_double), ("e", ctypes.c_double), ("C", ctypes.c_double),
                ("m", ctypes.c_double), ("m2", ctypes.c_double), ("chi", ctypes.c_double),
                ("lnQ", ctypes.c_double), ("minus_betaF", ctypes.c_double), ("rho_t", ctypes.c_double),
                ("families", ctypes.c_longlong), ("sum_E", ctypes.c_longlong), ("sum_E2", ctypes.c_longlong),
                ("sum_absM", ctypes.c_longlong), ("sum_M2", ctypes.c_longlong),
                ("sum_size2", ctypes.c_longlong), ("theta", ctypes.c_int), ("status", ctypes.c_int),
                ("sum_lnRratio", ctypes.c_double), ("R_target", ctypes.c_longlong)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class pa_analysis(ctypes.Structure):
    _fields_ = [("R", ctypes.c_longlong), ("families", ctypes.c_longlong), ("n_blocks", ctypes.c_int),
                ("pad", ctypes.c_int), ("beta", ctypes.c_double),
                ("mean_E", ctypes.c_double), ("var_E", ctypes.c_double), ("var_mean_E_jack", ctypes.c_double),
                ("var_mean_E_blocked", ctypes.c_double), ("R_eff_E", ctypes.c_double),
                ("mean_absM", ctypes.c_double), ("var_absM", ctypes.c_double),
                ("var_mean_absM_jack", ctypes.c_double), ("var_mean_absM_blocked", ctypes.c_double),
                ("R_eff_M", ctypes.c_double), ("C", ctypes.c_double), ("var_C_jack", ctypes.c_double),
                ("S_f", ctypes.c_double), ("rho_s", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "pad"}


class pa_weighted(ctypes.Structure):
    _fields_ = [("step", ctypes.c_longlong), ("M", ctypes.c_int), ("mode", ctypes.c_int), ("beta", ctypes.c_double),
                ("M_eff", ctypes.c_double), ("max_weight", ctypes.c_double), ("var_minus_betaF", ctypes.c_double),
                ("minus_betaF_combined", ctypes.c_double), ("e", ctypes.c_double), ("C", ctypes.c_double),
                ("m", ctypes.c_double), ("m2", ctypes.c_double), ("chi", ctypes.c_double),
                ("e_plain", ctypes.c_double), ("C_plain", ctypes.c_double), ("m_plain", ctypes.c_double),
                ("m2_plain", ctypes.c_double), ("chi_plain", ctypes.c_double), ("status", ctypes.c_int),
                ("pad", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "pad"}


class pa_sched_entry(ctypes.Structure):
    _fields_ = [("step", ctypes.c_longlong), ("beta", ctypes.c_double), ("dbeta", ctypes.c_double),
                ("alpha", ctypes.c_double), ("theta", ctypes.c_int), ("source", ctypes.c_int)]


PA_SCHED_CALLER, PA_SCHED_BISECT, PA_SCHED_LEARNED, PA_SCHED_FALLBACK = 0, 1, 2, 3


class pa_learned_model(ctypes.Structure):
    _fields_ = [("params_bf16", ctypes.c_void_p), ("norm", ctypes.c_void_p)]


class pa_proposal(ctypes.Structure):
    _fields_ = [("beta_next", ctypes.c_double), ("alpha", ctypes.c_double), ("dbeta_prop", ctypes.c_double),
                ("theta_next", ctypes.c_int), ("theta_prop", ctypes.c_int), ("source", ctypes.c_int),
                ("pad", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "pad"}

# name -> (restype, argtypes): every entry point declared in include/pa.h
_P = ctypes.POINTER
_vp = ctypes.c_void_p
SIGNATURES = {
    "pa_query_sizes": (ctypes.c_int, [_P(pa_config), _P(pa_sizes)]),
    "pa_init": (ctypes.c_int, [_P(pa_config), _P(pa_buffers), _vp, _P(_vp)]),
    "pa_resample": (ctypes.c_int, [_vp, ctypes.c_double]),
    "pa_anneal_step": (ctypes.c_int, [_vp, ctypes.c_int]),
    "pa_record": (ctypes.c_int, [_vp, _vp]),
    "pa_observables": (ctypes.c_int, [_vp, _P(pa_obs)]),
    "pa_analyze": (ctypes.c_int, [_vp, ctypes.c_int, _P(pa_analysis)]),
    "pa_weighted_average": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "pa_propose_schedule": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           _P(ctypes.c_double), _P(ctypes.c_double)]),
    "pa_schedule_log": (ctypes.c_int, [_vp, _vp, ctypes.c_longlong, _P(ctypes.c_longlong)]),
    "pa_mlp_param_count": (ctypes.c_size_t, []),
    "pa_mlp_forward": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _vp, _vp]),
    "pa_mlp_backward": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp]),
    "pa_mlp_adam": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_float, ctypes.c_float, _vp, _vp]),
    "pa_mlp_round": (ctypes.c_int, [_vp, _vp, _vp]),
    "pa_features": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "pa_decorrelation": (ctypes.c_int, [_vp, _P(ctypes.c_double), _vp]),
    "pa_propose_learned": (ctypes.c_int, [_vp, _P(pa_learned_model), ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                          _P(pa_proposal)]),
    "pa_sync": (ctypes.c_int, [_vp]),
    "pa_population": (ctypes.c_int, [_vp, _P(ctypes.c_longlong)]),
    "pa_histogram": (ctypes.c_int, [_vp, _vp]),
    "pa_replicas": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "pa_copy_counts": (ctypes.c_int, [_vp, _vp, _P(ctypes.c_longlong)]),
    "pa_hashes": (ctypes.c_int, [_vp, _vp]),
    "pa_export_spins": (ctypes.c_int, [_vp, ctypes.c_longlong, ctypes.c_longlong, _vp]),
    "pa_philox_xor": (ctypes.c_int, [ctypes.c_ulonglong, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "pa_copy_numbers_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong, _vp,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_uint,
                                              ctypes.c_ulonglong, ctypes.c_int, _vp, _P(ctypes.c_double),
                                              _P(ctypes.c_longlong), _vp]),
    "pa_shard_init": (ctypes.c_int, [_P(pa_config), ctypes.c_longlong, ctypes.c_longlong, _P(pa_buffers), _vp,
                                     _P(_vp)]),
    "pa_shard_summary_len": (ctypes.c_longlong, [ctypes.c_int]),
    "pa_shard_summary": (ctypes.c_int, [_vp, _vp]),
    "pa_shard_combine": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "pa_shard_copy": (ctypes.c_int, [_vp, ctypes.c_longlong, ctypes.c_longlong, _vp, _vp, _vp, _vp]),
    "pa_shard_adopt": (ctypes.c_int, [_vp, ctypes.c_longlong, ctypes.c_longlong]),
    "pa_shard_layout": (ctypes.c_int, [_vp, _P(ctypes.c_int), _P(ctypes.c_longlong), _P(ctypes.c_longlong)]),
    "pa_last_error": (ctypes.c_char_p, [_vp]),
    "pa_destroy": (None, [_vp]),
}


def lib_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load the library (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise ImportError(f"CUDA library {path} missing; build it with paper_2102_06611_gb300.build")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def load_without_build() -> ctypes.CDLL:
    """Load an already built library (used by the symbol-export test)."""
    L = ctypes.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


class pa_run_desc(ctypes.Structure):
    _fields_ = [("cfg", pa_config), ("n_temps", ctypes.c_int), ("theta", ctypes.c_int)]


class pa_batch_shape(ctypes.Structure):
    _fields_ = [("unified", ctypes.c_int), ("blocks_per_sm", ctypes.c_int), ("ipw_scale", ctypes.c_int),
                ("ms", ctypes.c_float)]


class pa_batch_tuning(ctypes.Structure):
    _fields_ = [("n_candidates", ctypes.c_int), ("chosen", ctypes.c_int), ("chosen_grid", ctypes.c_int),
                ("pad", ctypes.c_int), ("cand", pa_batch_shape * 16)]


SIGNATURES.update({
    "pa_batch_query_sizes": (ctypes.c_int, [ctypes.c_int, _P(pa_run_desc), _P(ctypes.c_size_t)]),
    "pa_batch_init": (ctypes.c_int, [ctypes.c_int, _P(pa_run_desc), _vp, ctypes.c_size_t, _vp, _P(_vp)]),
    "pa_batch_step": (ctypes.c_int, [_vp]),
    "pa_batch_status": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "pa_batch_record": (ctypes.c_int, [_vp, _vp]),
    "pa_batch_observables": (ctypes.c_int, [_vp, _vp]),
    "pa_batch_hashes": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _P(ctypes.c_longlong)]),
    "pa_batch_get_tuning": (ctypes.c_int, [_vp, _P(pa_batch_tuning)]),
    "pa_batch_set_shape": (ctypes.c_int, [_vp, _P(pa_batch_shape)]),
    "pa_batch_destroy": (None, [_vp]),
})

SIGNATURES.update({
    "pa_checkpoint_size": (ctypes.c_int, [_vp, _P(ctypes.c_size_t)]),
    "pa_save": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "pa_load": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
})
