"""GB300 (sm_103a) population annealing for the 2D Ising ferromagnet (arXiv:2102.06611).

The compute path is the CUDA library behind the C ABI in ``include/pa.h``; this package
only allocates device buffers with PyTorch, passes their pointers and the current CUDA
stream, and turns status codes into exceptions.  Method steps (Sec. II of the paper):

    pa = PopulationAnnealing(L=64, R=1_000_000, seed=7)   # step 1 at beta_0 = 0
    for i in range(1, 301):
        pa.resample(i / 300)                              # step 2
        pa.anneal_step(10)                                # step 3
        obs = pa.observables()                            # step 4
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import PAError, pa_obs

__all__ = ["PopulationAnnealing", "PAError", "pa_obs", "default_capacity", "SUPPORTED_L", "REGISTER_L", "OBS_BYTES",
           "weighted_average"]

SUPPORTED_L = tuple(range(4, 129, 2))              # even 4 <= L <= 128
REGISTER_L = (4, 8, 12, 16, 20, 24, 32, 40, 48, 64, 80, 96, 128)   # sizes with register-resident sweep kernels
OBS_BYTES = ctypes.sizeof(pa_obs)


def default_capacity(R: int) -> int:
    """Room for a fluctuating population: R + ceil(10 sqrt R) + 64."""
    import math
    return R + int(math.ceil(10.0 * math.sqrt(R))) + 64


def _check(lib, ctx, status: int):
    if status != _lib.PA_OK:
        msg = lib.pa_last_error(ctx) if ctx else b""
        raise PAError(status, (msg or b"").decode(errors="replace"))


def weighted_average(records: torch.Tensor, mode: str = "modified", stream: torch.cuda.Stream | None = None) -> dict:
    """Weighted average over independent runs at one temperature step (Sec. VIII):
    `records` is a device tensor holding M pa_obs records back to back (pa_record /
    Batch.record output for one step); mode "standard" is Eq. weighted-averages, "modified"
    Eq. modified-weights2.  Synchronises `stream` (default: the current stream)."""
    if not records.is_cuda or records.numel() * records.element_size() % OBS_BYTES:
        raise ValueError("records must be a device tensor of whole pa_obs records")
    M = records.numel() * records.element_size() // OBS_BYTES
    lib = _lib.lib()
    stream = stream if stream is not None else torch.cuda.current_stream(records.device)
    out = torch.zeros((ctypes.sizeof(_lib.pa_weighted) + 7) // 8, dtype=torch.int64, device=records.device)
    st = lib.pa_weighted_average(ctypes.c_void_p(records.data_ptr()), M, {"standard": 0, "modified": 1}[mode],
                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    _check(lib, None, st)
    stream.synchronize()
    w = _lib.pa_weighted.from_buffer_copy(out.cpu().numpy().tobytes()[: ctypes.sizeof(_lib.pa_weighted)])
    return w.as_dict()


class PopulationAnnealing:
    """One population-annealing run on one GPU (device buffers owned by this object)."""

    def __init__(self, L: int, R: int, seed: int, resample: str = "nearest", capacity: int | None = None,
                 device: str | torch.device | None = None, stream: torch.cuda.Stream | None = None,
                 update: str = "metropolis"):
        self.lib = _lib.lib()
        self.L, self.N, self.R_target = int(L), int(L) * int(L), int(R)
        self.capacity = int(capacity if capacity is not None else default_capacity(R))
        self.seed = int(seed)
        kind = {"nearest": _lib.PA_RESAMPLE_NEAREST, "poisson": _lib.PA_RESAMPLE_POISSON,
                "multinomial": _lib.PA_RESAMPLE_MULTINOMIAL}[resample]
        upd = {"metropolis": _lib.PA_UPDATE_METROPOLIS, "heatbath": _lib.PA_UPDATE_HEATBATH}[update]
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.cfg = _lib.pa_config(L=self.L, resample=kind, R=self.R_target, capacity=self.capacity,
                                  seed=self.seed, update=upd)
        sizes = _lib.pa_sizes()
        _check(self.lib, None, self.lib.pa_query_sizes(ctypes.byref(self.cfg), ctypes.byref(sizes)))
        self.sizes = sizes
        dev = self.device
        u8, i32 = torch.uint8, torch.int32
        self.spins = [torch.empty(sizes.spin_bytes, dtype=u8, device=dev) for _ in range(2)]
        self.level = [torch.empty(self.capacity, dtype=i32, device=dev) for _ in range(2)]
        self.mag = [torch.empty(self.capacity, dtype=i32, device=dev) for _ in range(2)]
        self.fam = [torch.empty(self.capacity, dtype=i32, device=dev) for _ in range(2)]
        self.work = torch.empty(sizes.work_bytes, dtype=u8, device=dev)
        bufs = _lib.pa_buffers()
        for b in range(2):
            bufs.spins[b] = self.spins[b].data_ptr()
            bufs.level[b] = self.level[b].data_ptr()
            bufs.mag[b] = self.mag[b].data_ptr()
            bufs.fam[b] = self.fam[b].data_ptr()
        bufs.work = self.work.data_ptr()
        self._bufs = bufs
        ctx = ctypes.c_void_p()
        with torch.cuda.device(dev):
            st = self.lib.pa_init(ctypes.byref(self.cfg), ctypes.byref(bufs),
                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx))
        _check(self.lib, None, st)
        self.ctx = ctx

    # ------------------------------------------------------------------ method steps
    def resample(self, beta_new: float) -> None:
        _check(self.lib, self.ctx, self.lib.pa_resample(self.ctx, float(beta_new)))

    def anneal_step(self, theta: int) -> None:
        _check(self.lib, self.ctx, self.lib.pa_anneal_step(self.ctx, int(theta)))

    def record(self, dst: torch.Tensor) -> None:
        """Write a pa_obs record into `dst` (a device tensor of at least OBS_BYTES bytes)."""
        assert dst.is_cuda and dst.numel() * dst.element_size() >= OBS_BYTES
        _check(self.lib, self.ctx, self.lib.pa_record(self.ctx, ctypes.c_void_p(dst.data_ptr())))

    def observables(self) -> dict:
        o = pa_obs()
        _check(self.lib, self.ctx, self.lib.pa_observables(self.ctx, ctypes.byref(o)))
        return o.as_dict()

    def analyze(self, n_blocks: int = 100) -> dict:
        """Blocked and jackknife errors of <E> and <|M|> over the tree-ordered population,
        R_eff(E), R_eff(|M|), the jackknife error of C and the family entropy S_f with
        rho_s = R / exp(S_f) (pa_analyze; synchronising)."""
        out = _lib.pa_analysis()
        _check(self.lib, self.ctx, self.lib.pa_analyze(self.ctx, int(n_blocks), ctypes.byref(out)))
        return out.as_dict()

    def propose_schedule(self, alpha_target: float = 0.8, dbeta_max: float = 0.1, beta_final: float = 1.0):
        """Adaptive step: (beta_next, alpha) from overlap bisection on the current histogram."""
        b, a = ctypes.c_double(), ctypes.c_double()
        _check(self.lib, self.ctx, self.lib.pa_propose_schedule(self.ctx, float(alpha_target), float(dbeta_max),
                                                                float(beta_final), ctypes.byref(b), ctypes.byref(a)))
        return b.value, a.value

    def features(self, theta0: int = 10) -> np.ndarray:
        """The 12 learned-schedule inputs of the current population (float32)."""
        out = np.zeros(12, np.float32)
        _check(self.lib, self.ctx, self.lib.pa_features(self.ctx, int(theta0), out.ctypes.data))
        return out

    def decorrelation(self, with_sums: bool = False):
        """Correlation over replicas of the energy level after this step's resampling and now."""
        c = ctypes.c_double()
        sums = np.zeros(5, np.int64)
        _check(self.lib, self.ctx, self.lib.pa_decorrelation(self.ctx, ctypes.byref(c), sums.ctypes.data))
        return (c.value, sums) if with_sums else c.value

    def propose_learned(self, model, alpha_floor: float = 0.7, alpha_target: float = 0.8, dbeta_max: float = 0.1,
                        beta_final: float = 1.0, theta0: int = 10, theta_max: int = 40) -> dict:
        """Learned step (network proposal checked against the overlap floor, bisection fallback)."""
        out = _lib.pa_proposal()
        _check(self.lib, self.ctx, self.lib.pa_propose_learned(
            self.ctx, ctypes.byref(model.c_model()), float(alpha_floor), float(alpha_target), float(dbeta_max),
            float(beta_final), int(theta0), int(theta_max), ctypes.byref(out)))
        return out.as_dict()

    def schedule_log(self) -> list[dict]:
        n = ctypes.c_longlong()
        _check(self.lib, self.ctx, self.lib.pa_schedule_log(self.ctx, None, 0, ctypes.byref(n)))
        buf = (_lib.pa_sched_entry * max(1, n.value))()
        _check(self.lib, self.ctx, self.lib.pa_schedule_log(self.ctx, buf, n.value, ctypes.byref(n)))
        return [{f: getattr(buf[i], f) for f, _ in _lib.pa_sched_entry._fields_} for i in range(n.value)]

    def sync(self) -> None:
        _check(self.lib, self.ctx, self.lib.pa_sync(self.ctx))

    # ------------------------------------------------------------------ accessors
    @property
    def R(self) -> int:
        r = ctypes.c_longlong()
        _check(self.lib, self.ctx, self.lib.pa_population(self.ctx, ctypes.byref(r)))
        return int(r.value)

    def histogram(self) -> np.ndarray:
        h = np.zeros(self.N + 1, np.int32)
        _check(self.lib, self.ctx, self.lib.pa_histogram(self.ctx, h.ctypes.data))
        return h

    def replicas(self):
        R = self.R
        lv, mg, fm = (np.zeros(R, np.int32) for _ in range(3))
        _check(self.lib, self.ctx, self.lib.pa_replicas(self.ctx, lv.ctypes.data, mg.ctypes.data, fm.ctypes.data))
        return lv, mg, fm

    def copy_counts(self) -> np.ndarray:
        """Copy numbers r_j of the last resampling, one per parent (R_{i-1} entries)."""
        out = np.zeros(self.capacity, np.int32)
        n = ctypes.c_longlong()
        _check(self.lib, self.ctx, self.lib.pa_copy_counts(self.ctx, out.ctypes.data, ctypes.byref(n)))
        return out[: n.value].copy()

    def hashes(self) -> np.ndarray:
        out = np.zeros(self.R, np.uint64)
        _check(self.lib, self.ctx, self.lib.pa_hashes(self.ctx, out.ctypes.data))
        return out

    def export_spins(self, first: int = 0, count: int | None = None) -> np.ndarray:
        """Canonical packed words, shape (count, L, ceil(L/32)), bit c%32 of word c//32 = column c."""
        if count is None:
            count = self.R - first
        nw = (self.L + 31) // 32
        out = np.zeros((count, self.L, nw), np.uint32)
        _check(self.lib, self.ctx, self.lib.pa_export_spins(self.ctx, int(first), int(count), out.ctypes.data))
        return out

    def save(self) -> bytes:
        """Checkpoint of the whole run state (host bytes)."""
        n = ctypes.c_size_t()
        _check(self.lib, self.ctx, self.lib.pa_checkpoint_size(self.ctx, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(self.lib, self.ctx, self.lib.pa_save(self.ctx, buf, n.value))
        return buf.raw

    def load(self, data: bytes) -> None:
        """Restore a checkpoint written by save() for the same configuration."""
        buf = ctypes.create_string_buffer(data, len(data))
        _check(self.lib, self.ctx, self.lib.pa_load(self.ctx, buf, len(data)))

    def close(self) -> None:
        if getattr(self, "ctx", None):
            self.lib.pa_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
