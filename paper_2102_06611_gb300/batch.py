"""Batches of independent population-annealing runs (C ABI pa_batch_*): each run has its own
L, R, number of temperatures (linear schedule beta_i = i / (n_temps - 1)), theta and seed; one
temperature step of every unfinished run per captured-graph replay."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib, _check, default_capacity


@dataclass
class RunSpec:
    L: int
    R: int
    seed: int
    n_temps: int
    theta: int
    resample: str = "nearest"
    capacity: int | None = None
    update: str = "metropolis"

    def desc(self) -> _lib.pa_run_desc:
        cap = self.capacity if self.capacity is not None else default_capacity(self.R)
        kind = {"nearest": _lib.PA_RESAMPLE_NEAREST, "poisson": _lib.PA_RESAMPLE_POISSON,
                "multinomial": _lib.PA_RESAMPLE_MULTINOMIAL}[self.resample]
        upd = {"metropolis": _lib.PA_UPDATE_METROPOLIS, "heatbath": _lib.PA_UPDATE_HEATBATH}[self.update]
        return _lib.pa_run_desc(_lib.pa_config(L=self.L, resample=kind, R=self.R, capacity=cap, seed=self.seed,
                                               update=upd),
                                self.n_temps, self.theta)


class Batch:
    def __init__(self, runs: list[RunSpec], device: str | torch.device | None = None,
                 stream: torch.cuda.Stream | None = None):
        self.lib = _lib.lib()
        self.runs = list(runs)
        self.n = len(runs)
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._descs = (_lib.pa_run_desc * self.n)(*[r.desc() for r in runs])
        nbytes = ctypes.c_size_t()
        _check(self.lib, None, self.lib.pa_batch_query_sizes(self.n, self._descs, ctypes.byref(nbytes)))
        self.arena = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(self.lib, None, self.lib.pa_batch_init(self.n, self._descs, ctypes.c_void_p(self.arena.data_ptr()),
                                                          nbytes.value, ctypes.c_void_p(self.stream.cuda_stream),
                                                          ctypes.byref(h)))
        self.h = h

    def step(self) -> None:
        _check(self.lib, None, self.lib.pa_batch_step(self.h))

    def status(self):
        active = np.zeros(self.n, np.int32)
        status = np.zeros(self.n, np.int32)
        step = np.zeros(self.n, np.int64)
        _check(self.lib, None, self.lib.pa_batch_status(self.h, active.ctypes.data, status.ctypes.data,
                                                        step.ctypes.data))
        return active, status, step

    def observables(self) -> list[dict]:
        recs = (_lib.pa_obs * self.n)()
        _check(self.lib, None, self.lib.pa_batch_observables(self.h, recs))
        return [recs[i].as_dict() for i in range(self.n)]

    def record(self, dst: torch.Tensor) -> None:
        _check(self.lib, None, self.lib.pa_batch_record(self.h, ctypes.c_void_p(dst.data_ptr())))

    def hashes(self, run: int) -> np.ndarray:
        cap = self._descs[run].cfg.capacity
        out = np.zeros(cap, np.uint64)
        n = ctypes.c_longlong()
        _check(self.lib, None, self.lib.pa_batch_hashes(self.h, run, out.ctypes.data, ctypes.byref(n)))
        return out[: n.value].copy()

    def tuning(self) -> dict:
        t = _lib.pa_batch_tuning()
        _check(self.lib, None, self.lib.pa_batch_get_tuning(self.h, ctypes.byref(t)))
        shapes = [{"unified": c.unified, "blocks_per_sm": c.blocks_per_sm, "ipw_scale": c.ipw_scale, "ms": c.ms}
                  for c in t.cand[: t.n_candidates]]
        chosen = shapes[t.chosen] if 0 <= t.chosen < len(shapes) else None
        return {"chosen": chosen, "chosen_grid": t.chosen_grid, "candidates": shapes}

    def set_shape(self, unified: int, blocks_per_sm: int, ipw_scale: int = 1) -> None:
        """Fix the sweep phase's shape instead of the autotuner's choice (same results)."""
        sh = _lib.pa_batch_shape(unified=int(unified), blocks_per_sm=int(blocks_per_sm), ipw_scale=int(ipw_scale))
        _check(self.lib, None, self.lib.pa_batch_set_shape(self.h, ctypes.byref(sh)))

    def run_to_end(self, max_steps: int = 100000) -> int:
        steps = 0
        while steps < max_steps:
            active, _, _ = self.status()
            if not active.any():
                break
            self.step()
            steps += 1
        return steps

    def close(self):
        if getattr(self, "h", None):
            self.lib.pa_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mixed_runs(n: int = 64, seed: int = 2102, first_seed: int = 100) -> list[RunSpec]:
    """A batch of n independent runs with L drawn from {8, 12, 16, 24, 32, 48, 64}, R
    log-uniform in [1e3, 2e5], 51 - 301 temperatures, theta in {1, 5, 10}, nearest-integer
    resampling, run seeds first_seed .. first_seed + n - 1 (the parameters come from a numpy
    generator seeded with `seed`)."""
    rng = np.random.default_rng(seed)
    Ls = np.array([8, 12, 16, 24, 32, 48, 64])
    out = []
    for i in range(n):
        L = int(rng.choice(Ls))
        R = int(round(10 ** rng.uniform(3.0, np.log10(2e5))))
        n_temps = int(rng.integers(51, 302))
        theta = int(rng.choice([1, 5, 10]))
        out.append(RunSpec(L, R, first_seed + i, n_temps, theta))
    return out
