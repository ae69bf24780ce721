"""Learned temperature schedule: training data from the plain adaptive method, training of the
schedule network with the library's own kernels, and annealing drivers for the plain and the
learned schedule.

The paper has no learned schedule (it names self-adaptive steps, Sec. II, an overlap of about
0.7 or more, and an adaptive number of sweeps, Sec. X).  Here a small network proposes the next
(dbeta, theta) from population statistics; the library keeps the step only if the energy-
histogram overlap reaches a floor, and falls back to the plain overlap bisection otherwise.

Training data come from plain runs: dbeta from the overlap bisection (target 0.8) and theta
from a decorrelation rule -- after resampling, sweeps are run one at a time and theta is the
first t <= theta_max at which the replicas' energies have decorrelated from their values right
after resampling, corr_j(E_j(0), E_j(t)) <= 0.3.  Copies made by resampling start identical, so
this measures how long the chain needs to make them independent; it grows where relaxation is
slow (near the critical point) and is one or two sweeps elsewhere.  Targets: ln(dbeta sigma_E)
with sigma_E the energy standard deviation of the population, and ln(theta).
"""
from __future__ import annotations

import ctypes
import math
import time

import numpy as np
import torch

from . import _lib
from . import PopulationAnnealing, _check

N_PARAMS, N_IN, N_OUT, N_HID = 9282, 12, 2, 64
SHAPES = [(N_HID, N_IN), (N_HID,), (N_HID, N_HID), (N_HID,), (N_HID, N_HID), (N_HID,), (N_OUT, N_HID), (N_OUT,)]


def _vp(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def initial_parameters(seed: int) -> np.ndarray:
    """Uniform(+-1/sqrt(fan_in)) weights and zero biases, in the flat parameter order."""
    rng = np.random.default_rng(seed)
    parts = []
    for shape in SHAPES:
        if len(shape) == 2:
            b = 1.0 / math.sqrt(shape[1])
            parts.append(rng.uniform(-b, b, size=shape).ravel())
        else:
            parts.append(np.zeros(shape))
    return np.concatenate(parts).astype(np.float32)


class ScheduleMLP:
    """Parameters (float32 master, Adam moments, bfloat16 copy) and input/output scaling on a GPU."""

    def __init__(self, master: np.ndarray | None = None, norm: np.ndarray | None = None, seed: int = 0,
                 device: str | torch.device = "cuda"):
        self.lib = _lib.lib()
        assert self.lib.pa_mlp_param_count() == N_PARAMS
        self.device = torch.device(device)
        m = initial_parameters(seed) if master is None else np.asarray(master, np.float32)
        self.master = torch.tensor(m, dtype=torch.float32, device=self.device)
        self.m = torch.zeros(N_PARAMS, dtype=torch.float32, device=self.device)
        self.v = torch.zeros(N_PARAMS, dtype=torch.float32, device=self.device)
        self.params = torch.zeros(N_PARAMS, dtype=torch.int16, device=self.device)  # bfloat16 patterns
        n = np.concatenate([np.zeros(N_IN), np.ones(N_IN), np.zeros(N_OUT), np.ones(N_OUT)]) if norm is None else norm
        self.norm = torch.tensor(np.asarray(n, np.float32), device=self.device)
        self.adam_steps = 0
        self._call(self.lib.pa_mlp_round(_vp(self.master), _vp(self.params), self._stream()))

    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    @staticmethod
    def _call(status: int):
        _check(_lib.lib(), None, status)

    def c_model(self) -> _lib.pa_learned_model:
        return _lib.pa_learned_model(self.params.data_ptr(), self.norm.data_ptr())

    # Lower bounds of the input scales: an input that barely varies in the training runs (ln R
    # at a fixed population size, the overlap near its target) must stay O(1) after
    # standardisation for other lattice or population sizes.  Order: beta, ln L, ln R, e,
    # ln(Var/N), skewness, kurtosis, dbeta_prev L, theta_prev/theta0, alpha_prev,
    # ln rho_t / ln R, zero-copy fraction.
    X_STD_FLOOR = np.array([0.05, 0.5, 2.0, 0.05, 0.1, 0.1, 0.1, 0.05, 0.1, 0.05, 0.05, 0.05])

    def set_norm(self, x_mean, x_std, y_mean, y_std):
        n = np.concatenate([x_mean, np.maximum(x_std, self.X_STD_FLOOR), y_mean,
                            np.maximum(y_std, 1e-6)]).astype(np.float32)
        self.norm.copy_(torch.from_numpy(n))

    def forward(self, x: torch.Tensor, act: torch.Tensor | None = None) -> torch.Tensor:
        """Standardised outputs for standardised inputs x (B x 12, float32, on the device)."""
        x = x.contiguous()
        y = torch.empty((x.shape[0], N_OUT), dtype=torch.float32, device=self.device)
        self._call(self.lib.pa_mlp_forward(_vp(self.params), _vp(x), x.shape[0], _vp(y),
                                           _vp(act) if act is not None else None, self._stream()))
        return y

    def gradient(self, x: torch.Tensor, t: torch.Tensor):
        B = x.shape[0]
        act = torch.empty((B, 3 * N_HID), dtype=torch.float32, device=self.device)
        y = self.forward(x, act)
        delta = torch.empty((B, 3 * N_HID + N_OUT), dtype=torch.float32, device=self.device)
        grad = torch.empty(N_PARAMS, dtype=torch.float32, device=self.device)
        self._call(self.lib.pa_mlp_backward(_vp(self.params), _vp(x), _vp(t.contiguous()), B, _vp(act), _vp(y),
                                            _vp(delta), _vp(grad), self._stream()))
        return grad, y

    def adam(self, grad: torch.Tensor, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
        self.adam_steps += 1
        self._call(self.lib.pa_mlp_adam(_vp(self.master), _vp(self.m), _vp(self.v), _vp(grad), self.adam_steps,
                                        float(lr), float(b1), float(b2), float(eps), _vp(self.params), self._stream()))

    def train(self, X: np.ndarray, Y: np.ndarray, steps: int = 3000, batch: int = 256, lr: float = 2e-3,
              seed: int = 0) -> list[float]:
        """Adam on the mean squared error of standardised outputs; the scaling is set from the data."""
        X = np.asarray(X, np.float64)
        Y = np.asarray(Y, np.float64)
        self.set_norm(X.mean(0), X.std(0), Y.mean(0), Y.std(0))
        n = self.norm.cpu().numpy().astype(np.float64)
        Xs = torch.tensor((X - n[:N_IN]) / n[N_IN:2 * N_IN], dtype=torch.float32, device=self.device)
        Ys = torch.tensor((Y - n[2 * N_IN:2 * N_IN + N_OUT]) / n[2 * N_IN + N_OUT:], dtype=torch.float32,
                          device=self.device)
        rng = np.random.default_rng(seed)
        losses = []
        for s in range(steps):
            idx = torch.from_numpy(rng.integers(0, len(X), size=min(batch, len(X)))).to(self.device)
            xb, tb = Xs[idx], Ys[idx]
            rate = lr * 0.5 * (1.0 + math.cos(math.pi * s / steps))
            grad, y = self.gradient(xb, tb)
            self.adam(grad, rate)
            if s % 200 == 0 or s == steps - 1:
                losses.append(float(0.5 * ((y - tb) ** 2).sum(1).mean()))
        return losses

    def save(self, path: str):
        np.savez(path, master=self.master.cpu().numpy(), norm=self.norm.cpu().numpy())

    @classmethod
    def load(cls, path: str, device="cuda") -> "ScheduleMLP":
        d = np.load(path)
        return cls(master=d["master"], norm=d["norm"], device=device)


# ------------------------------------------------------------------------------ data
THETA_CORR = 0.3


def _correlation(a: np.ndarray, b: np.ndarray) -> float:
    a = a - a.mean()
    b = b - b.mean()
    d = math.sqrt(float((a * a).sum()) * float((b * b).sum()))
    return float((a * b).sum()) / d if d > 0 else 0.0


def energy_width(L: int, raw_features: np.ndarray) -> float:
    """sigma_E of the population from raw feature 4 = ln(Var(E)/N + 1e-12), as the kernel does."""
    return math.sqrt(L * L * math.exp(float(np.float32(raw_features[4]))))


def plain_training_run(L: int, R: int, seed: int, alpha_target: float = 0.8, theta0: int = 10,
                       theta_max: int = 40, dbeta_max: float = 0.1, beta_final: float = 1.0, device="cuda"):
    """(features, targets) of one plain adaptive run: targets ln(dbeta sigma_E), ln(theta)."""
    pa = PopulationAnnealing(L, R, seed, device=device)
    X, Y = [], []
    beta = 0.0
    while beta < beta_final:
        f = pa.features(theta0)
        b_next, _ = pa.propose_schedule(alpha_target, dbeta_max, beta_final)
        pa.resample(b_next)
        theta = theta_max
        for t in range(1, theta_max + 1):
            pa.anneal_step(1)
            if pa.decorrelation() <= THETA_CORR:
                theta = t
                break
        X.append(f)
        Y.append([math.log((b_next - beta) * energy_width(L, f)), math.log(theta)])
        beta = b_next
    pa.close()
    return np.array(X, np.float64), np.array(Y, np.float64)


# ------------------------------------------------------------------------------ drivers
def anneal(pa: PopulationAnnealing, mode: str = "plain", model: ScheduleMLP | None = None,
           alpha_target: float = 0.8, alpha_floor: float = 0.7, theta0: int = 10, theta_max: int = 40,
           dbeta_max: float = 0.1, beta_final: float = 1.0, corr_target: float = THETA_CORR) -> dict:
    """Anneal from the population's current beta to beta_final and time it (every proposal and
    check included).

    plain:   overlap bisection (alpha_target) and theta0 sweeps per temperature.
    rule:    overlap bisection (alpha_target) for dbeta and the decorrelation rule without the
             network for theta: one sweep at a time until the replicas' energy levels have
             decorrelated from their values after resampling (corr <= corr_target) or theta_max
             sweeps have run -- the rule that labels the network's training data.
    learned: the network proposes (dbeta, theta); dbeta is kept if the overlap reaches
             alpha_floor (else the bisection decides and theta0 sweeps are used); theta - 1 of
             the proposed sweeps run in one launch (the proposal, whose error is about a sweep,
             taken as a lower estimate), then the decorrelation since resampling is measured
             and, while it is above corr_target, one more sweep runs (up to theta_max) -- the
             same stopping rule as "rule", with most sweeps batched into one launch.
    """
    if mode not in ("plain", "rule", "learned"):
        raise ValueError(f"unknown schedule mode {mode!r}")
    torch.cuda.synchronize(pa.device)
    t0 = time.perf_counter()
    beta, steps, sweeps, fallbacks, extended = 0.0, 0, 0, 0, 0
    while beta < beta_final:
        if mode in ("plain", "rule"):
            b, _ = pa.propose_schedule(alpha_target, dbeta_max, beta_final)
            theta = theta0
        else:
            p = pa.propose_learned(model, alpha_floor, alpha_target, dbeta_max, beta_final, theta0, theta_max)
            b, theta = p["beta_next"], p["theta_next"]
            fallbacks += p["source"] == _lib.PA_SCHED_FALLBACK
        pa.resample(b)
        if mode == "rule":
            theta = 0
            while theta < theta_max:
                pa.anneal_step(1)
                theta += 1
                if pa.decorrelation() <= corr_target:
                    break
        elif mode == "learned":
            if theta > 1 and p["source"] == _lib.PA_SCHED_LEARNED:
                theta -= 1
            pa.anneal_step(theta)
            while theta < theta_max and pa.decorrelation() > corr_target:
                pa.anneal_step(1)
                theta += 1
                extended += 1
        else:
            pa.anneal_step(theta)
        steps += 1
        sweeps += theta
        beta = b
    obs = pa.observables()
    wall = time.perf_counter() - t0
    return {"mode": mode, "wall_s": wall, "steps": steps, "sweeps": sweeps, "fallbacks": fallbacks,
            "extensions": extended, "minus_betaF": obs["minus_betaF"], "e": obs["e"], "R": obs["R"],
            "beta": obs["beta"]}
