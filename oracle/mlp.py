"""Oracle for the learned temperature schedule: features, MLP forward / backward, Adam.

TEST INFRASTRUCTURE (part of the oracle): plain numpy in float64.  Only tests/,
__graft_entry__.smoke() and bench.py's cpu_baseline leg may import it.

The network (a design choice; the paper has no learned schedule): 12 population-statistic
inputs -> 64 -> 64 -> 64 (tanh) -> 2 linear outputs, parameters stored as bfloat16 (round to
nearest even from float32), so the forward pass here uses exactly the parameter values the
GPU uses.  Loss: L = 1/(2B) sum_b sum_o (y_bo - t_bo)^2.
"""
from __future__ import annotations

import math

import numpy as np

IN, HID, OUT = 12, 64, 2
SHAPES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (HID, HID)), ("b3", (HID,)), ("W4", (OUT, HID)), ("b4", (OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)  # 9282


def unflatten(flat: np.ndarray) -> dict:
    out, off = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[off:off + n], dtype=np.float64).reshape(shape)
        off += n
    return out


def flatten(params: dict) -> np.ndarray:
    return np.concatenate([np.asarray(params[n], dtype=np.float64).ravel() for n, _ in SHAPES])


def bf16_round(x) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float32 values."""
    f = np.array(x, dtype=np.float32, copy=True, ndmin=1)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = ((bits + 0x7FFF + lsb) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).reshape(np.shape(x))


def forward(flat_bf16: np.ndarray, x: np.ndarray):
    """y and the hidden activations (a1, a2, a3) for a batch x of shape (B, 12)."""
    p = unflatten(flat_bf16)
    x = np.asarray(x, dtype=np.float64)
    a1 = np.tanh(x @ p["W1"].T + p["b1"])
    a2 = np.tanh(a1 @ p["W2"].T + p["b2"])
    a3 = np.tanh(a2 @ p["W3"].T + p["b3"])
    y = a3 @ p["W4"].T + p["b4"]
    return y, (a1, a2, a3)


def loss(flat_bf16: np.ndarray, x: np.ndarray, t: np.ndarray) -> float:
    y, _ = forward(flat_bf16, x)
    return float(0.5 * np.sum((y - t) ** 2) / len(x))


def backward(flat_bf16: np.ndarray, x: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Gradient of the loss with respect to the (flattened) parameters, by the chain rule."""
    p = unflatten(flat_bf16)
    x = np.asarray(x, dtype=np.float64)
    y, (a1, a2, a3) = forward(flat_bf16, x)
    B = len(x)
    g4 = (y - t) / B
    g3 = (g4 @ p["W4"]) * (1.0 - a3 ** 2)
    g2 = (g3 @ p["W3"]) * (1.0 - a2 ** 2)
    g1 = (g2 @ p["W2"]) * (1.0 - a1 ** 2)
    grads = {"W4": g4.T @ a3, "b4": g4.sum(0), "W3": g3.T @ a2, "b3": g3.sum(0),
             "W2": g2.T @ a1, "b2": g2.sum(0), "W1": g1.T @ x, "b1": g1.sum(0)}
    return flatten(grads)


def adam_step(theta, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) of the float64 master parameters; t counts from 1."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed: int) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    rng = np.random.default_rng(seed)
    out = []
    for name, shape in SHAPES:
        if name.startswith("W"):
            bound = 1.0 / math.sqrt(shape[1])
            out.append(rng.uniform(-bound, bound, size=shape).ravel())
        else:
            out.append(np.zeros(shape))
    return np.concatenate(out)


# ---------------------------------------------------------------------------- features
def features(L: int, hist, beta: float, dbeta_prev: float, theta_prev_over_theta0: float,
             alpha_prev: float, fam_sizes, counts_prev) -> np.ndarray:
    """The 12 inputs, computed in float64 from a population:
    beta, ln L, ln R, e = <E>/N, ln(Var(E)/N + 1e-12), skewness of E, excess kurtosis of E,
    previous dbeta * L, previous theta / theta0, previous overlap, ln(rho_t) / ln(R)
    (rho_t = sum of squared family sizes / R, Eq. rhot), fraction of parents with no copy in
    the last resampling."""
    N = L * L
    h = np.asarray(hist, dtype=np.float64)
    E = (4.0 * np.arange(N + 1) - 2.0 * N)
    R = h.sum()
    mean = (h * E).sum() / R
    d = E - mean
    var = (h * d * d).sum() / R
    m3 = (h * d ** 3).sum() / R
    m4 = (h * d ** 4).sum() / R
    skew = m3 / var ** 1.5 if var > 0 else 0.0
    kurt = m4 / var ** 2 - 3.0 if var > 0 else 0.0
    sizes = np.asarray(fam_sizes, dtype=np.float64)
    rho_t = (sizes ** 2).sum() / R
    lnR = math.log(R)
    c = np.asarray(counts_prev)
    frac0 = float((c == 0).mean()) if len(c) else 0.0
    return np.array([beta, math.log(L), lnR, mean / N, math.log(var / N + 1e-12), skew, kurt,
                     dbeta_prev * L, theta_prev_over_theta0, alpha_prev,
                     math.log(rho_t) / lnR if lnR > 0 else 0.0, frac0])


THETA_CORR = 0.3


def replica_correlation(E0, Et) -> float:
    """Pearson correlation over replicas of the energies right after resampling and after t
    sweeps (0 when either has no spread)."""
    a = np.asarray(E0, dtype=np.float64)
    b = np.asarray(Et, dtype=np.float64)
    a = a - a.mean()
    b = b - b.mean()
    d = math.sqrt(float((a * a).sum()) * float((b * b).sum()))
    return float((a * b).sum()) / d if d > 0 else 0.0


def theta_label(E0, E_after, theta_max: int, threshold: float = THETA_CORR) -> int:
    """Sweeps needed at a temperature step (a design rule; the paper's adaptive theta is not
    printed, Sec. X): the smallest t in 1..theta_max at which the replicas' energies after t
    sweeps have decorrelated from their values right after resampling,
    corr_j(E_j(0), E_j(t)) <= threshold; theta_max if none does.  E_after[t-1] holds the
    energies after t sweeps."""
    for t in range(1, min(len(E_after), theta_max) + 1):
        if replica_correlation(E0, E_after[t - 1]) <= threshold:
            return t
    return theta_max
