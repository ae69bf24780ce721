"""Pins of the oracle's learned-schedule pieces: bfloat16 rounding, the MLP gradient
(finite differences), the Adam step (closed forms of its first steps) and the features
(moments from per-replica energies instead of the histogram)."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp


def test_param_count():
    assert mlp.N_PARAMS == 9282


def test_bf16_round_to_nearest_even():
    one = 1.0
    cases = {one: one, one + 2.0 ** -8: one,            # tie -> even (mantissa ...0)
             one + 3 * 2.0 ** -8: one + 2.0 ** -6,      # tie -> even (rounds up)
             one + 2.0 ** -8 + 2.0 ** -20: one + 2.0 ** -7,
             -2.5: -2.5, 0.0: 0.0}
    for x, want in cases.items():
        got = float(mlp.bf16_round(np.float32(x)))
        assert got == pytest.approx(want, rel=1e-7), (x, got, want)
    r = np.random.default_rng(0).standard_normal(10000).astype(np.float32)
    b = mlp.bf16_round(r)
    assert np.all(b.view(np.uint32) & 0xFFFF == 0)
    assert np.max(np.abs(b - r) / np.abs(r)) <= 2.0 ** -8


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    flat = mlp.bf16_round(mlp.init_params(3)).astype(np.float64)
    x = rng.standard_normal((7, mlp.IN))
    t = rng.standard_normal((7, mlp.OUT))
    g = mlp.backward(flat, x, t)
    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 60, replace=False), [0, mlp.N_PARAMS - 1]])
    for i in idx:
        h = 1e-6
        e = np.zeros(mlp.N_PARAMS)
        e[i] = h
        fd = (mlp.loss(flat + e, x, t) - mlp.loss(flat - e, x, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_adam_first_step_is_lr_times_sign():
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = mlp.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, lr=0.01)
    assert np.allclose(th, -0.01 * np.sign(g), rtol=1e-4)


def test_adam_constant_gradient_steps_by_lr():
    """With the same gradient at every step the bias-corrected moments equal g and g^2 at
    every t (m_t = (1 - b1^t) g, v_t = (1 - b2^t) g^2), so each step moves lr * sign(g):
    after t steps theta = -t lr sign(g).  A bias correction with a fixed t = 1 would move
    (1 + b1) / sqrt(1 + b2) ~ 1.34 lr at step 2."""
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for t in (1, 2, 3):
        th, m, v = mlp.adam_step(th, m, v, g, t, lr=0.01)
        assert np.allclose(th, -0.01 * t * np.sign(g), rtol=1e-4), t


def test_adam_second_step_after_zero_gradient():
    """Gradient g at step 1 and 0 at step 2: m_2 = b1 (1 - b1) g and v_2 = b2 (1 - b2) g^2, so
    the bias-corrected step is lr sign(g) (b1 / (1 + b1)) / sqrt(b2 / (1 + b2)); with
    b1 = 0.9, b2 = 0.999 that is 0.670058 lr (to 6 digits)."""
    g = np.array([0.5, -4.0])
    th, m, v = mlp.adam_step(np.zeros(2), np.zeros(2), np.zeros(2), g, 1, lr=0.01)
    th2, _, _ = mlp.adam_step(th, m, v, np.zeros(2), 2, lr=0.01)
    assert np.allclose(th2 - th, -0.01 * 0.670058 * np.sign(g), rtol=2e-6)


def test_features_from_population():
    L, R = 8, 3000
    pa = oracle.PA(L, R, seed=5)
    pa.init()
    pa.resample(0.3)
    counts = pa.counts()
    pa.sweep(3)
    E, M, fam = pa.state()
    _, sizes = np.unique(fam, return_counts=True)
    f = mlp.features(L, pa.histogram(), 0.3, 0.3, 0.3, 0.9, sizes, counts)
    N = L * L
    Ef = E.astype(np.float64)
    assert f[0] == 0.3 and f[1] == pytest.approx(math.log(8)) and f[2] == pytest.approx(math.log(len(E)))
    assert f[3] == pytest.approx(Ef.mean() / N, rel=1e-12)
    assert f[4] == pytest.approx(math.log(Ef.var() / N + 1e-12), rel=1e-12)
    z = (Ef - Ef.mean()) / Ef.std()
    assert f[5] == pytest.approx((z ** 3).mean(), rel=1e-9, abs=1e-12)
    assert f[6] == pytest.approx((z ** 4).mean() - 3, rel=1e-9)
    assert f[7] == pytest.approx(0.3 * L) and f[8] == 0.3 and f[9] == 0.9
    assert f[10] == pytest.approx(math.log((sizes.astype(float) ** 2).sum() / len(E)) / math.log(len(E)))
    assert f[11] == pytest.approx((counts == 0).mean())


def test_theta_label_rule():
    """An AR(1) chain per replica with known autocorrelation rho^t crosses 0.3 at
    t = ceil(ln 0.3 / ln rho)."""
    rng = np.random.default_rng(6)
    R = 200000
    for rho, want in ((0.5, 2), (0.8, 6), (0.95, 24)):
        E0 = rng.standard_normal(R)
        E, after = E0.copy(), []
        for t in range(40):
            E = rho * E + math.sqrt(1 - rho * rho) * rng.standard_normal(R)
            after.append(E)
        assert mlp.theta_label(E0, after, 40) == want
        assert mlp.replica_correlation(E0, after[0]) == pytest.approx(rho, abs=0.01)
    assert mlp.theta_label(E0, [E0] * 5, 5) == 5          # never decorrelates: theta_max
    assert mlp.replica_correlation(np.ones(10), np.arange(10)) == 0.0
