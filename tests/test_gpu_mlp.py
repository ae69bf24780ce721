"""Learned-schedule kernels vs the oracle: network forward, gradients and Adam against the
float64 oracle on the same bfloat16 parameters; population features; and a learned anneal
replayed by the oracle (the overlap check and the fallback bisection bit for bit)."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from side_by_side import compare_population

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _model(seed=3, norm=None):
    from paper_2102_06611_gb300.learned import ScheduleMLP
    return ScheduleMLP(seed=seed, norm=norm)


def _bf16_params(model):
    return model.params.cpu().numpy().view(np.uint16).astype(np.uint32) << 16


def test_bf16_copy_is_round_to_nearest_even():
    m = _model()
    bits = _bf16_params(m).astype(np.uint32)
    want = omlp.bf16_round(m.master.cpu().numpy())
    assert np.array_equal(bits.view(np.float32), want)


def test_forward_matches_oracle():
    m = _model(seed=5)
    P = _bf16_params(m).view(np.float32).astype(np.float64)
    x = np.random.default_rng(1).standard_normal((37, 12)).astype(np.float32)
    y = m.forward(torch.tensor(x, device="cuda")).cpu().numpy()
    y_ref, _ = omlp.forward(P, x.astype(np.float64))
    assert np.max(np.abs(y - y_ref)) <= 1e-5 * (1 + np.max(np.abs(y_ref)))


@pytest.mark.parametrize("B", [1, 5, 300])
def test_gradient_matches_oracle(B):
    m = _model(seed=7)
    P = _bf16_params(m).view(np.float32).astype(np.float64)
    rng = np.random.default_rng(B)
    x = rng.standard_normal((B, 12)).astype(np.float32)
    t = rng.standard_normal((B, 2)).astype(np.float32)
    g, _ = m.gradient(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"))
    g = g.cpu().numpy().astype(np.float64)
    g_ref = omlp.backward(P, x.astype(np.float64), t.astype(np.float64))
    scale = np.max(np.abs(g_ref))
    assert np.max(np.abs(g - g_ref)) <= 1e-3 * scale
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)


def test_adam_step_matches_oracle():
    m = _model(seed=9)
    master0 = m.master.cpu().numpy().astype(np.float64)
    g = np.random.default_rng(2).standard_normal(omlp.N_PARAMS).astype(np.float32)
    gt = torch.tensor(g, device="cuda")
    th = master0
    mm = np.zeros_like(th)
    vv = np.zeros_like(th)
    for step in (1, 2, 3):
        m.adam(gt, 1e-3)
        th, mm, vv = omlp.adam_step(th, mm, vv, g.astype(np.float64), step, 1e-3)
    got = m.master.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - th)) <= 1e-6
    assert np.array_equal(_bf16_params(m).view(np.float32), omlp.bf16_round(m.master.cpu().numpy()))


def test_features_match_oracle():
    from paper_2102_06611_gb300 import PopulationAnnealing
    L, R, seed = 16, 3000, 4
    gpu = PopulationAnnealing(L, R, seed)
    ref = oracle.PA(L, R, seed, capacity=gpu.capacity)
    ref.init()
    f0 = gpu.features(10)
    f0_ref = omlp.features(L, ref.histogram(), 0.0, 0.0, 0.0, 1.0, np.ones(R), [])
    assert np.allclose(f0, f0_ref, rtol=2e-6, atol=1e-6)
    b, a = gpu.propose_schedule(0.8, 0.1, 1.0)
    gpu.resample(b)
    ref.resample(b)
    gpu.anneal_step(4)
    ref.sweep(4)
    counts = ref.counts()
    _, _, fam = ref.state()
    _, sizes = np.unique(fam, return_counts=True)
    f1 = gpu.features(10)
    f1_ref = omlp.features(L, ref.histogram(), b, b, 4 / 10, a, sizes, counts)
    assert np.allclose(f1, f1_ref, rtol=2e-6, atol=1e-6), (f1, f1_ref)


def test_decorrelation_sums_match_oracle():
    """The sweep kernel's exact sums of the levels at the step start and now, across two calls
    at the same temperature, against the oracle's energies."""
    from paper_2102_06611_gb300 import PopulationAnnealing
    L, R, seed = 16, 2000, 6
    N = L * L
    gpu = PopulationAnnealing(L, R, seed)
    ref = oracle.PA(L, R, seed, capacity=gpu.capacity)
    ref.init()
    gpu.resample(0.35)
    ref.resample(0.35)
    k0 = (ref.state()[0].astype(np.int64) + 2 * N) // 4
    for theta in (2, 3):
        gpu.anneal_step(theta)
        ref.sweep(theta)
        k1 = (ref.state()[0].astype(np.int64) + 2 * N) // 4
        c, sums = gpu.decorrelation(with_sums=True)
        want = [k0.sum(), (k0 * k0).sum(), k1.sum(), (k1 * k1).sum(), (k0 * k1).sum()]
        assert [int(x) for x in sums] == [int(x) for x in want]
        assert c == pytest.approx(float(np.corrcoef(k0, k1)[0, 1]), abs=1e-12)


def test_decorrelation_and_magnetisation_sums_in_the_ground_state():
    """Deep in the ordered phase nearly every replica starts the step at level 0; the sums
    must still count every replica (|M|, M^2 and the level sums)."""
    from paper_2102_06611_gb300 import PopulationAnnealing
    L, R, seed = 4, 3000, 9
    N = L * L
    gpu = PopulationAnnealing(L, R, seed)
    ref = oracle.PA(L, R, seed, capacity=gpu.capacity)
    ref.init()
    for beta in (0.5, 1.0, 2.0, 3.0):
        gpu.resample(beta)
        ref.resample(beta)
        k0 = (ref.state()[0].astype(np.int64) + 2 * N) // 4
        gpu.anneal_step(1)
        ref.sweep(1)
    E1, M1, _ = ref.state()
    k1 = (E1.astype(np.int64) + 2 * N) // 4
    assert (k0 == 0).mean() > 0.9
    c, sums = gpu.decorrelation(with_sums=True)
    assert [int(x) for x in sums] == [int(k0.sum()), int((k0 * k0).sum()), int(k1.sum()), int((k1 * k1).sum()),
                                      int((k0 * k1).sum())]
    o = gpu.observables()
    assert o["sum_absM"] == int(np.abs(M1).sum()) and o["sum_M2"] == int((M1.astype(np.int64) ** 2).sum())


def test_learned_anneal_replayed_by_oracle():
    """The network's proposals go through the overlap floor; the oracle, given each proposed
    dbeta, takes the same decision and the same fallback bisection, and the populations stay
    identical."""
    from paper_2102_06611_gb300 import PopulationAnnealing, _lib
    L, R, seed = 16, 2500, 8
    norm = np.concatenate([np.zeros(12), np.full(12, 5.0), [np.log(0.02 * L), np.log(5.0)], [0.6, 0.6]])
    model = _model(seed=11, norm=norm)
    gpu = PopulationAnnealing(L, R, seed)
    ref = oracle.PA(L, R, seed, capacity=gpu.capacity)
    ref.init()
    beta, sources = 0.0, []
    for i in range(200):
        p = gpu.propose_learned(model, alpha_floor=0.7, alpha_target=0.8, dbeta_max=0.1, beta_final=1.0,
                                theta0=10, theta_max=40)
        h = ref.histogram().astype(np.int64)
        b, a, src = oracle.accept_or_bisect(L * L, h, beta, 1.0, 0.1, p["dbeta_prop"], 0.7, 0.8)
        assert (p["beta_next"], p["alpha"], p["source"]) == (b, a, src), (i, p, b, a, src)
        assert 1 <= p["theta_prop"] <= 40
        assert p["theta_next"] == (p["theta_prop"] if src == 2 else 10)
        gpu.resample(b)
        assert ref.resample(b) == 0
        gpu.anneal_step(p["theta_next"])
        ref.sweep(p["theta_next"])
        sources.append(src)
        beta = b
        if beta == 1.0:
            break
    assert beta == 1.0
    compare_population(gpu, ref, "end of learned anneal")
    log = gpu.schedule_log()
    assert [e["source"] for e in log] == sources
    assert set(sources) <= {_lib.PA_SCHED_LEARNED, _lib.PA_SCHED_FALLBACK}


def test_training_reduces_the_loss():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((2000, 12))
    Y = np.stack([np.sin(X[:, 0]) + 0.5 * X[:, 1], X[:, 2] * X[:, 3]], 1)
    m = _model(seed=1)
    losses = m.train(X, Y, steps=800, batch=256, lr=3e-3)
    assert losses[-1] < 0.3 * losses[0]
