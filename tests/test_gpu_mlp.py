"""The warm-start network's CUDA kernels against the FP64 numpy oracle, and
what the trained network gains over cold starts."""
import numpy as np
import pytest

from oracle import mlp as ref
from paper_1204_4098_gb300 import inputs, lbm, warmstart

pytestmark = pytest.mark.gpu


def _setup(seed, n):
    rng = np.random.default_rng(seed)
    theta = ref.init_params(seed) + 0.05 * rng.standard_normal(ref.N_PARAMS)
    X = rng.uniform(-1, 1, (n, 4))
    T = rng.standard_normal((n, 3))
    return theta, X, T


@pytest.mark.parametrize("n", [1, 37, 128])
def test_gradient_matches_oracle(n):
    theta, X, T = _setup(n, n)
    net = lbm.MLP(theta.astype(np.float32))
    loss, g = net.gradient(X, T)
    want_loss, want = ref.gradient(theta.astype(np.float32).astype(np.float64),
                                   X.astype(np.float32), T.astype(np.float32))
    assert loss == pytest.approx(want_loss, rel=1e-5)
    assert np.max(np.abs(g - want)) <= 2e-5 * np.max(np.abs(want)) + 1e-8


def test_predict_matches_oracle():
    theta, X, _ = _setup(9, 1000)
    net = lbm.MLP(theta.astype(np.float32))
    y = net.predict(X)
    want, _ = ref.forward(theta.astype(np.float32).astype(np.float64), X.astype(np.float32))
    assert np.max(np.abs(y - want)) < 1e-5


def test_training_matches_oracle_adam():
    theta, X, T = _setup(4, 96)
    th32 = theta.astype(np.float32)
    rng = np.random.default_rng(0)
    order = np.stack([rng.permutation(96) for _ in range(4)])
    net = lbm.MLP(th32)
    net.train(X, T, order, batch=40, lr=1e-3)  # 3 minibatches (40, 40, 16) per epoch
    got = net.params()
    want, _ = ref.adam_train(th32.astype(np.float64), X.astype(np.float32),
                             T.astype(np.float32), order, batch=40, lr=1e-3)
    diff = np.abs(got - want)
    assert np.quantile(diff, 0.99) < 1e-5 and diff.max() < 2e-3
    assert ref.loss(got.astype(np.float64), X, T) == pytest.approx(ref.loss(want, X, T), rel=1e-3)


def test_warm_start_cuts_whole_sweep_gpu_time():
    """Train on cold runs of narrow slabs, then start held-out sweep points
    from the network's prediction.  Warm and cold batched runs stop by the
    same rule (TREND); the whole warm sweep -- fallbacks, divergences and the
    slowest run included -- takes less GPU time than the whole cold sweep,
    converges in fewer steps on average, and reaches the same coexistence
    densities (within 1e-3) on every run converged in both."""
    X, Y, info = warmstart.training_data(1500, seed=40, ny_range=(112, 160), max_steps=60000)
    assert info["converged"] >= 300, info
    model = warmstart.train(X, Y, stages=((800, 3e-3), (800, 5e-4), (800, 1e-4)), batch=64,
                            seed=1)
    held = inputs.sweep_instances(48, seed=41, nx_range=(64, 64), ny_range=(128, 128))
    warm, winfo = warmstart.run_warm(held, model, max_steps=60000)
    cold, cinfo = warmstart.run_cold_batched(held, max_steps=60000)
    both = [k for k in range(len(held)) if warm[k]["status"] == lbm.RUN_CONVERGED
            and cold[k]["status"] == lbm.RUN_CONVERGED]
    assert len(both) >= 8
    for k in both:
        assert warm[k]["rho_l"] == pytest.approx(cold[k]["rho_l"], rel=1e-3)
        assert warm[k]["rho_g"] == pytest.approx(cold[k]["rho_g"], rel=1e-3)
    s_warm = np.mean([warm[k]["steps"] for k in both])
    s_cold = np.mean([cold[k]["steps"] for k in both])
    print(f"warm start: {len(both)} converged in both; whole sweep GPU warm "
          f"{winfo['gpu_ms'] / 1e3:.2f} s, cold {cinfo['gpu_ms'] / 1e3:.2f} s; mean steps warm "
          f"{s_warm:.0f}, cold {s_cold:.0f}; fallbacks {winfo['fallbacks']}, train loss "
          f"{model.train_loss:.3e}")
    assert winfo["gpu_ms"] < cinfo["gpu_ms"]
    assert s_warm < s_cold
