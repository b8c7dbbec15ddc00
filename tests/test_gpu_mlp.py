"""The planner network's CUDA kernels (forward, MSE backward, Adam) against
the FP64 oracle, and the planner's ensemble on a synthetic timing law."""

import numpy as np
import pytest
import torch

from oracle import mlp as ref
from paper_2603_01443_gb300 import planner

pytestmark = pytest.mark.gpu

DIMS = [8, 64, 64, 64, 4]


def problem(seed, n=300):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, DIMS[0]))
    t = np.stack([np.sin(x[:, 0]) + x[:, 1], x[:, 2] * x[:, 3], np.abs(x[:, 4]), x[:, 5] - x[:, 6]],
                 axis=1)
    return x, t


def test_forward_matches_oracle(cuda_lib):
    net = planner.MLP(DIMS, seed=3)
    x, _ = problem(1)
    got = net.forward(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy()
    want = ref.forward(DIMS, net.params.cpu().numpy().astype(np.float64), x)[-1]
    assert np.max(np.abs(got - want)) <= 1e-5 * (1 + np.max(np.abs(want)))


def test_training_matches_oracle(cuda_lib):
    net = planner.MLP(DIMS, seed=5)
    x, t = problem(2)
    p0 = net.params.cpu().numpy().astype(np.float64)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    tt = torch.tensor(t, dtype=torch.float32, device="cuda")
    # first step: every parameter moves by lr against the sign of its gradient
    loss = net.train(xt, tt, 1, 1e-3).cpu().numpy()
    g = ref.gradient(DIMS, p0, x, t)
    p1_ref, _, _, losses = ref.adam_steps(DIMS, p0, x, t, 1, 1e-3)
    assert loss[0] == pytest.approx(losses[0], rel=1e-5)
    big = np.abs(g) > 1e-3 * np.max(np.abs(g))
    assert np.allclose(net.params.cpu().numpy()[big], p1_ref[big], atol=2e-6)
    # 40 more steps continue from the same moments (each call counts its
    # steps from 1 for the bias correction, the oracle likewise)
    loss = net.train(xt, tt, 40, 1e-3).cpu().numpy()
    _, m1, v1, _ = ref.adam_steps(DIMS, p0, x, t, 1, 1e-3)
    _, _, _, curve = ref.adam_steps(DIMS, p1_ref, x, t, 40, 1e-3, m1, v1)
    assert np.allclose(loss, curve, rtol=2e-3)
    assert loss[-1] < loss[0]


def test_planner_learns_a_timing_law(cuda_lib):
    rng = np.random.default_rng(0)
    n = 1500
    X = np.column_stack([rng.integers(14, 31, n), rng.uniform(2, 6, n), rng.integers(2, 5, n),
                         rng.integers(0, 17, n), rng.uniform(1, 20, n), rng.integers(8, 30, n),
                         rng.uniform(6, 12, n), rng.uniform(4, 10, n)]).astype(float)
    # seconds = 10^(linear law in the features), one law per stage
    law = np.array([[0.02, 0.1, 0.0, 0.03, 0.02, 0.0, 0.1, 0.0],
                    [0.05, 0.2, 0.0, 0.0, 0.1, 0.1, 0.0, 0.0],
                    [0.3, 0.0, 0.0, 0.15, 0.0, 0.0, 0.0, 0.0],
                    [0.3, 0.3, 0.0, 0.0, 0.0, 0.0, 0.0, 0.05]])
    sec = 10.0 ** (X @ law.T - 9.0)
    pl = planner.StagePlanner(n_models=3, seed=1)
    pl.fit(X[:1200], sec[:1200], epochs=3000, lr=2e-3)
    pr = pl.predict(X[1200:])
    for i, s in enumerate(planner.STAGES):
        rel = np.abs(pr[s] - sec[1200:, i]) / sec[1200:, i]
        assert np.median(rel) < 0.15, (s, np.median(rel))
