"""The outer loop's optimiser (MMA) on problems with known optima (no GPU), and one short run of
Algorithm 1 on the GPU."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2601_18272_gb300.optimize import MMA


def _run(mma, x, f, iters):
    for _ in range(iters):
        f0, df0, f1, df1 = f(x)
        x, lam = mma.step(x, f0, df0, f1, df1)
    return x, lam


def test_mma_reciprocal_objective_with_a_budget():
    """min sum c_j / x_j s.t. sum x_j <= b: the KKT point is x_j = b sqrt(c_j) / sum_k sqrt(c_k)
    (stationarity -c_j / x_j^2 + lambda = 0, the budget active)."""
    rng = np.random.default_rng(1)
    n, b = 12, 3.0
    c = rng.uniform(0.5, 2.0, n)
    xs = b * np.sqrt(c) / np.sum(np.sqrt(c))

    def f(x):
        return np.sum(c / x), -c / x ** 2, np.sum(x) - b, np.ones(n)

    x, _ = _run(MMA(n, xmin=0.01, xmax=2.0), np.full(n, 0.2), f, 60)
    np.testing.assert_allclose(x, xs, rtol=1e-6)


def test_mma_box_constrained_quadratic():
    """min sum (x_j - a_j)^2 s.t. sum x_j <= b on [0, 1]: x_j = clip(a_j - mu, 0, 1) with mu >= 0 set
    so that the budget holds (found here by bisection)."""
    rng = np.random.default_rng(2)
    n = 20
    a = rng.uniform(-0.3, 1.3, n)
    b = 0.4 * n * 0.5
    lo, hi = 0.0, 3.0
    for _ in range(200):
        mu = 0.5 * (lo + hi)
        lo, hi = (mu, hi) if np.clip(a - mu, 0, 1).sum() > b else (lo, mu)
    xs = np.clip(a - 0.5 * (lo + hi), 0, 1)

    def f(x):
        return np.sum((x - a) ** 2), 2 * (x - a), np.sum(x) - b, np.ones(n)

    x, _ = _run(MMA(n), np.full(n, 0.5), f, 200)
    np.testing.assert_allclose(x, xs, atol=1e-4)
    assert np.sum(x) <= b + 1e-6


def test_mma_recovers_from_an_infeasible_start():
    """A minimum-volume constraint (-sum x + b <= 0) violated at the start is met after a few
    iterations, while the objective pulls the other way."""
    n, b = 10, 6.0

    def f(x):
        return np.sum(x ** 2), 2 * x, b - np.sum(x), -np.ones(n)

    x, _ = _run(MMA(n), np.full(n, 0.1), f, 40)
    assert np.sum(x) >= b - 1e-6
    np.testing.assert_allclose(x, b / n, rtol=1e-5)


def test_mma_keeps_variables_without_gradient():
    """Design variables with zero derivative (points outside the design domain, or images of the
    cyclic expansion) stay where they are."""
    n = 8

    def f(x):
        d0 = np.zeros(n)
        d0[:4] = 2 * (x[:4] - 0.9)
        d1 = np.zeros(n)
        d1[:4] = 1.0
        return np.sum((x[:4] - 0.9) ** 2), d0, np.sum(x[:4]) - 2.0, d1

    x0 = np.linspace(0.1, 0.8, n)
    x, _ = _run(MMA(n), x0, f, 50)
    np.testing.assert_allclose(x[4:], x0[4:], rtol=0, atol=1e-12)
    np.testing.assert_allclose(x[:4], 0.5, atol=1e-5)


@pytest.mark.gpu
def test_algorithm1_improves_the_rotation_angle():
    """Algorithm 1 on a small rotating body: two continuation steps of a few MMA iterations raise the
    rotation angle J_2, keep the minimum-volume constraint at the end, and pass q and beta to the
    library."""
    from paper_2601_18272_gb300.lks import Solver
    from paper_2601_18272_gb300.optimize import optimize
    from tests.problems import DOF_ROT, body2d
    P, g = body2d(nt=40, mask=DOF_ROT, obj=(0, 0, 0, 0, 0, 0, 1, 0), nx=40, ny=24, nd=8, centre=(14.3, 12.1))
    P = P.replace(filter_radius=1.5, proj_eta=0.5, v_min=0.4)
    S = Solver(P, precision=64)
    try:
        r = optimize(S, g, q_steps=(0.1, 0.05), beta_steps=(1.0, 2.0), n_opt=6, move=0.1)
    finally:
        S.close()
    h = r.history
    assert {rec.step for rec in h} == {0, 1}
    first = [rec for rec in h if rec.step == 0]
    assert first[-1].J > first[0].J
    assert h[-1].feasible
    assert np.all((r.gamma >= 0) & (r.gamma <= 1))


@pytest.mark.gpu
def test_algorithm1_with_periodic_warm_start():
    """Algorithm 1 with the periodic warm start (Sec. 3.4) on a periodic channel: each gradient
    starts from the previous forward's final state and reverse sweep's initial adjoint; the loop
    runs, keeps gamma in [0, 1] and raises the angle turned over its first iterations."""
    from paper_2601_18272_gb300.lks import Solver
    from paper_2601_18272_gb300.optimize import optimize
    from tests.problems import BC_PERIODIC, DOF_ROT, body2d
    P, g = body2d(nt=30, mask=DOF_ROT, obj=(0, 0, 0, 0, 0, 0, 1, 0), nx=40, ny=24, nd=8, centre=(14.3, 12.1),
                  bc=(BC_PERIODIC,) * 3)
    P = P.replace(filter_radius=1.5, v_min=0.4)
    S = Solver(P, precision=64)
    try:
        r = optimize(S, g, q_steps=(0.1,), beta_steps=(0.0,), n_opt=5, move=0.1, warm_start=True)
    finally:
        S.close()
    J = [rec.J for rec in r.history]
    assert len(J) >= 3 and np.all(np.isfinite(J))
    assert max(J[1:]) > J[0]
    assert np.all((r.gamma >= 0) & (r.gamma <= 1))
