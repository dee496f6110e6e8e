"""Host logic of the autograd wrapper, with a stand-in solver (no GPU): the backward seeds the
reverse sweep with the incoming gradient and returns the sensitivity in gamma's shape and dtype,
and a backward that comes after a later forward on the same solver raises."""
from __future__ import annotations

import numpy as np
import pytest


class _FakeSolver:
    """Duck-typed Solver: J = sum(w * gamma), dJ/dgamma = w, and the call log."""

    class _P:
        n_design = 6

    def __init__(self):
        import torch
        self.P = self._P()
        self.forward_count = 0
        self.w = torch.arange(1.0, 7.0, dtype=torch.float64)
        self.seed = None
        self.last_gamma = None

    def forward(self, gamma):
        self.forward_count += 1
        self.last_gamma = gamma.clone()
        return float((self.w * gamma.reshape(-1)).sum())

    def adjoint(self, seed):
        self.seed = seed

    def sensitivity(self, out):
        out.copy_(self.seed * self.w)


def test_backward_returns_the_seeded_sensitivity():
    import torch
    from paper_2601_18272_gb300.autograd import objective
    S = _FakeSolver()
    gamma = torch.full((2, 3), 0.5, dtype=torch.float32, requires_grad=True)
    J = objective(gamma, S)
    assert J.item() == pytest.approx(0.5 * 21.0)
    (3.0 * J).backward()
    assert S.seed == 3.0
    assert gamma.grad.dtype == torch.float32 and gamma.grad.shape == (2, 3)
    np.testing.assert_array_equal(gamma.grad.reshape(-1).numpy(), 3.0 * np.arange(1.0, 7.0))


def test_backward_after_a_later_forward_raises():
    import torch
    from paper_2601_18272_gb300.autograd import objective
    S = _FakeSolver()
    g1 = torch.zeros(6, dtype=torch.float64, requires_grad=True)
    g2 = torch.ones(6, dtype=torch.float64, requires_grad=True)
    J1 = objective(g1, S)
    J2 = objective(g2, S)
    with pytest.raises(RuntimeError, match="another forward"):
        J1.backward()
    J2.backward()
    np.testing.assert_array_equal(g2.grad.numpy(), np.arange(1.0, 7.0))
