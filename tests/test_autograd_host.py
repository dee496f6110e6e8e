"""Host logic of the Python layer (no GPU). The autograd wrapper, with a stand-in solver: the
backward seeds the reverse sweep with the incoming gradient and returns the sensitivity in gamma's
shape and dtype, and a backward that comes after a later forward on the same solver raises. The
binding's size checks on host arrays the library reads by the problem's sizes."""
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


def test_initial_state_sizes_are_checked_before_the_library_reads_them():
    from paper_2601_18272_gb300.lks import check_initial_state
    N, dim, ndof = 12, 2, 8
    check_initial_state(N, dim, ndof, np.zeros(N), np.zeros((dim, N)), np.zeros(ndof))
    check_initial_state(N, dim, ndof)  # all defaults
    for bad in (dict(p=np.zeros(N - 1)), dict(u=np.zeros(N)), dict(s=np.zeros(ndof + 1))):
        with pytest.raises(ValueError):
            check_initial_state(N, dim, ndof, **bad)


def test_design_tensors_are_checked_before_the_library_touches_them():
    import torch
    from paper_2601_18272_gb300.lks import check_design_tensor
    with pytest.raises(TypeError):
        check_design_tensor(torch.zeros(6, dtype=torch.float64), 6)  # host memory
    with pytest.raises(TypeError):
        check_design_tensor(np.zeros(6), 6)
