"""The persistent coupling kernels (one cooperative launch per time step for the N_itr coupling
iterations of Sec. 3.1, and one for their reverse) through the C ABI.

- They run wherever the device holds their grid (2D, 3D single axis, six DOFs) when asked for, and
  by default for 2D bodies whose box has more tiles than the persistent grid has CTAs.
- They agree with the per-iteration kernels to rounding (FP64), and both with the oracle.
- Their grid barriers are bounded: with the test hook that makes the first CTA skip its arrivals, the
  other CTAs' waits run out after one second, the forward or the adjoint returns LKS_ERR_TIMEOUT, and
  the handle stays usable: the next calls give the same results as before, bit for bit.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

from oracle import oracle as O
from tests.problems import body2d, body3d, body6, perturbed_state, perturbed_state6
from workloads import CKPT_STORE_ALL, CKPT_UNIFORM

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _grad(S, g, p0=None, u0=None, s0=None):
    import torch
    S.set_initial_state(p0, u0, s0)
    gam = torch.tensor(g, dtype=torch.float64, device="cuda")
    J = S.forward(gam)
    S.adjoint(1.0)
    d = torch.empty_like(gam)
    S.sensitivity(d)
    torch.cuda.synchronize()
    return J, d.cpu().numpy()


CASES = [
    ("2d", lambda: body2d(nt=5), perturbed_state),
    ("3d-axis", lambda: body3d(nx=24, ny=16, nz=16, centre=(9.3, 7.6, 8.2), nt=4), perturbed_state),
    ("6dof", lambda: body6(ny=20, nz=20, centre=(8.3, 10.1, 9.7), nt=3), perturbed_state6),
]


@pytest.mark.parametrize("name,make,state", CASES, ids=[c[0] for c in CASES])
def test_persistent_matches_per_iteration_kernels_and_oracle(name, make, state):
    from paper_2601_18272_gb300 import lks
    from paper_2601_18272_gb300.lks import Solver
    P, g = make()
    p0, u0, s0 = state(P)
    S = Solver(P, precision=64, ckpt_policy=CKPT_STORE_ALL)
    try:
        assert lks.lks_persistent_coupling(S.handle, 1)
        Jc, dc = _grad(S, g, p0, u0, s0)
        hc = S.dof_history()
        assert not lks.lks_persistent_coupling(S.handle, 0)
        Jk, dk = _grad(S, g, p0, u0, s0)
        hk = S.dof_history()
        assert lks.lks_persistent_coupling(S.handle, 2) is False  # a small box: one launch per iteration
    finally:
        S.close()
    assert abs(Jc - Jk) <= 1e-13 * abs(Jk)
    np.testing.assert_allclose(hc, hk, rtol=1e-13, atol=1e-15)
    assert _rel(dc, dk) < 1e-12
    G = O.gradient(P, g, p0, u0, s0)
    assert abs(Jc - G["J"]) <= 1e-11 * abs(G["J"])
    assert _rel(dc, G["dJdgamma"]) < 1e-9


@pytest.mark.parametrize("precision", [32, 64])
def test_grid_barrier_timeout_is_reported_and_recoverable(precision):
    from paper_2601_18272_gb300 import lks
    from paper_2601_18272_gb300.lks import LksError, Solver
    import torch
    P, g = body2d(nt=4)
    p0, u0, s0 = perturbed_state(P)
    S = Solver(P, precision=precision, ckpt_policy=CKPT_UNIFORM, ckpt_every=2)
    try:
        assert lks.lks_persistent_coupling(S.handle, 1)
        J0, d0 = _grad(S, g, p0, u0, s0)
        gam = torch.tensor(g, dtype=torch.float64, device="cuda")
        # forward: the first barrier never completes; the wait runs out, later launches return at once
        lks.lks_debug_sync_skip(S.handle, True)
        t0 = time.perf_counter()
        with pytest.raises(LksError, match="LKS_ERR_TIMEOUT"):
            S.forward(gam)
        assert time.perf_counter() - t0 < 30.0
        lks.lks_debug_sync_skip(S.handle, False)
        with pytest.raises(LksError, match="LKS_ERR_ORDER"):
            S.adjoint(1.0)
        # adjoint: a completed forward, then a reverse sweep whose barriers time out
        assert S.forward(gam) == J0
        lks.lks_debug_sync_skip(S.handle, True)
        with pytest.raises(LksError, match="LKS_ERR_TIMEOUT"):
            S.adjoint(1.0)
        lks.lks_debug_sync_skip(S.handle, False)
        with pytest.raises(LksError, match="LKS_ERR_ORDER"):
            S.sensitivity(torch.empty_like(gam))
        # the handle and the context stay usable: the same gradient, bit for bit
        J1, d1 = _grad(S, g, p0, u0, s0)
    finally:
        S.close()
    assert J1 == J0
    assert np.array_equal(d1, d0)


def test_automatic_choice_on_a_large_2d_box():
    """The default (automatic) mode takes the persistent kernels for the 1024x512 / 256x256 workload's
    box (576 tiles) and the per-iteration kernels for the 512x256 / 128x128 one (144 tiles)."""
    from paper_2601_18272_gb300 import lks
    from paper_2601_18272_gb300.lks import Solver
    from workloads import config
    for idx, expect in ((3, True), (2, False)):
        P, _ = config(idx)
        S = Solver(P.replace(n_steps=4, ckpt_every=2))
        try:
            assert lks.lks_persistent_coupling(S.handle, -1) is expect, idx
        finally:
            S.close()
