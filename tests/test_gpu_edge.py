"""Edge cases of the CUDA path against the oracle: the shortest march (one step), an all-void and an
all-solid design, a non-square design grid on a ragged analysis grid, a checkpoint interval longer
than the march, the final state of ragged checkpointed marches, the empty march and a non-finite
initial state, which the library rejects, and the order of the calls: what needs the exact adjoint
refuses the paper-form one, and a new initial state voids the last forward."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from tests.problems import BC_INFLOW_OUTFLOW, BC_WALL, body2d, body3d, perturbed_state
from workloads import CKPT_BINOMIAL, CKPT_STORE_ALL, CKPT_UNIFORM, gamma_2d

pytestmark = pytest.mark.gpu


def _run(P, g, p0, u0, s0, paper=False, **kw):
    import torch
    from paper_2601_18272_gb300.lks import Solver
    S = Solver(P, **kw)
    try:
        S.set_initial_state(p0, u0, s0)
        gam = torch.tensor(g, dtype=torch.float64, device="cuda")
        J = S.forward(gam)
        (S.adjoint_alks if paper else S.adjoint)(1.0)
        dg = torch.empty_like(gam)
        S.sensitivity(dg)
        torch.cuda.synchronize()
        return J, dg.cpu().numpy(), S.dof_history()
    finally:
        S.close()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("make", [lambda: body2d(nt=1), lambda: body3d(nx=24, ny=16, nz=16, centre=(9.3, 7.6, 8.2), nt=1)],
                         ids=["2d", "3d"])
def test_single_step(make):
    """N_t = 1: the forward is one predictor and N_itr coupling iterations; both reverse sweeps
    are one step."""
    P, g = make()
    p0, u0, s0 = perturbed_state(P)
    G = O.gradient(P, g, p0, u0, s0)
    Ga = O.gradient_alks(P, g, p0, u0, s0)
    J, dg, hist = _run(P, g, p0, u0, s0, precision=64, ckpt_policy=CKPT_STORE_ALL)
    assert hist.shape[0] == 2
    assert abs(J - G["J"]) <= 1e-11 * abs(G["J"])
    assert _rel(dg, G["dJdgamma"]) < 1e-9
    _, dga, _ = _run(P, g, p0, u0, s0, paper=True, precision=64, ckpt_policy=CKPT_STORE_ALL)
    assert _rel(dga, Ga["dJdgamma"]) < 1e-9


@pytest.mark.parametrize("fill", [0.0, 1.0], ids=["void", "solid"])
def test_uniform_design(fill):
    """gamma = 0 everywhere (kappa^ref = 0: the body feels no fluid, yet dkappa^ref/dgamma is
    finite) and gamma = 1 everywhere (kappa^ref = kappa_max)."""
    P, g = body2d(nt=6)
    g = np.full_like(g, fill)
    p0, u0, s0 = perturbed_state(P)
    G = O.gradient(P, g, p0, u0, s0)
    J, dg, _ = _run(P, g, p0, u0, s0, precision=64, ckpt_policy=CKPT_STORE_ALL)
    assert abs(J - G["J"]) <= 1e-11 * max(abs(G["J"]), 1e-12)
    assert np.linalg.norm(G["dJdgamma"]) > 0
    assert _rel(dg, G["dJdgamma"]) < 1e-9


def test_non_square_design_on_ragged_grid():
    """A 7 x 5 design grid (pivot at (3, 2)) on a 37 x 21 grid with walls: odd extents everywhere."""
    P, _ = body2d(nx=37, ny=21, centre=(14.3, 10.4), bc=(BC_INFLOW_OUTFLOW, BC_WALL, BC_WALL), nt=6)
    P = P.replace(ndx=7, ndy=5)
    g = gamma_2d(7, 11)[:35]
    p0, u0, s0 = perturbed_state(P)
    G = O.gradient(P, g, p0, u0, s0)
    J, dg, _ = _run(P, g, p0, u0, s0, precision=64, ckpt_policy=CKPT_STORE_ALL)
    assert abs(J - G["J"]) <= 1e-11 * abs(G["J"])
    assert _rel(dg, G["dJdgamma"]) < 1e-9
    Ga = O.gradient_alks(P, g, p0, u0, s0)
    _, dga, _ = _run(P, g, p0, u0, s0, paper=True, precision=64, ckpt_policy=CKPT_STORE_ALL)
    assert _rel(dga, Ga["dJdgamma"]) < 1e-9


def test_checkpoint_interval_longer_than_march():
    """Uniform checkpoints every 50 steps on a 7-step march: one segment, the same gradient."""
    P, g = body2d(nt=7)
    p0, u0, s0 = perturbed_state(P)
    a = _run(P, g, p0, u0, s0, precision=64, ckpt_policy=CKPT_STORE_ALL)
    b = _run(P, g, p0, u0, s0, precision=64, ckpt_policy=CKPT_UNIFORM, ckpt_every=50)
    assert a[0] == b[0]
    assert _rel(b[1], a[1]) < 1e-12


def test_empty_march_is_rejected():
    from paper_2601_18272_gb300.lks import LksError, lks_create, problem_struct
    bad = problem_struct(body2d()[0])
    bad.n_steps = 0
    with pytest.raises(LksError, match="LKS_ERR_ARG"):
        lks_create(bad)


def test_call_order_rules():
    """lks_get_initial_adjoint and lks_warm_start(with_adjoint) need an exact adjoint of the last
    forward (the paper-form adjoint has no lambda(0) of the state); a new initial state voids the last
    forward, since the reverse sweep restarts from the initial state."""
    import torch
    from paper_2601_18272_gb300.lks import LksError, Solver
    P, g = body2d(nt=3)
    p0, u0, s0 = perturbed_state(P)
    S = Solver(P, precision=64, ckpt_policy=CKPT_UNIFORM, ckpt_every=2)
    try:
        gam = torch.tensor(g, dtype=torch.float64, device="cuda")
        S.set_initial_state(p0, u0, s0)
        S.forward(gam)
        S.adjoint_alks(1.0)
        with pytest.raises(LksError, match="LKS_ERR_ORDER"):
            S.initial_adjoint()
        with pytest.raises(LksError, match="LKS_ERR_ORDER"):
            S.warm_start(True)
        S.adjoint(1.0)
        lp = S.initial_adjoint()[0]
        S.adjoint_alks(1.0)  # leaves the exact adjoint's lambda(0) in place
        assert np.array_equal(S.initial_adjoint()[0], lp)
        S.alks_adjoint()
        S.set_initial_state(p0, u0, s0)
        for call in (lambda: S.adjoint(1.0), S.initial_adjoint, S.alks_adjoint, S.state):
            with pytest.raises(LksError, match="LKS_ERR_ORDER"):
                call()
        S.forward(gam)
        S.adjoint(1.0)
        assert np.array_equal(S.initial_adjoint()[0], lp)
    finally:
        S.close()


@pytest.mark.parametrize("policy", [dict(ckpt_policy=CKPT_UNIFORM, ckpt_every=3), dict(ckpt_policy=CKPT_BINOMIAL, ckpt_every=2)],
                         ids=["uniform", "binomial"])
def test_final_state_of_a_ragged_checkpointed_march(policy):
    """7 steps with checkpoints every 3 (a short last segment) or 2 binomial snapshots: the final
    state read back equals the store-all forward's, bit for bit (the same kernels in the same order)."""
    import torch
    from paper_2601_18272_gb300.lks import Solver
    P, g = body2d(nt=7)
    p0, u0, s0 = perturbed_state(P)
    out = []
    for kw in (dict(ckpt_policy=CKPT_STORE_ALL), policy):
        S = Solver(P, precision=64, **kw)
        try:
            S.set_initial_state(p0, u0, s0)
            S.forward(torch.tensor(g, dtype=torch.float64, device="cuda"))
            out.append(S.state())
        finally:
            S.close()
    np.testing.assert_array_equal(out[1][0], out[0][0])
    np.testing.assert_array_equal(out[1][1], out[0][1])


def test_nonfinite_initial_state_is_refused():
    """A NaN or an infinity in a host-built initial state is refused on the host before any device
    work (LKS_ERR_NONFINITE); the last forward and the handle stay usable."""
    import torch
    from paper_2601_18272_gb300.lks import LksError, Solver
    P, g = body2d(nt=2)
    p0, u0, s0 = perturbed_state(P)
    S = Solver(P, precision=64, ckpt_policy=CKPT_STORE_ALL)
    try:
        gam = torch.tensor(g, dtype=torch.float64, device="cuda")
        S.set_initial_state(p0, u0, s0)
        J = S.forward(gam)
        state = S.state()
        for name, src, bad in (("p", p0, np.nan), ("u", u0, np.inf), ("s", s0, -np.inf)):
            arr = np.array(src, dtype=np.float64)
            arr.flat[3] = bad
            with pytest.raises(LksError, match="LKS_ERR_NONFINITE"):
                S.set_initial_state(**{name: arr})
        np.testing.assert_array_equal(S.state()[0], state[0])
        S.set_initial_state(p0, u0, s0)
        assert S.forward(gam) == J
    finally:
        S.close()


@pytest.mark.parametrize("precision", [32, 64])
def test_nonfinite_design_is_found_on_the_device(precision):
    """A NaN or an infinity in the device design field is found by the kernel that forms kappa^ref:
    it reports through the device status word (LKS_ERR_NONFINITE) and the march runs with that point
    void, so nothing non-finite enters it; the handle stays usable and a finite design gives the
    same J as before."""
    import torch
    from paper_2601_18272_gb300.lks import LksError, Solver
    P, g = body2d(nt=3)
    p0, u0, s0 = perturbed_state(P)
    S = Solver(P, precision=precision, ckpt_policy=CKPT_STORE_ALL)
    try:
        S.set_initial_state(p0, u0, s0)
        gam = torch.tensor(g, dtype=torch.float64, device="cuda")
        J = S.forward(gam)
        for bad in (np.nan, np.inf):
            gb = gam.clone()
            gb[7] = bad
            with pytest.raises(LksError, match="LKS_ERR_NONFINITE"):
                S.forward(gb)
            with pytest.raises(LksError, match="LKS_ERR_ORDER"):
                S.adjoint(1.0)  # a failed forward leaves nothing to reverse
        assert S.forward(gam) == J
    finally:
        S.close()


def test_workspace_budget():
    """hbm_budget_bytes bounds the workspace: a budget below what the problem needs is refused at
    creation (LKS_ERR_BUDGET) before any allocation is kept; one at the exact need is accepted."""
    from paper_2601_18272_gb300 import lks
    from paper_2601_18272_gb300.lks import LksError, Solver
    P, _ = body2d(nt=20)
    S = Solver(P, precision=32, ckpt_policy=CKPT_UNIFORM, ckpt_every=5)
    need = lks.lks_workspace_bytes(S.handle)
    S.close()
    for budget in (1 << 10, need - 256):
        with pytest.raises(LksError, match="LKS_ERR_BUDGET"):
            Solver(P, precision=32, ckpt_policy=CKPT_UNIFORM, ckpt_every=5, hbm_budget_bytes=budget)
    S = Solver(P, precision=32, ckpt_policy=CKPT_UNIFORM, ckpt_every=5, hbm_budget_bytes=need)
    assert lks.lks_workspace_bytes(S.handle) == need
    S.close()
