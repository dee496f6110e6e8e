"""Parity of the row-streamed 3D stencils (FP32 fields, grids periodic in y and z, nx a multiple of 4
and at least 64) with the oracle: the forward fields after the march, the adjoint fields at t = 0
(which pass through every transposed predictor of the sweep), J and dJ/dgamma.

The grids give several 64-column windows with a ragged last one (the window after the grid's end
holds wrapped or boundary columns), several 12-row tiles with a last one aligned to the grid's end,
the fewest rows the form takes (16: both tiles wrap across y = 0), z chunks of unequal length, and
the three x boundary kinds (inflow/outflow, pressure, periodic).

Tolerances: FP32 fields carry about 1e-7 relative rounding per operation; after a few steps of
the coupled march the field errors measured about 1e-7 (forward) and 1e-6 (adjoint), so the bars
are 1e-5 and 1e-4; J and dJ/dgamma keep the FP32 bars of the other parity tests (1e-4, 1e-3).
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from tests.problems import BC_INFLOW_OUTFLOW, BC_PERIODIC, BC_PRESSURE, body3d, perturbed_state
from workloads import CKPT_STORE_ALL, CKPT_UNIFORM

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


CASES_Q = [
    ("inflow-64x20x16", lambda: body3d(nx=64, ny=20, nz=16, centre=(20.3, 9.6, 7.9), nt=3)),
    ("periodic-68x26x18-rotz", lambda: body3d(nx=68, ny=26, nz=18, centre=(40.3, 13.2, 8.8), bc=(BC_PERIODIC,) * 3,
                                              rot_axis=2, nt=3)),
    ("pressure-124x20x14-rotx", lambda: body3d(nx=124, ny=20, nz=14, centre=(60.4, 9.7, 6.6),
                                               bc=(BC_PRESSURE, BC_PERIODIC, BC_PERIODIC), rot_axis=0, nt=3)),
    ("inflow-188x40x21", lambda: body3d(nx=188, ny=40, nz=21, centre=(90.3, 19.6, 10.4), nt=2)),
    # the fewest rows the form takes: both row tiles wrap across y = 0 (one below, one above)
    ("periodic-64x16x16-rotz", lambda: body3d(nx=64, ny=16, nz=16, centre=(30.2, 7.7, 8.1), bc=(BC_PERIODIC,) * 3,
                                              rot_axis=2, nt=3)),
]


def run(P, g, p0, u0, s0, **kw):
    import torch
    from paper_2601_18272_gb300 import lks
    from paper_2601_18272_gb300.lks import Solver
    S = Solver(P, **kw)
    try:
        S.set_initial_state(p0, u0, s0)
        gam = torch.tensor(g, dtype=torch.float64, device="cuda")
        out = {"form": lks.lks_stencil_form(S.handle), "J": S.forward(gam)}
        out["p"], out["u"] = S.state()
        S.adjoint(1.0)
        dg = torch.empty_like(gam)
        S.sensitivity(dg)
        torch.cuda.synchronize()
        out["dJdgamma"] = dg.cpu().numpy()
        out["lam_p0"], out["lam_u0"], _ = S.initial_adjoint()
        return out
    finally:
        S.close()


@pytest.mark.parametrize("name,make", CASES_Q, ids=[c[0] for c in CASES_Q])
def test_row_streamed_3d_matches_oracle(name, make):
    P, g = make()
    p0, u0, s0 = perturbed_state(P)
    G = O.gradient(P, g, p0, u0, s0)
    po, uo, _, Jo = O.forward(P, g, p0, u0, s0)
    r = run(P, g, p0, u0, s0, precision=32, ckpt_policy=CKPT_STORE_ALL)
    assert r["form"] == 1
    assert rel(r["p"], po) < 1e-5 and rel(r["u"], uo) < 1e-5
    assert abs(r["J"] - Jo) <= 1e-4 * abs(Jo)
    assert rel(r["lam_p0"], G["lam_p0"]) < 1e-4 and rel(r["lam_u0"], G["lam_u0"]) < 1e-4
    assert rel(r["dJdgamma"], G["dJdgamma"]) <= 1e-3


def test_row_streamed_3d_checkpointed_matches_store_all():
    """Uniform checkpoints recompute the march with the same kernels: the gradient is the store-all one."""
    P, g = CASES_Q[0][1]()
    P = P.replace(n_steps=5)
    p0, u0, s0 = perturbed_state(P)
    a = run(P, g, p0, u0, s0, precision=32, ckpt_policy=CKPT_STORE_ALL)
    b = run(P, g, p0, u0, s0, precision=32, ckpt_policy=CKPT_UNIFORM, ckpt_every=2)
    assert a["form"] == b["form"] == 1
    np.testing.assert_array_equal(a["dJdgamma"], b["dJdgamma"])
    np.testing.assert_array_equal(a["lam_u0"], b["lam_u0"])


def test_general_form_where_the_row_streamed_one_does_not_apply():
    """FP64 fields, walls in y, or nx not a multiple of 4 keep the general kernels."""
    from paper_2601_18272_gb300 import lks
    from paper_2601_18272_gb300.lks import Solver
    from tests.problems import BC_WALL
    for P, prec in ((body3d(nx=64, ny=20, nz=16, centre=(20.3, 9.6, 7.9))[0], 64),
                    (body3d(nx=64, ny=20, nz=16, centre=(20.3, 9.6, 7.9), bc=(BC_INFLOW_OUTFLOW, BC_WALL, BC_PERIODIC))[0], 32),
                    (body3d(nx=66, ny=20, nz=16, centre=(20.3, 9.6, 7.9))[0], 32)):
        S = Solver(P, precision=prec)
        try:
            assert lks.lks_stencil_form(S.handle) == 0
        finally:
            S.close()


def test_tile_copy_timeout_is_reported_and_recoverable():
    """A tile copy that never arrives (test hook: each CTA withholds one plane's copy) makes the
    bounded waits run out: the forward and the adjoint return LKS_ERR_TIMEOUT, and after the hook is
    cleared the handle gives the same gradient as before, bit for bit."""
    import time
    import torch
    from paper_2601_18272_gb300 import lks
    from paper_2601_18272_gb300.lks import LksError, Solver
    P, g = CASES_Q[0][1]()
    P = P.replace(n_steps=2)
    p0, u0, s0 = perturbed_state(P)
    S = Solver(P, precision=32, ckpt_policy=CKPT_STORE_ALL)
    try:
        assert lks.lks_stencil_form(S.handle) == 1
        S.set_initial_state(p0, u0, s0)
        gam = torch.tensor(g, dtype=torch.float64, device="cuda")

        def grad():
            J = S.forward(gam)
            S.adjoint(1.0)
            d = torch.empty_like(gam)
            S.sensitivity(d)
            torch.cuda.synchronize()
            return J, d.cpu().numpy()

        J0, d0 = grad()
        lks.lks_debug_copy_skip(S.handle, True)
        t0 = time.perf_counter()
        with pytest.raises(LksError, match="LKS_ERR_TIMEOUT"):
            S.forward(gam)
        assert time.perf_counter() - t0 < 30.0
        lks.lks_debug_copy_skip(S.handle, False)
        assert S.forward(gam) == J0
        lks.lks_debug_copy_skip(S.handle, True)
        with pytest.raises(LksError, match="LKS_ERR_TIMEOUT"):
            S.adjoint(1.0)
        lks.lks_debug_copy_skip(S.handle, False)
        J1, d1 = grad()
        assert J1 == J0
        np.testing.assert_array_equal(d1, d0)
    finally:
        S.close()
