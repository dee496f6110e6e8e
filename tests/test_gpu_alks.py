"""Parity of the CUDA path's paper-form adjoint (ALKS, Sec. 2.5; lks_adjoint_alks through the C ABI)
with the oracle's statement of it, on the same seeded inputs.

Tolerances as for the exact adjoint: the FP64 form agrees with the FP64 oracle to rounding
(dJ/dgamma and the moments at t = 0 to 1e-9 relative, the body multipliers to 1e-9); the FP32 form
within dJ/dgamma relative L2 1e-3. The CUDA path sums the coupling terms in a different order (it
reduces them once per step and runs the fixed-point iterations on the sums), which changes only
rounding.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from tests.problems import (BC_INFLOW_OUTFLOW, BC_PERIODIC, BC_PRESSURE, BC_WALL, DOF_ROT, DOF_TX, DOF_TY, DOF_TZ,
                            W_BILINEAR, body2d, body3d, body6, perturbed_state)
from workloads import CKPT_BINOMIAL, CKPT_STORE_ALL, CKPT_UNIFORM, config, initial_state

pytestmark = pytest.mark.gpu


def gpu_alks(P, g, p0=None, u0=None, s0=None, exact_too=False, **overrides):
    import torch
    from paper_2601_18272_gb300.lks import Solver
    S = Solver(P, **overrides)
    try:
        S.set_initial_state(p0, u0, s0)
        gam = torch.tensor(g, dtype=torch.float64, device="cuda")
        out = {"J": S.forward(gam)}
        S.adjoint_alks(1.0)
        dg = torch.empty_like(gam)
        S.sensitivity(dg)
        torch.cuda.synchronize()
        out["dJdgamma"] = dg.cpu().numpy()
        out["p0"], out["u0"], out["s0"], out["body1"] = S.alks_adjoint()
        if exact_too:
            S.adjoint(1.0)
            S.sensitivity(dg)
            torch.cuda.synchronize()
            out["exact"] = dg.cpu().numpy()
        return out
    finally:
        S.close()


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


CASES = [
    ("2d-rot-cos4", lambda: body2d()),
    ("2d-x-bilinear", lambda: body2d(mask=DOF_TX, wk=W_BILINEAR)),
    ("2d-nitr1", lambda: body2d(n_itr=1)),
    ("2d-walls-pressure", lambda: body2d(bc=(BC_PRESSURE, BC_WALL, BC_PERIODIC), mask=DOF_TX | DOF_ROT)),
    ("2d-periodic", lambda: body2d(bc=(BC_PERIODIC,) * 3)),
    ("2d-odd-37x21-walls", lambda: body2d(nx=37, ny=21, centre=(14.3, 10.4), bc=(BC_INFLOW_OUTFLOW, BC_WALL, BC_PERIODIC))),
    ("2d-ragged-40x20", lambda: body2d(nx=40, ny=20, nd=7, centre=(15.6, 9.3), nt=9)),
    ("3d-rot-y", lambda: body3d(nx=24, ny=16, nz=16, centre=(9.3, 7.6, 8.2))),
    ("3d-walls-pressure-rotx", lambda: body3d(nx=40, ny=18, nz=14, centre=(12.4, 8.7, 6.6),
                                              bc=(BC_PRESSURE, BC_WALL, BC_WALL), rot_axis=0)),
    ("3d-periodic-rotz", lambda: body3d(nx=20, ny=16, nz=18, centre=(9.1, 8.4, 8.8), bc=(BC_PERIODIC,) * 3,
                                        rot_axis=2)),
    ("3d-trans-bilinear-walls", lambda: body3d(nx=34, ny=18, nz=13, centre=(10.2, 9.1, 6.4),
                                               mask=DOF_TX | DOF_TY | DOF_TZ, wk=W_BILINEAR,
                                               bc=(BC_INFLOW_OUTFLOW, BC_WALL, BC_WALL))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_alks_fp64_store_all_matches_oracle(name, make):
    P, g = make()
    p0, u0, s0 = perturbed_state(P)
    G = O.gradient_alks(P, g, p0, u0, s0)
    r = gpu_alks(P, g, p0, u0, s0, precision=64, ckpt_policy=CKPT_STORE_ALL)
    assert abs(r["J"] - G["J"]) <= 1e-11 * abs(G["J"])
    assert rel(r["dJdgamma"], G["dJdgamma"]) < 1e-9
    assert rel(r["p0"], G["adj_p0"]) < 1e-9 and rel(r["u0"], G["adj_u0"]) < 1e-9
    assert rel(r["s0"], G["adj_s0"]) < 1e-9
    np.testing.assert_allclose(r["body1"], G["body1"], rtol=1e-9, atol=1e-13)


@pytest.mark.parametrize("policy", ["uniform", "binomial"])
@pytest.mark.parametrize("name,make", [CASES[0], CASES[3], CASES[7]], ids=[CASES[i][0] for i in (0, 3, 7)])
def test_alks_fp32_checkpointed_matches_oracle(name, make, policy):
    P, g = make()
    P = P.replace(n_steps=10)
    p0, u0, s0 = perturbed_state(P)
    G = O.gradient_alks(P, g, p0, u0, s0)
    kw = dict(ckpt_policy=CKPT_UNIFORM, ckpt_every=4) if policy == "uniform" else \
        dict(ckpt_policy=CKPT_BINOMIAL, ckpt_every=2)
    r = gpu_alks(P, g, p0, u0, s0, precision=32, **kw)
    assert abs(r["J"] - G["J"]) <= 1e-4 * abs(G["J"])
    assert rel(r["dJdgamma"], G["dJdgamma"]) <= 1e-3


def test_alks_binomial_reproduces_store_all_fp64():
    P, g = body2d(nt=13)
    p0, u0, s0 = perturbed_state(P)
    a = gpu_alks(P, g, p0, u0, s0, precision=64, ckpt_policy=CKPT_STORE_ALL)
    b = gpu_alks(P, g, p0, u0, s0, precision=64, ckpt_policy=CKPT_BINOMIAL, ckpt_every=3)
    assert rel(b["dJdgamma"], a["dJdgamma"]) < 1e-12
    np.testing.assert_allclose(b["body1"], a["body1"], rtol=1e-12, atol=1e-15)


def test_alks_turbine2d_512x256_truncated_fp32():
    """The 512x256 / 128x128 rotating workload in its benchmark precision (FP32 fields, uniform
    checkpoints), truncated to 20 steps so the oracle finishes in seconds."""
    P, g = config(2)
    P = P.replace(n_steps=20, ckpt_every=10)
    p0, u0, s0 = initial_state(P)
    G = O.gradient_alks(P, g, p0, u0, s0)
    r = gpu_alks(P, g, p0, u0, s0)
    assert abs(r["J"] - G["J"]) <= 1e-4 * abs(G["J"])
    assert rel(r["dJdgamma"], G["dJdgamma"]) <= 1e-3


def test_alks_turbine2d_full_size_approaches_exact_gradient():
    """Full 5000-step rotating workload in the benchmark's configuration: the paper's adjoint and the
    exact adjoint from the same forward. A property that holds at any size: a consistent
    discretisation of the same continuous adjoint stays within a few per cent of the exact gradient."""
    P, g = config(2)
    p0, u0, s0 = initial_state(P)
    r = gpu_alks(P, g, p0, u0, s0, exact_too=True)
    a, b = r["exact"], r["dJdgamma"]
    assert np.all(np.isfinite(b))
    assert rel(b, a) <= 0.1
    assert a @ b >= 0.99 * np.linalg.norm(a) * np.linalg.norm(b)


def test_alks_then_exact_adjoint_on_one_handle():
    """The two reverse sweeps share the forward and the schedulers: running the paper's adjoint first
    leaves the exact adjoint unchanged."""
    P, g = body2d(nt=7)
    p0, u0, s0 = perturbed_state(P)
    G = O.gradient(P, g, p0, u0, s0)
    r = gpu_alks(P, g, p0, u0, s0, exact_too=True, precision=64, ckpt_policy=CKPT_UNIFORM, ckpt_every=3)
    assert rel(r["exact"], G["dJdgamma"]) < 1e-9


def test_alks_free_rotation_is_unsupported():
    import torch
    from paper_2601_18272_gb300.lks import LksError, Solver
    P, g = body6(nt=2, ny=20, nz=20, centre=(8.3, 10.1, 9.7))  # the 18-cell free-rotation box fits
    S = Solver(P, precision=64)
    try:
        S.forward(torch.tensor(g, dtype=torch.float64, device="cuda"))
        with pytest.raises(LksError):
            S.adjoint_alks(1.0)
    finally:
        S.close()


def test_alks_sail2d_80x40_full_fp64():
    """The 80x40 / 16x16 / 400-step translation workload at its full size, FP64, every state stored:
    the paper's adjoint element by element against the oracle's."""
    P, g = config(1)
    p0, u0, s0 = initial_state(P)
    G = O.gradient_alks(P, g, p0, u0, s0)
    r = gpu_alks(P, g, p0, u0, s0)
    assert abs(r["J"] - G["J"]) <= 1e-11 * abs(G["J"])
    assert rel(r["dJdgamma"], G["dJdgamma"]) < 1e-8
    np.testing.assert_allclose(r["body1"], G["body1"], rtol=1e-8, atol=1e-14)
