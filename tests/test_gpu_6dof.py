"""Parity of the CUDA path with the oracle for freely rotating 3D bodies (six DOFs) and
ball-shaped design domains, through the C ABI.

Tolerances as for the single-axis parity tests: FP64 to rounding (J 1e-11 relative, histories
1e-11, gradients 1e-9), FP32 fields J <= 1e-4 relative and dJ/dgamma relative L2 <= 1e-3.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from tests.problems import (BC_PERIODIC, BC_PRESSURE, BC_WALL, DOF_ROT, DOF_TX, DOF_TZ, W_BILINEAR, body6,
                            perturbed_state6)
from tests.test_gpu_parity import gpu_run, rel
from workloads import CKPT_BINOMIAL, CKPT_FP32, CKPT_STORE_ALL, CKPT_UNIFORM, config, initial_state

pytestmark = pytest.mark.gpu


def b6(**kw):
    """body6 on a 20x20x20 grid: a freely rotating 6^3 design needs an 18-cell body box, which
    must fit the periodic y and z extents."""
    kw.setdefault("ny", 20)
    kw.setdefault("nz", 20)
    kw.setdefault("centre", (8.3, 10.1, 9.7))
    return body6(**kw)


CASES = [
    ("free", lambda: b6()),
    ("free-ball-domain", lambda: body6(nd=7, radius=2.6)),
    ("free-bilinear", lambda: body6(wk=W_BILINEAR)),
    ("free-walls-pressure", lambda: body6(bc=(BC_PRESSURE, BC_WALL, BC_WALL), centre=(9.2, 7.8, 8.1))),
    ("free-nitr1", lambda: b6(n_itr=1, nt=3)),
    ("free-rotation-masked", lambda: b6(mask=DOF_TX | DOF_TZ)),
    ("free-rotation-only", lambda: b6(mask=DOF_ROT)),
    ("free-periodic-larger", lambda: body6(nx=36, ny=24, nz=20, nd=9, centre=(14.6, 11.3, 9.8),
                                           bc=(BC_PERIODIC,) * 3, radius=3.9, nt=6)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_free_fp64_store_all_matches_oracle(name, make):
    P, g = make()
    p0, u0, s0 = perturbed_state6(P)
    G = O.gradient(P, g, p0, u0, s0)
    po, uo, ho, Jo = O.forward(P, g, p0, u0, s0)
    r = gpu_run(P, g, p0, u0, s0, precision=64, ckpt_policy=CKPT_STORE_ALL)
    assert r["hist"].shape == ho.shape == (P.n_steps + 1, 21)
    assert abs(r["J"] - Jo) <= 1e-11 * abs(Jo)
    np.testing.assert_allclose(r["hist"], ho, rtol=1e-11, atol=1e-12)
    assert rel(r["p"], po) < 1e-10 and rel(r["u"], uo) < 1e-10
    assert rel(r["dJdgamma"], G["dJdgamma"]) < 1e-9
    assert rel(r["lam_u0"], G["lam_u0"]) < 1e-9 and rel(r["lam_p0"], G["lam_p0"]) < 1e-9
    np.testing.assert_allclose(r["lam_dof0"], G["lam_dof0"], rtol=1e-9, atol=1e-10 * np.abs(G["lam_dof0"]).max())
    if P.design_radius > 0:  # points outside the design domain: exactly zero sensitivity
        assert np.all(r["dJdgamma"][G["dJdgamma"] == 0.0] == 0.0)


@pytest.mark.parametrize("policy", ["store_all", "uniform"])
@pytest.mark.parametrize("name,make", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_free_fp32_matches_oracle(name, make, policy):
    P, g = make()
    P = P.replace(n_steps=8)
    p0, u0, s0 = perturbed_state6(P)
    G = O.gradient(P, g, p0, u0, s0)
    kw = dict(precision=32, ckpt_policy=CKPT_STORE_ALL) if policy == "store_all" else \
        dict(precision=32, ckpt_policy=CKPT_UNIFORM, ckpt_every=3)
    r = gpu_run(P, g, p0, u0, s0, **kw)
    assert abs(r["J"] - G["J"]) <= 1e-4 * abs(G["J"])
    assert rel(r["dJdgamma"], G["dJdgamma"]) <= 1e-3


def test_free_binomial_reproduces_store_all():
    P, g = b6(nt=9)
    p0, u0, s0 = perturbed_state6(P)
    a = gpu_run(P, g, p0, u0, s0, precision=64, ckpt_policy=CKPT_STORE_ALL)
    b = gpu_run(P, g, p0, u0, s0, precision=64, ckpt_policy=CKPT_BINOMIAL, ckpt_every=2)
    assert a["J"] == b["J"]
    assert rel(b["dJdgamma"], a["dJdgamma"]) < 1e-12
    np.testing.assert_allclose(b["lam_dof0"], a["lam_dof0"], rtol=1e-12, atol=1e-14)


def test_free_default_state_starts_unrotated():
    """The library's default initial state with free rotation: body at rest at body_centre, R = I."""
    P, g = b6(nt=2)
    r = gpu_run(P, g, adjoint=False, precision=64, ckpt_policy=CKPT_STORE_ALL)
    p0, u0, s0 = initial_state(P)
    np.testing.assert_array_equal(r["hist"][0], s0)
    _, _, ho, _ = O.forward(P, g, p0, u0, s0)
    np.testing.assert_allclose(r["hist"], ho, rtol=1e-11, atol=1e-12)


def test_turbine3d_6dof_truncated_fp32():
    """The 256x128x128 D3Q15 / 96^3 sphere-masked six-DOF workload (design domain radius 46) in the
    launch configuration the benchmark times, FP32 fields, two steps against the oracle."""
    P, g = config(5)
    P = P.replace(n_steps=2)
    p0, u0, s0 = initial_state(P)
    po, uo, ho, Jo = O.forward(P, g, p0, u0, s0)
    r = gpu_run(P, g, p0, u0, s0, adjoint=False, precision=32, ckpt_policy=CKPT_STORE_ALL, ckpt_format=CKPT_FP32)
    # x^G to the FP32 field accuracy; u^G, h, omega relative to their scale; R within 1e-9
    np.testing.assert_allclose(r["hist"][:, 0:3], ho[:, 0:3], rtol=1e-9)
    for cols in (slice(3, 6), slice(6, 9), slice(9, 12)):
        scale = np.abs(ho[:, cols]).max()
        assert np.abs(r["hist"][:, cols] - ho[:, cols]).max() <= 1e-4 * scale, cols
    assert np.abs(r["hist"][:, 12:21] - ho[:, 12:21]).max() < 1e-9
    assert rel(r["u"], uo) < 1e-5 and rel(r["p"], po) < 1e-4


def test_turbine3d_6dof_adjoint_from_rotated_state():
    """The 256x128x128 / 96^3 six-DOF workload's gradient against the oracle's over two steps, from
    a rotated, spinning and drifting body (perturbed_state6), in the benchmark's field precision
    with FP32 and with BF16 checkpoints at every step (the second segment restarts from a
    quantised state): J relative error <= 1e-4, dJ/dgamma relative L2 <= 1e-3."""
    from workloads import CKPT_BF16
    P, g = config(5)
    P = P.replace(n_steps=2)
    p0, u0, s0 = perturbed_state6(P)
    G = O.gradient(P, g, p0, u0, s0)
    for fmt in (CKPT_FP32, CKPT_BF16):
        r = gpu_run(P, g, p0, u0, s0, precision=32, ckpt_policy=CKPT_UNIFORM, ckpt_every=1, ckpt_format=fmt)
        assert abs(r["J"] - G["J"]) <= 1e-4 * abs(G["J"]), fmt
        assert rel(r["dJdgamma"], G["dJdgamma"]) <= 1e-3, fmt


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
def test_free_binomial_reduced_snapshots(fmt):
    """Binomial checkpointing with BF16 / FP16 snapshots (the six-DOF workload's memory policy): the
    forward is the FP32 run's bit for bit (snapshots are copies on the side); the gradient carries the
    quantisation of the restored and re-stored states and stays within the reduced-precision tolerance
    of the uniform policy (1.2e-3 BF16, 1e-4 FP16) of the oracle's."""
    from workloads import CKPT_BF16, CKPT_FP16
    P, g = b6(nt=9)
    p0, u0, s0 = perturbed_state6(P)
    G = O.gradient(P, g, p0, u0, s0)
    code, tol = (CKPT_BF16, 1.2e-3) if fmt == "bf16" else (CKPT_FP16, 1e-4)
    r32 = gpu_run(P, g, p0, u0, s0, precision=32, ckpt_policy=CKPT_BINOMIAL, ckpt_every=2)
    rq = gpu_run(P, g, p0, u0, s0, precision=32, ckpt_policy=CKPT_BINOMIAL, ckpt_every=2, ckpt_format=code)
    assert rq["J"] == r32["J"]
    np.testing.assert_array_equal(rq["hist"], r32["hist"])
    assert rel(r32["dJdgamma"], G["dJdgamma"]) <= 1e-3
    assert rel(rq["dJdgamma"], G["dJdgamma"]) <= tol


def test_binomial_snapshots_sized_by_the_budget():
    """ckpt_every = 0 with a budget: the binomial schedule gets as many BF16 snapshots as the budget
    holds after the rest of the workspace; the workspace stays within the budget and the gradient is
    that of an explicit handle with the same snapshot count, bit for bit."""
    import torch
    from paper_2601_18272_gb300 import lks
    from paper_2601_18272_gb300.lks import Solver
    from workloads import CKPT_BF16
    P, g = b6(nt=12)
    gam = torch.tensor(g, dtype=torch.float64, device="cuda")
    S3 = Solver(P, precision=32, ckpt_policy=CKPT_BINOMIAL, ckpt_every=3, ckpt_format=CKPT_BF16)
    budget = lks.lks_workspace_bytes(S3.handle)
    S3.close()
    Sa = Solver(P, precision=32, ckpt_policy=CKPT_BINOMIAL, ckpt_every=0, ckpt_format=CKPT_BF16,
                hbm_budget_bytes=budget)
    n = lks.lks_checkpoint_slots(Sa.handle)
    assert 2 <= n <= 3
    assert lks.lks_workspace_bytes(Sa.handle) <= budget
    Sn = Solver(P, precision=32, ckpt_policy=CKPT_BINOMIAL, ckpt_every=n, ckpt_format=CKPT_BF16)
    out = []
    for S in (Sa, Sn):
        try:
            J = S.forward(gam)
            S.adjoint(1.0)
            d = torch.empty_like(gam)
            S.sensitivity(d)
            torch.cuda.synchronize()
            out.append((J, d.cpu().numpy()))
        finally:
            S.close()
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1])
