"""Parity of the CUDA path (through the C ABI) with the oracle on the same seeded inputs.

Tolerances: the FP64 form must agree with the FP64 oracle to rounding (J to 1e-11 relative,
gradients to 1e-9); the FP32-field form must meet J relative error <= 1e-4 and dJ/dgamma relative
L2 error <= 1e-3.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from tests.problems import (BC_INFLOW_OUTFLOW, BC_PERIODIC, BC_PRESSURE, BC_WALL, DOF_ROT, DOF_TX, DOF_TY, DOF_TZ,
                            W_BILINEAR, W_COS4, body2d, body3d, perturbed_state)
from workloads import CKPT_BF16, CKPT_BINOMIAL, CKPT_FP16, CKPT_STORE_ALL, CKPT_UNIFORM, config, initial_state

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def gpu_run(P, g, p0=None, u0=None, s0=None, adjoint=True, **overrides):
    torch = _torch()
    from paper_2601_18272_gb300.lks import Solver
    S = Solver(P, **overrides)
    try:
        S.set_initial_state(p0, u0, s0)
        gam = torch.tensor(g, dtype=torch.float64, device="cuda")
        out = {"J": S.forward(gam), "hist": S.dof_history()}
        if S.struct.ckpt_policy == CKPT_STORE_ALL or S.n_steps % max(S.struct.ckpt_every, 1) == 0:
            out["p"], out["u"] = S.state()
        if adjoint:
            S.adjoint(1.0)
            dg = torch.empty_like(gam)
            S.sensitivity(dg)
            torch.cuda.synchronize()
            out["dJdgamma"] = dg.cpu().numpy()
            out["lam_p0"], out["lam_u0"], out["lam_dof0"] = S.initial_adjoint()
        out["launches"] = S.launches()
        return out
    finally:
        S.close()


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


CASES_2D = [
    ("rot-cos4", lambda: body2d()),
    ("x-bilinear", lambda: body2d(mask=DOF_TX, wk=W_BILINEAR)),
    ("rot-nitr1", lambda: body2d(n_itr=1)),
    ("walls-pressure", lambda: body2d(bc=(BC_PRESSURE, BC_WALL, BC_PERIODIC), mask=DOF_TX | DOF_ROT)),
    ("periodic", lambda: body2d(bc=(BC_PERIODIC,) * 3)),
    ("ragged-40x20", lambda: body2d(nx=40, ny=20, nd=7, centre=(15.6, 9.3), nt=9)),
    # odd widths (scalar column path), several column tiles, a tile width reduced so that the last
    # two columns share a tile (nx - 1 = 56)
    ("odd-37x21-walls", lambda: body2d(nx=37, ny=21, centre=(14.3, 10.4), bc=(BC_INFLOW_OUTFLOW, BC_WALL, BC_PERIODIC))),
    ("odd-33x18-periodic", lambda: body2d(nx=33, ny=18, centre=(16.1, 8.7), bc=(BC_PERIODIC,) * 3)),
    ("wide-130x20-pressure", lambda: body2d(nx=130, ny=20, centre=(60.2, 9.6), bc=(BC_PRESSURE, BC_WALL, BC_PERIODIC))),
    ("57x16-tile54", lambda: body2d(nx=57, ny=16, centre=(40.4, 7.7))),
]


@pytest.mark.parametrize("name,make", CASES_2D, ids=[c[0] for c in CASES_2D])
def test_fp64_store_all_matches_oracle(name, make):
    P, g = make()
    p0, u0, s0 = perturbed_state(P)
    G = O.gradient(P, g, p0, u0, s0)
    po, uo, ho, Jo = O.forward(P, g, p0, u0, s0)
    r = gpu_run(P, g, p0, u0, s0, precision=64, ckpt_policy=CKPT_STORE_ALL)
    assert abs(r["J"] - Jo) <= 1e-11 * abs(Jo)
    np.testing.assert_allclose(r["hist"], ho, rtol=1e-11, atol=1e-12)
    assert rel(r["p"], po) < 1e-10 and rel(r["u"], uo) < 1e-10
    assert rel(r["dJdgamma"], G["dJdgamma"]) < 1e-9
    assert rel(r["lam_u0"], G["lam_u0"]) < 1e-9 and rel(r["lam_p0"], G["lam_p0"]) < 1e-9
    np.testing.assert_allclose(r["lam_dof0"], G["lam_dof0"], rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("policy", ["store_all", "uniform"])
@pytest.mark.parametrize("name,make", CASES_2D[:4], ids=[c[0] for c in CASES_2D[:4]])
def test_fp32_matches_oracle(name, make, policy):
    P, g = make()
    P = P.replace(n_steps=10)
    p0, u0, s0 = perturbed_state(P)
    G = O.gradient(P, g, p0, u0, s0)
    kw = dict(precision=32, ckpt_policy=CKPT_STORE_ALL) if policy == "store_all" else \
        dict(precision=32, ckpt_policy=CKPT_UNIFORM, ckpt_every=4)
    r = gpu_run(P, g, p0, u0, s0, **kw)
    assert abs(r["J"] - G["J"]) <= 1e-4 * abs(G["J"])
    assert rel(r["dJdgamma"], G["dJdgamma"]) <= 1e-3


def test_uniform_checkpointing_reproduces_store_all_fp64():
    P, g = body2d(nt=11)
    p0, u0, s0 = perturbed_state(P)
    a = gpu_run(P, g, p0, u0, s0, precision=64, ckpt_policy=CKPT_STORE_ALL)
    b = gpu_run(P, g, p0, u0, s0, precision=64, ckpt_policy=CKPT_UNIFORM, ckpt_every=3)
    assert a["J"] == b["J"]
    assert rel(b["dJdgamma"], a["dJdgamma"]) < 1e-12


def test_deterministic():
    P, g = body2d(nt=8)
    p0, u0, s0 = perturbed_state(P)
    a = gpu_run(P, g, p0, u0, s0, precision=32, ckpt_policy=CKPT_UNIFORM, ckpt_every=3)
    b = gpu_run(P, g, p0, u0, s0, precision=32, ckpt_policy=CKPT_UNIFORM, ckpt_every=3)
    assert a["J"] == b["J"]
    assert np.array_equal(a["dJdgamma"], b["dJdgamma"])


def test_sail2d_80x40_full_fp64():
    """The 80x40 / 16x16 / 400-step translation workload, FP64, every state stored."""
    P, g = config(1)
    p0, u0, s0 = initial_state(P)
    G = O.gradient(P, g, p0, u0, s0)
    r = gpu_run(P, g, p0, u0, s0)
    assert abs(r["J"] - G["J"]) <= 1e-11 * abs(G["J"])
    assert rel(r["dJdgamma"], G["dJdgamma"]) < 1e-8
    assert r["launches"] >= 400 * 4  # per step at least: stencil, coupling, reverse coupling, transposed stencil


def test_turbine2d_512x256_truncated_fp32():
    """The 512x256 / 128x128 rotating workload in its benchmark precision (FP32 fields, uniform
    checkpoints), truncated to 30 steps so the oracle finishes in seconds."""
    P, g = config(2)
    P = P.replace(n_steps=30, ckpt_every=10)
    p0, u0, s0 = initial_state(P)
    G = O.gradient(P, g, p0, u0, s0)
    r = gpu_run(P, g, p0, u0, s0)
    assert abs(r["J"] - G["J"]) <= 1e-4 * abs(G["J"])
    assert rel(r["dJdgamma"], G["dJdgamma"]) <= 1e-3


def test_turbine2d_full_size_fp32_vs_fp64_and_fd():
    """Full 5000-step rotating workload in the benchmark's configuration: the FP32 checkpointed
    gradient against the FP64 store-all gradient (J <= 1e-4, dJ/dgamma rel L2 <= 1e-3), and the
    FP64 adjoint against a central difference of the FP64 forward along a random direction."""
    torch = _torch()
    from paper_2601_18272_gb300.lks import Solver
    P, g = config(2)
    r32 = gpu_run(P, g)
    r64 = gpu_run(P, g, precision=64, ckpt_policy=CKPT_STORE_ALL)
    assert abs(r32["J"] - r64["J"]) <= 1e-4 * abs(r64["J"])
    assert rel(r32["dJdgamma"], r64["dJdgamma"]) <= 1e-3
    v = np.random.default_rng(0).standard_normal(g.shape)
    eps = 1e-4
    S = Solver(P, precision=64, ckpt_policy=CKPT_UNIFORM, ckpt_every=100)
    try:
        Jp = S.forward(torch.tensor(g + eps * v, device="cuda"))
        Jm = S.forward(torch.tensor(g - eps * v, device="cuda"))
    finally:
        S.close()
    fd = (Jp - Jm) / (2 * eps)
    adj = r64["dJdgamma"] @ v
    assert abs(fd - adj) <= 1e-5 * abs(adj)


def test_gradient_host_matches_device_path():
    torch = _torch()
    from paper_2601_18272_gb300.lks import Solver
    P, g = body2d(nt=7)
    S = Solver(P, precision=32, ckpt_policy=CKPT_UNIFORM, ckpt_every=3)
    try:
        J1, d1 = S.gradient_host(g)
        gam = torch.tensor(g, device="cuda")
        J2 = S.forward(gam)
        S.adjoint(1.0)
        d2 = S.sensitivity(torch.empty_like(gam)).cpu().numpy()
    finally:
        S.close()
    assert J1 == J2 and np.array_equal(d1, d2)


def test_autograd_function():
    torch = _torch()
    from paper_2601_18272_gb300.autograd import objective
    from paper_2601_18272_gb300.lks import Solver
    P, g = body2d(nt=6)
    S = Solver(P, precision=64, ckpt_policy=CKPT_STORE_ALL)
    try:
        gam = torch.tensor(g, device="cuda", requires_grad=True)
        J = objective(gam, S)
        (2.5 * J).backward()
        G = O.gradient(P, g, *initial_state(P))
        assert abs(J.item() - G["J"]) < 1e-11 * abs(G["J"])
        assert rel(gam.grad.cpu().numpy(), 2.5 * G["dJdgamma"]) < 1e-9
    finally:
        S.close()


def test_error_paths():
    torch = _torch()
    from paper_2601_18272_gb300.lks import LksError, Solver, lks_create, problem_struct
    P, g = body2d(centre=(4.5, 8.0), nt=3)
    S = Solver(P)
    try:
        with pytest.raises(LksError, match="LKS_ERR_ORDER"):
            S.adjoint(1.0)
        with pytest.raises(LksError, match="BODY_OUTSIDE"):
            S.forward(torch.tensor(g, device="cuda"))
    finally:
        S.close()
    bad = problem_struct(body2d()[0])
    bad.nu = -0.01
    with pytest.raises(LksError, match="UNSTABLE"):
        lks_create(bad)
    bad = problem_struct(body2d()[0])
    bad.nx = 2
    with pytest.raises(LksError, match="LKS_ERR_ARG"):
        lks_create(bad)


# ---- 3D (D3Q15) ------------------------------------------------------------------------------

CASES_3D = [
    ("3d-rot-y", lambda: body3d(nx=24, ny=16, nz=16, centre=(9.3, 7.6, 8.2))),
    ("3d-walls-pressure-rotx", lambda: body3d(nx=40, ny=18, nz=14, centre=(12.4, 8.7, 6.6),
                                              bc=(BC_PRESSURE, BC_WALL, BC_WALL), rot_axis=0)),
    ("3d-periodic-rotz", lambda: body3d(nx=20, ny=16, nz=18, centre=(9.1, 8.4, 8.8), bc=(BC_PERIODIC,) * 3,
                                        rot_axis=2)),
    ("3d-trans-bilinear-walls", lambda: body3d(nx=34, ny=18, nz=13, centre=(10.2, 9.1, 6.4),
                                               mask=DOF_TX | DOF_TY | DOF_TZ, wk=W_BILINEAR,
                                               bc=(BC_INFLOW_OUTFLOW, BC_WALL, BC_WALL))),
    # several 32x16 column tiles (one of them two nodes clear of every boundary) and z chunks
    ("3d-multitile-walls", lambda: body3d(nx=100, ny=40, nz=14, centre=(30.3, 19.6, 6.9),
                                          bc=(BC_INFLOW_OUTFLOW, BC_WALL, BC_WALL), rot_axis=0, nt=4)),
    ("3d-multitile-periodic", lambda: body3d(nx=70, ny=36, nz=22, centre=(40.3, 17.6, 10.9),
                                             bc=(BC_PERIODIC,) * 3, rot_axis=2, nt=4)),
]


@pytest.mark.parametrize("name,make", CASES_3D, ids=[c[0] for c in CASES_3D])
def test_3d_fp64_store_all_matches_oracle(name, make):
    P, g = make()
    p0, u0, s0 = perturbed_state(P)
    G = O.gradient(P, g, p0, u0, s0)
    po, uo, ho, Jo = O.forward(P, g, p0, u0, s0)
    r = gpu_run(P, g, p0, u0, s0, precision=64, ckpt_policy=CKPT_STORE_ALL)
    assert abs(r["J"] - Jo) <= 1e-11 * abs(Jo)
    np.testing.assert_allclose(r["hist"], ho, rtol=1e-11, atol=1e-12)
    assert rel(r["p"], po) < 1e-10 and rel(r["u"], uo) < 1e-10
    assert rel(r["dJdgamma"], G["dJdgamma"]) < 1e-9
    assert rel(r["lam_u0"], G["lam_u0"]) < 1e-9 and rel(r["lam_p0"], G["lam_p0"]) < 1e-9
    np.testing.assert_allclose(r["lam_dof0"], G["lam_dof0"], rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("name,make", CASES_3D[:2], ids=[c[0] for c in CASES_3D[:2]])
def test_3d_fp32_uniform_matches_oracle(name, make):
    P, g = make()
    P = P.replace(n_steps=9)
    p0, u0, s0 = perturbed_state(P)
    G = O.gradient(P, g, p0, u0, s0)
    r = gpu_run(P, g, p0, u0, s0, precision=32, ckpt_policy=CKPT_UNIFORM, ckpt_every=4)
    assert abs(r["J"] - G["J"]) <= 1e-4 * abs(G["J"])
    assert rel(r["dJdgamma"], G["dJdgamma"]) <= 1e-3


def test_sailturbine2d_1024x512_truncated_fp32():
    """The 1024x512 / 256x256 rotating workload in its benchmark precision (FP32 fields, uniform
    checkpoints, and the persistent coupling kernels the automatic choice takes for its 576 box
    tiles), truncated to 8 steps so the oracle finishes in about half a minute."""
    from paper_2601_18272_gb300 import lks
    from paper_2601_18272_gb300.lks import Solver
    P, g = config(3)
    P = P.replace(n_steps=8, ckpt_every=4)
    S = Solver(P)
    try:
        assert lks.lks_persistent_coupling(S.handle, -1) is True
    finally:
        S.close()
    p0, u0, s0 = initial_state(P)
    G = O.gradient(P, g, p0, u0, s0)
    r = gpu_run(P, g, p0, u0, s0)
    assert abs(r["J"] - G["J"]) <= 1e-4 * abs(G["J"])
    assert rel(r["dJdgamma"], G["dJdgamma"]) <= 1e-3


def test_body3d_128x64x64_truncated_fp32():
    """The 128x64x64 D3Q15 / 48^3 translating workload in its benchmark precision (FP32 fields,
    uniform checkpoints), truncated to 2 steps so the oracle finishes in about half a minute."""
    P, g = config(4)
    P = P.replace(n_steps=2, ckpt_every=1)
    p0, u0, s0 = initial_state(P)
    G = O.gradient(P, g, p0, u0, s0)
    r = gpu_run(P, g, p0, u0, s0)
    assert abs(r["J"] - G["J"]) <= 1e-4 * abs(G["J"])
    assert rel(r["dJdgamma"], G["dJdgamma"]) <= 1e-3


# ---- reduced-precision checkpoints -----------------------------------------------------------

# tolerances about ten times the largest error measured on these cases (BF16 1.1e-4, FP16 8.6e-6;
# FP32 checkpoints 4e-7)
@pytest.mark.parametrize("fmt,tol", [(CKPT_BF16, 1.2e-3), (CKPT_FP16, 1e-4)], ids=["bf16", "fp16"])
@pytest.mark.parametrize("name,make", CASES_2D[:2] + CASES_3D[:1], ids=[c[0] for c in CASES_2D[:2] + CASES_3D[:1]])
def test_reduced_precision_checkpoints(name, make, fmt, tol):
    """BF16 / FP16 checkpoints with a per-plane affine range: the forward (and J) is that of the
    FP32 run bit for bit; the gradient carries the quantisation of the restored segment starts."""
    P, g = make()
    P = P.replace(n_steps=12)
    p0, u0, s0 = perturbed_state(P)
    G = O.gradient(P, g, p0, u0, s0)
    r32 = gpu_run(P, g, p0, u0, s0, precision=32, ckpt_policy=CKPT_UNIFORM, ckpt_every=4)
    rq = gpu_run(P, g, p0, u0, s0, precision=32, ckpt_policy=CKPT_UNIFORM, ckpt_every=4, ckpt_format=fmt)
    assert rq["J"] == r32["J"]
    np.testing.assert_array_equal(rq["hist"], r32["hist"])
    e32 = rel(r32["dJdgamma"], G["dJdgamma"])
    eq = rel(rq["dJdgamma"], G["dJdgamma"])
    assert eq <= tol, f"dJ/dgamma rel err {eq:.3e} (FP32 checkpoints: {e32:.3e})"


def test_reduced_precision_first_segment_exact():
    """With a single segment the restore is the exact initial state: the gradient equals the FP32
    checkpointed one bit for bit."""
    P, g = body2d(nt=4)
    p0, u0, s0 = perturbed_state(P)
    a = gpu_run(P, g, p0, u0, s0, precision=32, ckpt_policy=CKPT_UNIFORM, ckpt_every=4)
    b = gpu_run(P, g, p0, u0, s0, precision=32, ckpt_policy=CKPT_UNIFORM, ckpt_every=4, ckpt_format=CKPT_BF16)
    assert np.array_equal(a["dJdgamma"], b["dJdgamma"])


# ---- binomial checkpointing ------------------------------------------------------------------

@pytest.mark.parametrize("nt,snaps", [(11, 1), (11, 2), (23, 3), (40, 5), (7, 9)])
def test_binomial_checkpointing_reproduces_store_all(nt, snaps):
    """Binomial snapshots (the reverse sweep re-advances from the nearest snapshot along the
    optimal recursion): the recomputed states are those of the forward, so the gradient equals the
    store-all gradient (FP64) to rounding."""
    P, g = body2d(nt=nt)
    p0, u0, s0 = perturbed_state(P)
    a = gpu_run(P, g, p0, u0, s0, precision=64, ckpt_policy=CKPT_STORE_ALL)
    b = gpu_run(P, g, p0, u0, s0, precision=64, ckpt_policy=CKPT_BINOMIAL, ckpt_every=snaps)
    assert a["J"] == b["J"]
    np.testing.assert_array_equal(a["hist"], b["hist"])
    assert rel(b["dJdgamma"], a["dJdgamma"]) < 1e-12
    assert rel(b["lam_u0"], a["lam_u0"]) < 1e-12
    np.testing.assert_allclose(b["lam_dof0"], a["lam_dof0"], rtol=1e-12, atol=1e-15)


def test_binomial_fp32_3d_matches_oracle():
    P, g = CASES_3D[0][1]()
    P = P.replace(n_steps=10)
    p0, u0, s0 = perturbed_state(P)
    G = O.gradient(P, g, p0, u0, s0)
    r = gpu_run(P, g, p0, u0, s0, precision=32, ckpt_policy=CKPT_BINOMIAL, ckpt_every=2)
    assert abs(r["J"] - G["J"]) <= 1e-4 * abs(G["J"])
    assert rel(r["dJdgamma"], G["dJdgamma"]) <= 1e-3


# ------------------------------------------------------------------ design chain ----------
CHAIN_CASES = [
    ("filter", dict(filter_radius=1.9)),
    ("projection", dict(proj_beta=4.0, proj_eta=0.45)),
    ("cyclic4-filter-projection", dict(filter_radius=2.2, proj_beta=3.0, proj_eta=0.5, cyclic_order=4)),
    ("cyclic2-odd-grid", dict(cyclic_order=2, filter_radius=1.5)),
]


@pytest.mark.parametrize("name,kw", CHAIN_CASES, ids=[c[0] for c in CHAIN_CASES])
def test_design_chain_gradient_matches_oracle(name, kw):
    """Forward through gamma-bar and dJ/dgamma through the chain's transpose (FP64 fields)."""
    nd = 9 if "odd" in name else 8
    P, g = body2d(nd=nd, nx=30, ny=24, centre=(12.3, 11.8), mask=DOF_TX | DOF_ROT, nt=5)
    P = P.replace(**kw)
    p0, u0, s0 = perturbed_state(P)
    G = O.gradient(P, g, p0, u0, s0)
    r = gpu_run(P, g, p0, u0, s0, precision=64, ckpt_policy=CKPT_STORE_ALL)
    assert abs(r["J"] - G["J"]) <= 1e-11 * abs(G["J"])
    assert rel(r["dJdgamma"], G["dJdgamma"]) < 1e-9


def test_volume_constraint_matches_oracle():
    torch = _torch()
    from paper_2601_18272_gb300.lks import Solver
    P, g = body2d(nd=12, nx=40, ny=32, centre=(16.3, 15.8), bc=(BC_PERIODIC,) * 3)
    P = P.replace(v_min=0.3, filter_radius=2.2, proj_beta=3.0, cyclic_order=4, design_radius=5.0)
    Go, dGo = O.constraint(P, g)
    S = Solver(P, precision=64)
    try:
        gam = torch.tensor(g, dtype=torch.float64, device="cuda")
        dG = torch.empty_like(gam)
        Gg = S.constraint(gam, dG)
        torch.cuda.synchronize()
        assert abs(Gg - Go) <= 1e-13 * max(abs(Go), 1.0)
        np.testing.assert_allclose(dG.cpu().numpy(), dGo, rtol=1e-12, atol=1e-15)
    finally:
        S.close()


# ------------------------------------------------------- periodic warm start (Sec. 3.4) ----
@pytest.mark.parametrize("policy", ["store_all_fp64", "uniform_fp32"])
def test_periodic_warm_start_matches_oracle(policy):
    """A second gradient after lks_warm_start starts from the first forward's final state and
    reverses from the first adjoint's initial adjoint: the oracle's reverse sweep from that terminal
    adjoint on the same initial state."""
    torch = _torch()
    from paper_2601_18272_gb300.lks import Solver
    P, g = body2d(nt=8)
    p0, u0, s0 = perturbed_state(P)
    first = O.gradient(P, g, p0, u0, s0)
    pf, uf, hf, _ = O.forward(P, g, p0, u0, s0)
    second = O.gradient_terminal(P, g, pf, uf, hf[-1], first["lam_p0"], first["lam_u0"], first["lam_dof0"])
    fp64 = policy.endswith("fp64")
    kw = dict(precision=64, ckpt_policy=CKPT_STORE_ALL) if fp64 else \
        dict(precision=32, ckpt_policy=CKPT_UNIFORM, ckpt_every=4)
    S = Solver(P, **kw)
    try:
        S.set_initial_state(p0, u0, s0)
        gam = torch.tensor(g, dtype=torch.float64, device="cuda")
        dg = torch.empty_like(gam)
        S.forward(gam)
        S.adjoint(1.0)
        S.sensitivity(dg)
        S.warm_start(True)
        J2 = S.forward(gam)
        np.testing.assert_allclose(S.dof_history()[0], hf[-1], rtol=1e-11 if fp64 else 1e-5, atol=1e-12)
        S.adjoint(1.0)
        S.sensitivity(dg)
        torch.cuda.synchronize()
        tj, tg = (1e-11, 1e-9) if fp64 else (1e-4, 1e-3)
        assert abs(J2 - second["J"]) <= tj * abs(second["J"])
        assert rel(dg.cpu().numpy(), second["dJdgamma"]) < tg
    finally:
        S.close()
