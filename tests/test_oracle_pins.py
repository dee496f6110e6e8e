"""Pins for the oracle against what the paper and the mathematics fix (no GPU).

Each test names the passage it follows. The paper prints no state, objective or sensitivity value
(all results are figures), so the pins are the printed lattice weights, closed-form solutions,
conservation laws, exact fixed points, and derivative identities (complex step, central
differences, dot-product tests) chosen so that a dropped term, a wrong sign or index, or a
transposed operand fails at least one of them.
"""
from __future__ import annotations

import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from tests.problems import (BC_INFLOW_OUTFLOW, BC_PERIODIC, BC_PRESSURE, BC_WALL, DOF_ROT, DOF_TX, DOF_TY, DOF_TZ,
                            W_BILINEAR, W_COS4, body2d, body3d, box, perturbed_state)
from workloads import Problem, initial_state

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _centre(P):
    s = np.zeros(8)
    s[:3] = P.body_centre
    return s


# ---------------------------------------------------------------- lattice (Sec. 2.2) ------
def test_lattice_weights_match_paper():
    """The weights the paper prints for D2Q9 and D3Q15 (Sec. 2.2)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "lattice_weights.txt")) if l.strip() and l[0] != "#"]
    for model, rng, frac in rows:
        dim = 2 if model == "D2Q9" else 3
        c, w = O.lattice(dim)
        lo, hi = (int(rng), int(rng)) if "-" not in rng else map(int, rng.split("-"))
        for i in range(lo, hi + 1):
            assert w[i] == float(Fraction(frac)), (model, i)
        assert len(w) == (9 if dim == 2 else 15)


@pytest.mark.parametrize("dim", [2, 3])
def test_lattice_moments_isotropic(dim):
    """Moments that give p* = p, u* = u and nu = 1/6 - 2A/9 (Sec. 2.2): sum w = 1, sum w c = 0,
    sum w c_a c_b = delta/3, 4th moment = (dd + dd + dd)/9. A velocity order inconsistent with the
    printed weight ranges breaks these."""
    c, w = O.lattice(dim)
    c = c[:, :dim].astype(float)
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(w @ c).max() < 1e-15
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(dim) / 3, atol=1e-15)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(dim)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9
    np.testing.assert_allclose(m4, iso, atol=1e-15)
    assert len({tuple(v) for v in c}) == len(c)


# ------------------------------------------------------------ weight kernel (Sec. 2.3) ------
def test_weight_kernel_values():
    """w(r) = (1 + cos(pi r/2))/4 on |r| < 2 (the paper's '1 - cos' read as '1 + cos'), bilinear 1 - |r|."""
    assert O.weight(W_COS4, 0.0)[0] == 0.5
    assert abs(O.weight(W_COS4, 1.0)[0] - 0.25) < 1e-16
    assert abs(O.weight(W_COS4, -1.0)[0] - 0.25) < 1e-16
    assert O.weight(W_COS4, 2.0)[0] == 0.0 and O.weight(W_COS4, 2.5)[0] == 0.0
    assert O.weight(W_BILINEAR, 0.25)[0] == 0.75 and O.weight(W_BILINEAR, -0.25)[0] == 0.75
    assert O.weight(W_BILINEAR, 1.0)[0] == 0.0
    for kind in (W_COS4, W_BILINEAR):
        for r in np.linspace(-2.3, 2.3, 47):
            if abs(abs(r) - 1) < 1e-9 or abs(r) < 1e-9:
                continue
            h = 1e-7
            fd = (O.weight(kind, r + h)[0] - O.weight(kind, r - h)[0]) / (2 * h)
            assert abs(fd - O.weight(kind, r)[1]) < 1e-6, (kind, r)


@pytest.mark.parametrize("kind", [W_COS4, W_BILINEAR])
def test_weight_kernel_partition_of_unity(kind):
    """sum_n w(n - X) = 1 over the integers for any X, so the interpolation of a uniform field is exact."""
    for X in np.random.default_rng(3).uniform(-5, 5, 25):
        n = np.arange(np.floor(X) - 3, np.floor(X) + 4)
        assert abs(sum(O.weight(kind, v - X)[0] for v in n) - 1.0) < 1e-14


# --------------------------------------------------------------- fluid closed forms ---------
def test_quiescent_fluid_stays_exactly_at_rest():
    """p = 0, u = 0 is an exact fixed point of the LKS step, also with a resting body in the flow."""
    P, g = body2d(bc=(BC_PERIODIC,) * 3, mask=0, nt=20)
    N = P.n_cells
    p, u, hist, _ = O.forward(P, g, np.zeros(N), np.zeros((2, N)), _centre(P))
    assert not p.any() and not u.any()
    P3, g3 = body3d(bc=(BC_PERIODIC,) * 3, mask=0, nt=5)
    p, u, _, _ = O.forward(P3, g3, np.zeros(P3.n_cells), np.zeros((3, P3.n_cells)), _centre(P3))
    assert not p.any() and not u.any()


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_state_is_fixed_point(dim):
    """A uniform (p0, U) is kept by the LKS step. With '+3/2 u^2' in f^eq (as printed) the pressure
    would grow by |U|^2 per step; with '-3/2 |u|^2' sum_i f_i^eq = 3p and p* = p (Sec. 2.2)."""
    P = box(8, 6, 6 if dim == 3 else 1, dim=dim, nt=30)
    N = P.n_cells
    U = [0.03, -0.02, 0.01][:dim]
    u0 = np.array([np.full(N, v) for v in U])
    p, u, _, _ = O.forward(P, np.zeros(1), np.full(N, 0.01), u0, _centre(P))
    assert np.abs(p - 0.01).max() < 1e-15
    assert np.abs(u - u0).max() < 1e-15


@pytest.mark.parametrize("dim", [2, 3])
def test_mass_and_momentum_conserved_periodic(dim):
    """Periodic box, no body: sum p* = sum p (the A-term's trace is a divergence) and sum u* = sum u."""
    P = box(10, 8, 6 if dim == 3 else 1, dim=dim)
    rng = np.random.default_rng(11)
    p = 0.01 * rng.standard_normal(P.n_cells)
    u = 0.05 * rng.standard_normal((dim, P.n_cells))
    ps, us = O.stencil(P, p, u)
    assert abs(ps.sum() - p.sum()) < 1e-13 * np.abs(p).sum()
    np.testing.assert_allclose(us.sum(axis=1), u.sum(axis=1), rtol=0, atol=1e-13 * np.abs(u).sum())
    assert np.abs(ps - p).max() > 1e-4  # the state did change


def _shear_wave_nu(ny, nu, nt=200, dim=2):
    P = box(4, ny, 4 if dim == 3 else 1, dim=dim, nu=nu, nt=nt)
    y = np.arange(ny)
    s = np.sin(2 * np.pi * y / ny)
    U = 1e-3
    shape = (P.nz, ny, 4)
    ux = np.broadcast_to((U * s)[None, :, None], shape).reshape(-1)
    u0 = np.zeros((dim, P.n_cells))
    u0[0] = ux
    _, u, _, _ = O.forward(P, np.zeros(1), np.zeros(P.n_cells), u0, _centre(P))
    prof = u[0].reshape(shape)[0, :, 0]
    amp = (prof @ s) / (s @ s)
    return -np.log(amp / U) / ((2 * np.pi / ny) ** 2 * nt)


def test_shear_wave_decay_gives_paper_viscosity():
    """u_x = U sin(k y) decays as exp(-nu k^2 t) with nu = (1/6 - 2A/9) dx (Sec. 2.2) at the
    paper's nu = 0.1 (Sec. 4), converging at second order in the grid spacing."""
    e32 = abs(_shear_wave_nu(32, 0.1) / 0.1 - 1)
    e64 = abs(_shear_wave_nu(64, 0.1) / 0.1 - 1)
    assert e32 < 0.006 and e64 < 0.0015
    assert 3.5 < e32 / e64 < 4.5
    assert abs(_shear_wave_nu(32, 0.05, dim=3) / 0.05 - 1) < 0.025


def _poiseuille_error(H, nu=0.1, dp=1e-4, nx=32):
    nt = int(12 * H * H / nu / np.pi ** 2)
    P = box(nx, H + 1, bc=(BC_PRESSURE, BC_WALL, BC_PERIODIC), nu=nu, nt=nt, dp=dp)
    p, u, _, _ = O.forward(P, np.zeros(1), np.zeros(P.n_cells), np.zeros((2, P.n_cells)), _centre(P))
    y = np.arange(H + 1)
    exact = dp / (2 * nu * (nx - 1)) * y * (H - y)
    num = u[0].reshape(H + 1, nx)[:, nx // 2]
    assert np.abs(u[1]).max() < 1e-4 * exact.max()
    return np.abs(num - exact).max() / exact.max()


def test_plane_poiseuille_closed_form():
    """Pressure-driven channel between no-slip walls: u_x(y) = dp/(2 nu L) y (H - y)."""
    e8, e16 = _poiseuille_error(8), _poiseuille_error(16)
    assert e16 < 0.006
    assert 3.0 < e8 / e16 < 5.0


def test_brinkman_decay_closed_form():
    """Uniform kappa over a periodic box, resting body: u(t) = U (1 + kappa)^-t (Eq. u), p unchanged,
    with kappa = kappa_max q gamma / (1 - gamma + q) (Eq. brinkman_coefficient)."""
    n = 8
    gam = 0.6
    for kind in (W_COS4, W_BILINEAR):
        P = Problem(dim=2, nx=n, ny=n, nz=1, ndx=n, ndy=n, ndz=1, body_centre=(3.5 + 0.37, 3.5 - 0.21, 0.0),
                    rot_axis=2, dof_mask=0, mass=1.0, inertia=1.0, nu=0.1, u_in=0.0, dp=0.0,
                    bc=(BC_PERIODIC,) * 3, kappa_max=1.7, q=0.1, weight_kind=kind, n_steps=7, n_itr=2,
                    obj_weights=(0,) * 8)
        kap = 1.7 * 0.1 * gam / (1 - gam + 0.1)
        u0 = np.zeros((2, P.n_cells))
        u0[0], u0[1] = 0.04, -0.01
        p, u, _, _ = O.forward(P, np.full(P.n_design, gam), np.full(P.n_cells, 0.002), u0, _centre(P))
        np.testing.assert_allclose(u[0], 0.04 * (1 + kap) ** -7, rtol=1e-13)
        np.testing.assert_allclose(u[1], -0.01 * (1 + kap) ** -7, rtol=1e-13)
        np.testing.assert_allclose(p, 0.002, rtol=1e-13)


# ------------------------------------------------------------------ coupling and EOM -------
def _framed_gamma(nd, border, seed=5):
    g = np.random.default_rng(seed).uniform(0.2, 1.0, (nd, nd))
    g[:border, :] = g[-border:, :] = g[:, :border] = g[:, -border:] = 0
    return g.reshape(-1)


@pytest.mark.parametrize("kind", [W_COS4, W_BILINEAR])
def test_galilean_free_body(kind):
    """A free body moving with a uniform periodic flow feels no force (Sec. 2.1 EOM): x^G = x0 + U t,
    and the flow stays uniform."""
    nd = 12
    g = _framed_gamma(nd, 4)
    U = (0.03, 0.01)
    P = Problem(dim=2, nx=32, ny=24, nz=1, ndx=nd, ndy=nd, ndz=1, body_centre=(12.3, 11.8, 0.0), rot_axis=2,
                dof_mask=DOF_TX | DOF_TY, mass=50.0, inertia=1.0, nu=0.05, u_in=0.0, dp=0.0, bc=(BC_PERIODIC,) * 3,
                kappa_max=2.0, q=0.1, weight_kind=kind, n_steps=15, n_itr=3, obj_weights=(1,) + (0,) * 7)
    u0 = np.zeros((2, P.n_cells))
    u0[0], u0[1] = U
    s0 = _centre(P)
    s0[3], s0[4] = U
    p, u, hist, _ = O.forward(P, g, np.zeros(P.n_cells), u0, s0)
    t = np.arange(16)
    np.testing.assert_allclose(hist[:, 0], 12.3 + U[0] * t, atol=1e-12)
    np.testing.assert_allclose(hist[:, 1], 11.8 + U[1] * t, atol=1e-12)
    assert np.abs(u[0] - U[0]).max() < 1e-13 and np.abs(u[1] - U[1]).max() < 1e-13


@pytest.mark.parametrize("n_itr", [1, 5])
def test_momentum_exchange_conserved(n_itr):
    """Fluid + body momentum sum_n u_n + M u^G is conserved exactly in a periodic box: the force on
    the body (Sec. 2.4) is the reaction of the Brinkman term (Eq. u) because the spread is the
    transpose of the interpolation, for any N_itr (both use the same iterate)."""
    nd = 12
    g = _framed_gamma(nd, 4)
    P = Problem(dim=2, nx=32, ny=24, nz=1, ndx=nd, ndy=nd, ndz=1, body_centre=(12.3, 11.8, 0.0), rot_axis=2,
                dof_mask=DOF_TX | DOF_TY, mass=30.0, inertia=1.0, nu=0.05, u_in=0.0, dp=0.0, bc=(BC_PERIODIC,) * 3,
                kappa_max=2.0, q=0.1, weight_kind=W_COS4, n_steps=12, n_itr=n_itr, obj_weights=(1,) + (0,) * 7)
    rng = np.random.default_rng(2)
    u0 = 0.02 * rng.standard_normal((2, P.n_cells)) + np.array([[0.04], [0.0]])
    s0 = _centre(P)
    p, u, hist, _ = O.forward(P, g, np.zeros(P.n_cells), u0, s0)
    before = u0.sum(axis=1)
    after = u.sum(axis=1) + P.mass * hist[-1, 3:5]
    np.testing.assert_allclose(after, before, atol=1e-12 * np.abs(u0).sum())
    assert np.abs(hist[-1, 3:5]).max() > 1e-4  # the body did pick up momentum


def test_eom_is_velocity_first_euler():
    """Sec. 2.4: u^G(t) = u^G(t-1) + F/M then x^G(t) = x^G(t-1) + u^G(t); same for omega, theta.
    Masked DOFs stay put."""
    P, g = body2d(mask=DOF_TX | DOF_ROT, nt=10)
    p0, u0, s0 = perturbed_state(P)
    _, _, h, _ = O.forward(P, g, p0, u0, s0)
    np.testing.assert_allclose(np.diff(h[:, 0]), h[1:, 3], rtol=0, atol=1e-15)
    np.testing.assert_allclose(np.diff(h[:, 6]), h[1:, 7], rtol=0, atol=1e-15)
    assert np.all(h[:, 1] == h[0, 1]) and np.all(h[:, 4] == h[0, 4])
    assert np.abs(np.diff(h[:, 3])).max() > 0 and np.abs(np.diff(h[:, 7])).max() > 0


def test_interpolation_of_uniform_field_is_exact():
    """u^ref = sum_n W u_n (Eq. u_mapping) reproduces a uniform u for any body position and angle."""
    for kind in (W_COS4, W_BILINEAR):
        P, g = body2d(wk=kind, bc=(BC_PERIODIC,) * 3)
        s = _centre(P)
        s[6] = 0.7
        u = np.zeros((2, P.n_cells))
        u[0], u[1] = 0.3, -0.2
        uref = O.interp(P, s, u)
        np.testing.assert_allclose(uref[:, 0], 0.3, rtol=1e-14)
        np.testing.assert_allclose(uref[:, 1], -0.2, rtol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_spread_is_transpose_of_interpolation(dim):
    """sum_n kappa_n u_n = sum_m kappa^ref_m u^ref_m (Eqs. kappa_mapping and u_mapping share W)."""
    P, g = body2d(wk=W_COS4) if dim == 2 else body3d(wk=W_COS4)
    s = _centre(P)
    s[6] = 0.4
    rng = np.random.default_rng(4)
    u = rng.standard_normal((dim, P.n_cells))
    kap, _, cnt = O.spread(P, g, s)
    uref = O.interp(P, s, u)
    kref = P.kappa_max * P.q * g / (1 - g + P.q)
    np.testing.assert_allclose(kap @ u.T, kref @ uref[:, :dim], rtol=1e-13)
    assert cnt.max() > 0


def test_body_outside_domain_is_an_error():
    P, g = body2d(centre=(4.5, 8.0), nt=2)
    p0, u0, s0 = initial_state(P)
    with pytest.raises(O.OracleError):
        O.forward(P, g, p0, u0, s0)


# ------------------------------------------------------------------- the adjoint ----------
CASES = [
    ("2d-rot-cos4", lambda: body2d()),
    ("2d-x-bilinear", lambda: body2d(mask=DOF_TX, wk=W_BILINEAR)),
    ("2d-rot-nitr1", lambda: body2d(n_itr=1)),
    ("2d-walls-pressure", lambda: body2d(bc=(BC_PRESSURE, BC_WALL, BC_PERIODIC), mask=DOF_TX | DOF_ROT)),
    ("2d-periodic", lambda: body2d(bc=(BC_PERIODIC,) * 3)),
    ("3d-6dof-axis-y", lambda: body3d()),
    ("3d-xyz-bilinear", lambda: body3d(mask=DOF_TX | DOF_TY | DOF_TZ, wk=W_BILINEAR, rot_axis=2)),
    ("3d-walls", lambda: body3d(bc=(BC_PRESSURE, BC_WALL, BC_WALL), rot_axis=0)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_adjoint_matches_complex_step(name, make):
    """The hand-written reverse sweep equals the complex-step derivative of the forward march
    (exact to rounding) along a random design direction and a random initial-state direction."""
    P, g = make()
    p0, u0, s0 = perturbed_state(P)
    G = O.gradient(P, g, p0, u0, s0)
    rng = np.random.default_rng(9)
    v = rng.standard_normal(g.shape)
    J, dJ = O.forward_cs(P, g, p0, u0, s0, dgamma=v)
    assert abs(J - G["J"]) <= 1e-14 * abs(J)
    assert abs(dJ - G["dJdgamma"] @ v) <= 1e-11 * abs(dJ) + 1e-16
    dp, du, ds = rng.standard_normal(p0.shape), rng.standard_normal(u0.shape), rng.standard_normal(8)
    _, dJs = O.forward_cs(P, g, p0, u0, s0, dp0=dp, du0=du, ddof0=ds)
    adj = G["lam_p0"] @ dp + (G["lam_u0"] * du).sum() + G["lam_dof0"] @ ds
    assert abs(dJs - adj) <= 1e-11 * abs(dJs)


def test_adjoint_matches_central_differences():
    """dJ/dgamma against central differences of the forward on single design variables."""
    P, g = body2d(nt=8)
    p0, u0, s0 = perturbed_state(P)
    G = O.gradient(P, g, p0, u0, s0)
    h = 1e-6
    for m in (0, 7, 14, 21, 35):
        gp, gm = g.copy(), g.copy()
        gp[m] += h
        gm[m] -= h
        Jp = O.forward(P, gp, p0, u0, s0)[3]
        Jm = O.forward(P, gm, p0, u0, s0)[3]
        fd = (Jp - Jm) / (2 * h)
        assert abs(fd - G["dJdgamma"][m]) < 1e-6 * np.abs(G["dJdgamma"]).max(), m


_STENCIL_BCS = [(BC_INFLOW_OUTFLOW, BC_PERIODIC, BC_PERIODIC), (BC_PRESSURE, BC_WALL, BC_PERIODIC),
                (BC_PERIODIC,) * 3, (BC_PRESSURE, BC_WALL, BC_WALL)]


@pytest.mark.parametrize("dim,bc", [(d, bc) for d in (2, 3) for bc in _STENCIL_BCS if d == 3 or bc[2] != BC_WALL])
def test_stencil_dot_product(dim, bc):
    """<J v, w> = <v, J^T w> for the LKS predictor with its boundary rules (Sec. 2.2), with J v by
    complex step and J^T w from the hand-written transpose (z walls only in 3D)."""
    P = box(9, 7, 6 if dim == 3 else 1, dim=dim, bc=bc, nu=0.03, u_in=0.04, dp=0.01)
    rng = np.random.default_rng(6)
    p = 0.01 * rng.standard_normal(P.n_cells)
    u = 0.05 * rng.standard_normal((dim, P.n_cells))
    vp, vu = rng.standard_normal(p.shape), rng.standard_normal(u.shape)
    wp, wu = rng.standard_normal(p.shape), rng.standard_normal(u.shape)
    jp, ju = O.stencil_jvp(P, p, u, vp, vu)
    lp, lu = O.stencil_vjp(P, p, u, wp, wu)
    lhs = jp @ wp + (ju * wu).sum()
    rhs = lp @ vp + (lu * vu).sum()
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


# ------------------------------------------------------- periodic warm start (Sec. 3.4) ----
def test_terminal_adjoint_is_the_derivative_of_the_terminal_functional():
    """A reverse sweep started from a terminal adjoint (lam_p, lam_u, lam_s at N_t) differentiates
    J + lam_p.p(N_t) + lam_u.u(N_t) + lam_s.s(N_t): checked against the complex-step derivative of
    that functional, with the terminal adjoint taken from a previous sweep's initial adjoint as the
    warm start of periodic problems does."""
    P, g = body2d(nt=6)
    p0, u0, s0 = perturbed_state(P)
    first = O.gradient(P, g, p0, u0, s0)
    pT, uT, sT = first["lam_p0"], first["lam_u0"], first["lam_dof0"]
    G = O.gradient_terminal(P, g, p0, u0, s0, pT, uT, sT)
    assert abs(G["J"] - first["J"]) == 0.0
    v = np.random.default_rng(12).standard_normal(g.shape)
    dJ = O.forward_cs_terminal(P, g, p0, u0, s0, pT, uT, sT, v)
    assert abs(dJ - G["dJdgamma"] @ v) <= 1e-11 * abs(dJ)
    assert np.abs(G["dJdgamma"] - first["dJdgamma"]).max() > 1e-6 * np.abs(first["dJdgamma"]).max()


def test_openmp_timing_build_is_bitwise_the_oracle():
    """The OpenMP timing build of the oracle (used only to time the CPU baseline on all host cores)
    gives the single-threaded oracle's results bit for bit: it only spreads independent per-node
    loops, each output computed by the same operations in the same order."""
    from tests.problems import body2d, body3d, perturbed_state
    if not O.set_variant("openmp"):
        pytest.skip("no OpenMP build on this host")
    try:
        outs = {}
        for variant in ("openmp", "serial"):
            assert O.set_variant(variant)
            for name, (P, g) in (("2d", body2d(nt=4)), ("3d", body3d(nt=3))):
                p0, u0, s0 = perturbed_state(P)
                outs[(variant, name)] = O.gradient(P, g, p0, u0, s0)
        for name in ("2d", "3d"):
            a, b = outs[("openmp", name)], outs[("serial", name)]
            assert a["J"] == b["J"]
            for k in ("dJdgamma", "lam_p0", "lam_u0", "lam_dof0"):
                assert np.array_equal(a[k], b[k]), (name, k)
    finally:
        O.set_variant("serial")
