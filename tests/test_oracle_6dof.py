"""Pins for the oracle's freely rotating 3D body (six DOFs) and its ball-shaped design domain (no GPU).

The paper integrates one rotation axis and names Euler angles or quaternions as the way to more;
the six-DOF scheme here keeps its explicit, velocity-first Euler form: h^(k) = h(t-1) + T^(k),
omega^(k) = R(t-1) I_b^-1 R(t-1)^T h^(k), R^(k) = exp([omega^(k)]x) R(t-1). The pins: the
closed-form torque-free motion of an isotropic body, scipy's exponential map for an anisotropic one,
exact reduction to the pinned single-axis scheme, momentum exchange with a rotated body, a
brute-force count of the design points each node sees, and complex-step derivatives for the adjoint.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from tests.problems import (BC_INFLOW_OUTFLOW, BC_PERIODIC, BC_PRESSURE, BC_WALL, DOF_ROT, DOF_TX, DOF_TY, DOF_TZ,
                            W_BILINEAR, W_COS4, body3d, body6, perturbed_state6, rotvec_matrix)
from workloads import initial_state

PERIODIC = (BC_PERIODIC,) * 3


def _free_state(P, R0, h0, om0, ug=(0.0, 0.0, 0.0)):
    p0, u0, s0 = initial_state(P)
    s0[3:6] = ug
    s0[6:9] = h0
    s0[9:12] = om0
    s0[12:21] = np.asarray(R0).reshape(-1)
    return p0, u0, s0


@pytest.mark.parametrize("omega", [(0.01, -0.02, 0.015), (0.12, 0.2, -0.09)])
def test_torque_free_isotropic_body_closed_form(omega):
    """kappa_max = 0 leaves the body without force or torque. With I_b = c 1 the angular velocity
    is h / c, constant, and R(t) = exp(t [omega]x) R0: the rotation by t |omega| about omega.
    The two speeds take the small-angle series and the closed form of Rodrigues' formula."""
    c = 37.0
    P, g = body6(bc=PERIODIC, kappa_max=0.0, nt=25)
    P = P.replace(inertia_tensor=(c, 0, 0, 0, c, 0, 0, 0, c))
    om = np.array(omega)
    R0 = rotvec_matrix((0.4, -0.1, 0.7))
    ug = np.array([0.01, 0.002, -0.003])
    p0, u0, s0 = _free_state(P, R0, c * om, om, ug)
    _, _, hist, _ = O.forward(P, g, p0, u0, s0)
    t = np.arange(P.n_steps + 1)
    np.testing.assert_allclose(hist[:, 0:3], np.array(P.body_centre) + t[:, None] * ug, rtol=0, atol=1e-13)
    assert np.all(hist[:, 6:9] == c * om)  # h untouched by a zero torque
    np.testing.assert_allclose(hist[1:, 9:12], np.tile(om, (P.n_steps, 1)), rtol=1e-13, atol=0)
    for k in (1, 7, 25):
        np.testing.assert_allclose(hist[k, 12:21].reshape(3, 3), rotvec_matrix(k * om) @ R0, rtol=0, atol=2e-14)


def test_torque_free_anisotropic_body_exponential_map():
    """Torque-free anisotropic body: h is conserved exactly, each step is R(t) = exp([w]x) R(t-1)
    with w = R(t-1) I_b^-1 R(t-1)^T h (scipy's rotation-vector map, numpy's inverse), and R stays
    orthogonal with determinant 1."""
    P, g = body6(bc=PERIODIC, kappa_max=0.0, nt=30, scale_inertia=0.01)
    Ib = np.array(P.inertia_tensor).reshape(3, 3)
    assert np.abs(np.linalg.eigvalsh(Ib) - np.linalg.eigvalsh(Ib).mean()).max() > 0.05 * np.abs(Ib).max()
    h0 = np.array([0.5, -0.3, 0.8])
    p0, u0, s0 = _free_state(P, rotvec_matrix((0.2, 0.5, -0.3)), h0, np.zeros(3))
    _, _, hist, _ = O.forward(P, g, p0, u0, s0)
    Jinv = np.linalg.inv(Ib)
    assert np.all(hist[:, 6:9] == h0)
    for t in range(1, P.n_steps + 1):
        Rp = hist[t - 1, 12:21].reshape(3, 3)
        w = Rp @ Jinv @ Rp.T @ h0
        np.testing.assert_allclose(hist[t, 9:12], w, rtol=1e-13)
        np.testing.assert_allclose(hist[t, 12:21].reshape(3, 3), rotvec_matrix(w) @ Rp, rtol=0, atol=1e-14)
    R = hist[-1, 12:21].reshape(3, 3)
    np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-14)
    assert abs(np.linalg.det(R) - 1) < 1e-14
    assert np.abs(hist[-1, 9:12] - hist[1, 9:12]).max() > 1e-4  # the axis does precess


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_free_rotation_reduces_to_single_axis(axis):
    """Starting unrotated and spinning about a principal axis a, one step with N_itr = 1 of the
    six-DOF scheme equals the (pinned) single-axis scheme about a: the same fields, body position
    and velocity, and omega_a(1) = omega(1), h_a(1) = I_aa omega(1). This pins the torque
    component about each axis, the solid velocity omega x R r and the angular update."""
    P6, g = body6(n_itr=1, nt=1, scale_inertia=0.01)
    Ib = np.diag(np.diag(np.array(P6.inertia_tensor).reshape(3, 3)))
    P6 = P6.replace(inertia_tensor=tuple(Ib.reshape(-1)))
    Ia = Ib[axis, axis]
    P1 = body3d(nx=P6.nx, ny=P6.ny, nz=P6.nz, nd=P6.ndx, centre=P6.body_centre, rot_axis=axis, n_itr=1, nt=1,
                mass=P6.mass, inertia=Ia)[0]
    P1 = P1.replace(kappa_max=P6.kappa_max)
    om = 0.02
    ug = np.array([0.01, -0.004, 0.003])
    p0, u0, s6 = _free_state(P6, np.eye(3), Ia * om * np.eye(3)[axis], om * np.eye(3)[axis], ug)
    s1 = np.zeros(8)
    s1[0:3] = P6.body_centre
    s1[3:6] = ug
    s1[7] = om
    pa, ua, h6, _ = O.forward(P6, g, p0, u0, s6)
    pb, ub, h1, _ = O.forward(P1, g, p0, u0, s1)
    np.testing.assert_allclose(pa, pb, rtol=0, atol=1e-15)
    np.testing.assert_allclose(ua, ub, rtol=0, atol=1e-15)
    np.testing.assert_allclose(h6[1, 0:6], h1[1, 0:6], rtol=1e-14, atol=1e-17)
    assert abs(h6[1, 9 + axis] - h1[1, 7]) <= 1e-14 * abs(h1[1, 7])
    assert abs(h6[1, 6 + axis] - Ia * h1[1, 7]) <= 1e-13 * abs(Ia * h1[1, 7])
    assert abs(h1[1, 7] - om) > 1e-6  # the torque did act


def test_momentum_exchange_with_rotated_body():
    """Periodic box, translating body held at a fixed rotation R0 that maps the design lattice onto
    itself (a cyclic permutation of the axes): the fluid + body momentum sum_n u_n + M u^G is
    conserved to rounding. The force of Sec. 2.4 is the reaction of the Brinkman term, and a
    uniform u^S spreads to a uniform field inside a design grid whose border carries gamma = 0 (the
    weights of an axis-aligned lattice sum to one; a generic rotation would break that)."""
    P, g = body6(nx=24, ny=20, nz=20, nd=10, centre=(11.2, 9.7, 10.4), bc=PERIODIC,
                 mask=DOF_TX | DOF_TY | DOF_TZ, n_itr=3, nt=8)
    g = g.reshape(10, 10, 10).copy()  # zero border of 3 points: every cell near gamma > 0 sees a full lattice
    g[:3], g[-3:], g[:, :3], g[:, -3:], g[:, :, :3], g[:, :, -3:] = 0, 0, 0, 0, 0, 0
    g = g.reshape(-1)
    rng = np.random.default_rng(5)
    R0 = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    p0, u0, s0 = _free_state(P, R0, np.zeros(3), np.zeros(3))
    u0 = 0.02 * rng.standard_normal(u0.shape) + np.array([[0.04], [0.0], [0.01]])
    p, u, hist, _ = O.forward(P, g, p0, u0, s0)
    before = u0.sum(axis=1)
    after = u.sum(axis=1) + P.mass * hist[-1, 3:6]
    np.testing.assert_allclose(after, before, atol=1e-12 * np.abs(u0).sum())
    assert np.abs(hist[-1, 3:6]).max() > 1e-5
    assert np.all(hist[:, 12:21] == s0[12:21])  # the rotation DOF is masked: R stays


@pytest.mark.parametrize("radius", [0.0, 2.2, 3.1])
def test_design_domain_brute_force_count(radius):
    """The design points a node sees: those of the domain |r_m| <= radius (all if radius = 0)
    whose mapped position x^G + R r_m lies within the open support |x_n - x^ref_m|_a < 2 on every
    axis. Counted here by brute force over all (node, design point) pairs."""
    P, g = body6(nx=16, ny=14, nz=14, centre=(7.3, 6.9, 7.1), bc=PERIODIC, radius=radius)
    R = rotvec_matrix((0.3, -0.7, 0.45))
    s = np.zeros(21)
    s[0:3] = P.body_centre
    s[12:21] = R.reshape(-1)
    _, _, cnt = O.spread(P, g, s)
    nd = P.ndx
    k, j, i = np.meshgrid(np.arange(nd), np.arange(nd), np.arange(nd), indexing="ij")
    r = np.stack([i, j, k], -1).reshape(-1, 3) - (nd - 1) / 2.0
    if radius > 0:
        r = r[(r ** 2).sum(1) <= radius * radius]
    xref = np.array(P.body_centre) + r @ R.T
    n = np.array([P.nx, P.ny, P.nz])
    zz, yy, xx = np.meshgrid(np.arange(P.nz), np.arange(P.ny), np.arange(P.nx), indexing="ij")
    nodes = np.stack([xx, yy, zz], -1).reshape(-1, 3)
    d = nodes[:, None, :] - xref[None, :, :]
    d = (d + n / 2) % n - n / 2  # periodic nearest image
    brute = np.all(np.abs(d) < 2.0, axis=2).sum(axis=1)
    assert np.array_equal(cnt, brute)
    assert brute.sum() > 0


def test_design_radius_covering_the_grid_changes_nothing():
    """A domain radius at least the design grid's half diagonal keeps every point: identical results."""
    P, g = body6(nt=3)
    p0, u0, s0 = perturbed_state6(P)
    a = O.forward(P, g, p0, u0, s0)
    b = O.forward(P.replace(design_radius=np.sqrt(3) * (P.ndx - 1) / 2 + 1e-9), g, p0, u0, s0)
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[1], b[1])


CASES = [
    ("free", lambda: body6()),
    ("free-ball-domain", lambda: body6(nd=7, radius=2.6)),
    ("free-bilinear", lambda: body6(wk=W_BILINEAR)),
    ("free-walls-pressure", lambda: body6(bc=(BC_PRESSURE, BC_WALL, BC_WALL), centre=(9.2, 7.8, 8.1))),
    ("free-nitr1", lambda: body6(n_itr=1, nt=3)),
    ("free-rotation-masked", lambda: body6(mask=DOF_TX | DOF_TZ)),
    ("free-rotation-only", lambda: body6(mask=DOF_ROT, scale_inertia=0.01)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_free_rotation_adjoint_matches_complex_step(name, make):
    """The reverse sweep with six DOFs equals the complex-step derivative of the forward march along
    random design and initial-state directions (all 21 DOF components, R included)."""
    P, g = make()
    p0, u0, s0 = perturbed_state6(P)
    G = O.gradient(P, g, p0, u0, s0)
    rng = np.random.default_rng(11)
    v = rng.standard_normal(g.shape)
    J, dJ = O.forward_cs(P, g, p0, u0, s0, dgamma=v)
    assert abs(J - G["J"]) <= 1e-14 * abs(J)
    assert abs(dJ - G["dJdgamma"] @ v) <= 1e-11 * abs(dJ) + 1e-16
    dp, du, ds = rng.standard_normal(p0.shape), rng.standard_normal(u0.shape), rng.standard_normal(21)
    _, dJs = O.forward_cs(P, g, p0, u0, s0, dp0=dp, du0=du, ddof0=ds)
    adj = G["lam_p0"] @ dp + (G["lam_u0"] * du).sum() + G["lam_dof0"] @ ds
    assert abs(dJs - adj) <= 1e-11 * abs(dJs)
    if P.design_radius > 0:
        nd = P.ndx
        k, j, i = np.meshgrid(np.arange(nd), np.arange(nd), np.arange(nd), indexing="ij")
        r2 = ((np.stack([i, j, k], -1).reshape(-1, 3) - (nd - 1) / 2.0) ** 2).sum(1)
        out = r2 > P.design_radius ** 2
        assert out.any() and np.all(G["dJdgamma"][out] == 0.0)
