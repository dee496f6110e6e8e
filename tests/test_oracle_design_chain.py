"""Pins for the oracle's design chain (no GPU): cyclic expansion (Sec. 4.2), density filter
(Sec. 3.2, Eq. filter), Heaviside projection (Eq. projection), the volume constraint
(Eq. constraint) and the chain's transpose inside the gradient.

The pins are properties the definitions fix: a normalised symmetric filter reproduces constant
fields everywhere and linear fields wherever its support is whole, a radius of one keeps the
field; the projection maps 0 to 0 and 1 to 1 and tends to a step at eta; the cyclic expansion is
invariant under the lattice rotation; the transposes pass dot-product tests against complex-step
Jacobian-vector products; the gradient with the chain matches the complex-step derivative of the
whole forward march.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from tests.problems import BC_PERIODIC, DOF_ROT, DOF_TX, body2d, body3d, perturbed_state

PERIODIC = (BC_PERIODIC,) * 3


def _design2d(nd=16, **kw):
    P, g = body2d(nd=nd, nx=40, ny=32, centre=(16.3, 15.8), bc=PERIODIC)
    return P.replace(**kw), g


def test_filter_keeps_constant_fields():
    P, _ = _design2d(filter_radius=2.7)
    g = np.full(P.n_design, 0.37)
    np.testing.assert_allclose(O.design_chain(P, g), 0.37, rtol=1e-15)


def test_filter_reproduces_linear_fields_away_from_the_edges():
    """Symmetric weights: the filtered value of a + b x + c y is exact wherever the whole disc of
    radius R lies inside the design grid."""
    R = 2.7
    P, _ = _design2d(nd=16, filter_radius=R)
    j, i = np.meshgrid(np.arange(16), np.arange(16), indexing="ij")
    g = (0.2 + 0.03 * i - 0.017 * j).reshape(-1)
    out = O.design_chain(P, g).reshape(16, 16)
    inner = (i >= 3) & (i <= 12) & (j >= 3) & (j <= 12)
    np.testing.assert_allclose(out[inner], g.reshape(16, 16)[inner], rtol=0, atol=1e-15)
    assert np.abs(out[~inner] - g.reshape(16, 16)[~inner]).max() > 1e-4  # truncated at the edges


def test_filter_radius_one_is_the_identity():
    P, g = _design2d(filter_radius=1.0)
    np.testing.assert_array_equal(O.design_chain(P, g), g)


def test_projection_endpoints_and_step_limit():
    for eta in (0.5, 0.3):
        P, _ = _design2d(proj_beta=6.0, proj_eta=eta)
        out = O.design_chain(P, np.array([0.0, 1.0] + [0.5] * (P.n_design - 2)))
        assert abs(out[0]) < 1e-15 and abs(out[1] - 1.0) < 1e-15
    P, _ = _design2d(proj_beta=6.0, proj_eta=0.5)
    assert abs(O.design_chain(P, np.full(P.n_design, 0.5))[0] - 0.5) < 1e-15  # symmetric about eta = 1/2
    x = np.linspace(0, 1, P.n_design)
    y = O.design_chain(P, x)
    assert np.all(np.diff(y) > 0)  # monotone
    P, _ = _design2d(proj_beta=400.0, proj_eta=0.4)
    y = O.design_chain(P, x)
    np.testing.assert_allclose(y[x < 0.35], 0.0, atol=1e-8)
    np.testing.assert_allclose(y[x > 0.45], 1.0, atol=1e-8)


@pytest.mark.parametrize("order", [2, 4])
def test_cyclic_expansion_is_invariant_under_the_rotation(order):
    """With order 4 (2) the design is unchanged by rotating the design grid by 90 (180) degrees
    about its centre; filter and projection keep that symmetry; every orbit takes its
    representative's value."""
    P, _ = _design2d(nd=12, cyclic_order=order)
    rng = np.random.default_rng(3)
    g = rng.random(P.n_design)
    raw = O.design_chain(P, g).reshape(12, 12)
    k = 1 if order == 4 else 2
    np.testing.assert_array_equal(np.rot90(raw, k), raw)
    assert len(np.unique(raw)) == 144 // order  # orbits of 4 (2) points, all distinct values
    P2 = P.replace(filter_radius=2.2, proj_beta=4.0)
    out = O.design_chain(P2, g).reshape(12, 12)
    np.testing.assert_allclose(np.rot90(out, k), out, rtol=0, atol=1e-15)


def test_cyclic_expansion_3d_about_the_rotation_axis():
    P, g = body3d(nd=6, rot_axis=0, nx=20, ny=16, nz=16, centre=(8.3, 7.9, 8.1), bc=PERIODIC)
    P = P.replace(cyclic_order=4)
    rng = np.random.default_rng(4)
    out = O.design_chain(P, rng.random(P.n_design)).reshape(6, 6, 6)  # [z][y][x]
    # rotation about x maps (y, z) -> (-z, y): in the [z][y] array that is a quarter turn
    np.testing.assert_array_equal(np.rot90(out, 1, axes=(0, 1)), out)


@pytest.mark.parametrize("kw", [dict(filter_radius=2.3), dict(proj_beta=5.0, proj_eta=0.4),
                                dict(cyclic_order=4), dict(filter_radius=1.8, proj_beta=3.0, cyclic_order=4),
                                dict(filter_radius=2.1, proj_beta=2.0, design_radius=5.2)])
def test_chain_transpose_dot_product(kw):
    """<J v, w> = <v, J^T w> with J v by complex step and J^T w by the hand-written transpose."""
    P, _ = _design2d(nd=12, **kw)
    rng = np.random.default_rng(5)
    g = rng.random(P.n_design)
    v, w = rng.standard_normal(P.n_design), rng.standard_normal(P.n_design)
    lhs = O.design_chain_jvp(P, g, v) @ w
    rhs = v @ O.design_chain_vjp(P, g, w)
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)


def test_gradient_through_the_design_chain_matches_complex_step():
    P, g = body2d(nd=8, nx=30, ny=24, centre=(12.3, 11.8), mask=DOF_ROT, nt=5)
    P = P.replace(filter_radius=1.9, proj_beta=4.0, proj_eta=0.45, cyclic_order=4)
    p0, u0, s0 = perturbed_state(P)
    G = O.gradient(P, g, p0, u0, s0)
    rng = np.random.default_rng(6)
    v = rng.standard_normal(g.shape)
    J, dJ = O.forward_cs(P, g, p0, u0, s0, dgamma=v)
    assert abs(dJ - G["dJdgamma"] @ v) <= 1e-11 * abs(dJ)
    # only orbit representatives (the smallest index among the four quarter-turn images) carry
    # sensitivity
    nd = P.ndx
    idx = np.arange(nd * nd).reshape(nd, nd)
    orbit_min = np.minimum.reduce([np.rot90(idx, k) for k in range(4)]).reshape(-1)
    reps = orbit_min == np.arange(nd * nd)
    assert np.all(G["dJdgamma"][~reps] == 0.0) and np.abs(G["dJdgamma"][reps]).max() > 0


def test_volume_constraint():
    P, _ = _design2d(v_min=0.25)
    G, _ = O.constraint(P, np.ones(P.n_design))
    assert abs(G - (1 / 0.25 - 1)) < 1e-14
    P, _ = _design2d(nd=12, v_min=0.3, filter_radius=2.2, proj_beta=3.0, cyclic_order=2, design_radius=5.0)
    rng = np.random.default_rng(7)
    g = rng.random(P.n_design)
    G, dG = O.constraint(P, g)
    v = rng.standard_normal(P.n_design)
    r = np.arange(12) - 5.5
    dom = ((r[None, :] ** 2 + r[:, None] ** 2) <= 25.0).reshape(-1)
    jv = O.design_chain_jvp(P, g, v)
    assert abs(dG @ v - jv[dom].sum() / (0.3 * dom.sum())) <= 1e-13 * abs(dG @ v)
    assert abs(G - (O.design_chain(P, g)[dom].sum() / (0.3 * dom.sum()) - 1)) < 1e-14


def test_cyclic_transpose_on_an_odd_grid():
    """On an odd grid the centre is its own image under every rotation: its sensitivity is counted
    once. Pinned by the dot-product test against the complex-step expansion."""
    P, _ = _design2d(nd=9, cyclic_order=4, filter_radius=1.5)
    rng = np.random.default_rng(8)
    g = rng.random(P.n_design)
    v, w = rng.standard_normal(P.n_design), rng.standard_normal(P.n_design)
    lhs = O.design_chain_jvp(P, g, v) @ w
    rhs = v @ O.design_chain_vjp(P, g, w)
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)
