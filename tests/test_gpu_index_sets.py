"""Bit-exact integer indexing of the CUDA path against the oracle (through the C ABI).

Spread (Sec. 2.3, Eqs. kappa_mapping, us_mapping, weight_function): for a DOF iterate, the design
points the coupling's gather accepts for each cell of the body box (lks_support_sets) must be the
oracle's index sets (oracle support_sets: the nodes of each design point's support window), compared
as integers with np.array_equal: count, least and largest index, and the sums of the indices and
their squares per cell. The acceptance is decided in FP64 on both sides (FP64 handles). Cases: 2D
cosine and bilinear kernels at a generic angle, support edges placed exactly on nodes (|r| = 2 for
the cosine kernel, |r| = 1 for the bilinear one, on a wrapped periodic grid too), a 3D single-axis
rotation, six DOFs with a rotated R and a ball-shaped design domain.

Stencil (Sec. 2.2, Eqs. p_tmp, u_tmp, local_equilibrium_function, boundary values): one FP64 step
from a unit probe in p, u_x or u_y at interior, boundary and wrapped nodes; the set of nodes the
probe reaches (|value| above 1e-13 of the largest) must be the oracle's, node for node, and the
values must agree to rounding.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from tests.problems import BC_INFLOW_OUTFLOW, BC_PERIODIC, BC_PRESSURE, BC_WALL, box
from tests.test_oracle_index_sets import _cases

pytestmark = pytest.mark.gpu


def _box_to_grid(P, lo, B):
    """Grid node of every box cell (x fastest), or -1 outside a non-periodic axis."""
    n = (P.nx, P.ny, P.nz)
    j = np.indices((B[2], B[1], B[0])).reshape(3, -1)[::-1]  # (x, y, z) of box cells, x fastest
    node = np.zeros(j.shape[1], dtype=np.int64)
    ok = np.ones(j.shape[1], dtype=bool)
    stride = 1
    for a in range(3):
        if a >= P.dim:
            continue
        p = lo[a] + j[a]
        if P.bc[a] == BC_PERIODIC:
            p = np.mod(p, n[a])
        else:
            ok &= (p >= 0) & (p < n[a])
        node += stride * np.where(ok, p, 0)
        stride *= n[a]
    return np.where(ok, node, -1)


@pytest.mark.parametrize("name,P,s", list(_cases()), ids=[c[0] for c in _cases()])
def test_spread_index_sets_bit_exact(name, P, s):
    from paper_2601_18272_gb300 import lks
    from paper_2601_18272_gb300.lks import Solver
    S = Solver(P, precision=64, ckpt_policy=0)
    try:
        lo, B, gpu = lks.lks_support_sets(S.handle, s)
    finally:
        S.close()
    ref = O.support_sets(P, s)
    node = _box_to_grid(P, lo, B)
    inside = node >= 0
    assert np.array_equal(gpu[inside], ref[node[inside]])
    assert np.all(gpu[~inside, 0] == 0)  # nothing accepted outside a non-periodic boundary
    covered = np.zeros(P.n_cells, dtype=bool)
    covered[node[inside]] = True
    assert np.all(ref[~covered, 0] == 0)  # the box holds every node the body reaches
    assert ref[:, 0].sum() > 0


def _probe_cases():
    yield "periodic", box(20, 12, nt=1), [(0, 0), (19, 11), (5, 6), (0, 6)]
    yield "inflow-walls", box(20, 12, bc=(BC_INFLOW_OUTFLOW, BC_WALL, BC_PERIODIC), nt=1), \
        [(0, 5), (1, 5), (2, 0), (18, 11), (19, 3), (10, 0), (10, 1), (1, 1), (19, 10)]
    yield "pressure-periodic", box(21, 13, bc=(BC_PRESSURE, BC_PERIODIC, BC_PERIODIC), nt=1, dp=0.01), \
        [(0, 0), (1, 12), (20, 6), (19, 0), (10, 6)]


@pytest.mark.parametrize("name,P,probes", list(_probe_cases()), ids=[c[0] for c in _probe_cases()])
def test_stencil_probe_supports(name, P, probes):
    from paper_2601_18272_gb300.lks import Solver
    import torch
    nx, ny, N = P.nx, P.ny, P.n_cells
    S = Solver(P, precision=64, ckpt_policy=0)
    try:
        for (x, y) in probes:
            for field in range(3):
                p0 = np.zeros(N)
                u0 = np.zeros((2, N))
                if field == 0:
                    p0[x + nx * y] = 1.0
                else:
                    u0[field - 1, x + nx * y] = 0.01
                S.set_initial_state(p0, u0, None)
                S.forward(torch.zeros(P.n_design, dtype=torch.float64, device="cuda"))
                pg, ug = S.state()
                po, uo, _, _ = O.forward(P, np.zeros(P.n_design), p0, u0, O_state(P), n_steps=1)
                for a, b in ((pg, po), (ug[0], uo[0]), (ug[1], uo[1])):
                    scale = max(np.abs(b).max(), 1e-300)
                    assert np.array_equal(np.abs(a) > 1e-13 * scale, np.abs(b) > 1e-13 * scale), (x, y, field)
                    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13 * max(scale, 1e-3))
    finally:
        S.close()


def O_state(P):
    from workloads import initial_state
    return initial_state(P)[2]
