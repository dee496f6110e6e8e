"""The oracle's index sets of the spread (Sec. 2.3, Eqs. kappa_mapping, weight_function) against a
brute force over (node, design point) pairs.

The oracle enumerates each design point's support window from floor(x^ref) (its scatter); the brute
force here instead tests every design point of the domain against the strict support condition
|p - x^ref_a| < s for the unwrapped integer positions p of each axis, with periodic images. These
index sets are what the GPU's gather must reproduce bit-exactly (tests/test_gpu_index_sets.py).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import oracle as O
from tests.problems import (BC_INFLOW_OUTFLOW, BC_PERIODIC, DOF_TX, W_BILINEAR, body2d, body3d, body6,
                            perturbed_state, perturbed_state6)


def _rotation(P, s):
    if P.rot_axis == -1:
        return np.asarray(s[12:21], dtype=float).reshape(3, 3)
    a = P.rot_axis
    b, c = (a + 1) % 3, (a + 2) % 3
    R = np.eye(3)
    ct, st = math.cos(s[6]), math.sin(s[6])
    R[b, b], R[b, c], R[c, b], R[c, c] = ct, -st, st, ct
    return R


def brute_force_sets(P, s):
    d = P.dim
    n = (P.nx, P.ny, P.nz)
    nd = (P.ndx, P.ndy, P.ndz)
    sup = 1 if P.weight_kind == W_BILINEAR else 2
    R = _rotation(P, s)
    stats = np.zeros((P.n_cells, 5), dtype=np.int64)
    stats[:, 1] = -1
    stats[:, 2] = -1
    rad4 = math.floor(4 * P.design_radius ** 2) if P.design_radius > 0 else None
    for m in range(P.n_design):
        i = (m % nd[0], (m // nd[0]) % nd[1], m // (nd[0] * nd[1]))
        r = np.array([(i[a] - (nd[a] - 1) / 2.0) if a < d else 0.0 for a in range(3)])
        if rad4 is not None and sum((2 * i[a] - (nd[a] - 1)) ** 2 for a in range(d)) > rad4:
            continue
        xref = np.array(s[:3], dtype=float) + R @ r
        per_axis = []
        for a in range(3):
            if a >= d:
                per_axis.append([0])
                continue
            cand = range(int(math.floor(xref[a])) - sup - 1, int(math.floor(xref[a])) + sup + 2)
            ps = [p for p in cand if abs(p - xref[a]) < sup]
            if P.bc[a] == BC_PERIODIC:
                ps = [p % n[a] for p in ps]
            per_axis.append(ps)
        for pz in per_axis[2]:
            for py in per_axis[1]:
                for px in per_axis[0]:
                    node = px + n[0] * (py + n[1] * pz)
                    st = stats[node]
                    if st[0] == 0 or m < st[1]:
                        st[1] = m
                    st[2] = max(st[2], m)
                    st[0] += 1
                    st[3] += m
                    st[4] += m * m
    return stats


def _cases():
    P, _ = body2d()
    _, _, s = perturbed_state(P)
    s[6] = 0.37
    yield "2d-cos-rotated", P, s
    P, _ = body2d(wk=W_BILINEAR, nd=5, centre=(10.4, 7.7))
    _, _, s = perturbed_state(P)
    s[6] = -0.83
    yield "2d-bilinear-rotated", P, s
    P, _ = body2d(nd=7, centre=(10.0, 8.0), mask=DOF_TX)
    _, _, s = perturbed_state(P)
    s[6] = 0.0
    yield "2d-edge-ties", P, s
    P, _ = body2d(nd=7, centre=(11.0, 8.0), wk=W_BILINEAR, mask=DOF_TX, bc=(BC_PERIODIC,) * 3)
    _, _, s = perturbed_state(P)
    s[6] = 0.0
    yield "2d-bilinear-ties-periodic", P, s
    P, _ = body3d(nx=24, ny=16, nz=16, centre=(9.3, 7.6, 8.2))
    _, _, s = perturbed_state(P)
    s[6] = 0.41
    yield "3d-axis-rotated", P, s
    P, _ = body6(radius=2.6, sphere=True)
    _, _, s = perturbed_state6(P)
    yield "6dof-ball", P, s


@pytest.mark.parametrize("name,P,s", list(_cases()), ids=[c[0] for c in _cases()])
def test_oracle_index_sets_match_brute_force(name, P, s):
    got = O.support_sets(P, s)
    ref = brute_force_sets(P, s)
    assert np.array_equal(got, ref)
    assert got[:, 0].sum() > 0


def test_index_sets_are_not_vacuous():
    """A shifted body changes the sets: the comparison above sees the position."""
    P, _ = body2d()
    _, _, s = perturbed_state(P)
    a = O.support_sets(P, s)
    s2 = s.copy()
    s2[0] += 0.5
    assert not np.array_equal(a, O.support_sets(P, s2))
    assert BC_INFLOW_OUTFLOW == P.bc[0]
