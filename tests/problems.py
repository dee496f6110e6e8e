"""Small seeded problems used by the oracle pins and the GPU parity tests."""
from __future__ import annotations

import numpy as np

from workloads import (BC_INFLOW_OUTFLOW, BC_PERIODIC, BC_PRESSURE, BC_WALL, DOF_ROT, DOF_TX, DOF_TY, DOF_TZ,
                       ROT_FREE, W_BILINEAR, W_COS4, Problem, gamma_2d, gamma_3d, inertia_tensor, initial_state,
                       mass_properties)

__all__ = ["box", "body2d", "body3d", "body6", "perturbed_state", "perturbed_state6", "rotvec_matrix",
           "BC_INFLOW_OUTFLOW", "BC_PERIODIC", "BC_PRESSURE", "BC_WALL", "DOF_ROT", "DOF_TX", "DOF_TY", "DOF_TZ",
           "ROT_FREE", "W_BILINEAR", "W_COS4"]


def box(nx, ny, nz=1, dim=2, bc=(BC_PERIODIC,) * 3, nu=0.1, nt=100, dp=0.0, u_in=0.0):
    """A grid with a single design point carrying gamma = 0: the fluid alone."""
    c = (nx / 2.0, ny / 2.0, nz / 2.0 if dim == 3 else 0.0)
    return Problem(dim=dim, nx=nx, ny=ny, nz=nz, ndx=1, ndy=1, ndz=1, body_centre=c, rot_axis=2,
                   dof_mask=0, mass=1.0, inertia=1.0, nu=nu, u_in=u_in, dp=dp, bc=bc, kappa_max=1.0, q=0.1,
                   weight_kind=W_BILINEAR, n_steps=nt, n_itr=1, obj_weights=(0.0,) * 8)


def body2d(nx=24, ny=16, nd=6, centre=(10.3, 8.2), mask=DOF_TX | DOF_TY | DOF_ROT, wk=W_COS4,
           bc=(BC_INFLOW_OUTFLOW, BC_PERIODIC, BC_PERIODIC), n_itr=3, nt=6, mass=None, inertia=None, seed=7,
           nu=0.05, kappa_max=2.0, q=0.1, obj=(0.3, 0.2, 0.0, 0.1, 0.05, 0.0, 1.0, 0.5), precision=64):
    g = gamma_2d(nd, seed)
    M, I = mass_properties(g, (nd, nd, 1), 2, 2)
    P = Problem(dim=2, nx=nx, ny=ny, nz=1, ndx=nd, ndy=nd, ndz=1, body_centre=(centre[0], centre[1], 0.0),
                rot_axis=2, dof_mask=mask, mass=M if mass is None else mass, inertia=I if inertia is None else inertia,
                nu=nu, u_in=0.05, dp=0.0, bc=bc, kappa_max=kappa_max, q=q, weight_kind=wk, n_steps=nt, n_itr=n_itr,
                obj_weights=obj, field_precision=precision)
    return P, g


def body3d(nx=16, ny=12, nz=12, nd=4, centre=(7.3, 6.2, 5.9), mask=DOF_TX | DOF_TY | DOF_TZ | DOF_ROT, rot_axis=1,
           wk=W_COS4, bc=(BC_INFLOW_OUTFLOW, BC_PERIODIC, BC_PERIODIC), n_itr=3, nt=6, mass=80.0, inertia=300.0,
           seed=7, nu=0.05, obj=(0.3, 0.2, 0.1, 0.1, 0.05, 0.0, 1.0, 0.5), precision=64):
    g = gamma_3d(nd, seed)
    P = Problem(dim=3, nx=nx, ny=ny, nz=nz, ndx=nd, ndy=nd, ndz=nd, body_centre=centre, rot_axis=rot_axis,
                dof_mask=mask, mass=mass, inertia=inertia, nu=nu, u_in=0.05, dp=0.0, bc=bc, kappa_max=2.0, q=0.1,
                weight_kind=wk, n_steps=nt, n_itr=n_itr, obj_weights=obj, field_precision=precision)
    return P, g


def perturbed_state(P, seed=1, amp=0.01, ug=0.01, omega=0.003):
    """Impulsive-start state plus seeded noise, with a moving body, for derivative tests."""
    p0, u0, s0 = initial_state(P)
    rng = np.random.default_rng(seed)
    p0 = p0 + amp * rng.standard_normal(p0.shape)
    u0 = u0 + amp * rng.standard_normal(u0.shape)
    s0[3] = ug
    s0[7] = omega
    return p0, u0, s0


def body6(nx=20, ny=16, nz=16, nd=6, centre=(8.3, 8.1, 7.7), mask=DOF_TX | DOF_TY | DOF_TZ | DOF_ROT, wk=W_COS4,
          bc=(BC_INFLOW_OUTFLOW, BC_PERIODIC, BC_PERIODIC), n_itr=2, nt=4, seed=7, nu=0.05, kappa_max=2.0,
          radius=0.0, sphere=False, obj=None, precision=64, scale_inertia=1.0):
    """A freely rotating 3D body (six DOFs) with its own inertia tensor; radius > 0 makes the
    design domain a ball."""
    g = gamma_3d(nd, seed, sphere_mask=sphere)
    M, _ = mass_properties(g, (nd, nd, nd), 3, 0)
    It = tuple(scale_inertia * v for v in inertia_tensor(g, (nd, nd, nd)))
    if obj is None:
        obj = tuple(np.random.default_rng(seed + 100).standard_normal(21))
    P = Problem(dim=3, nx=nx, ny=ny, nz=nz, ndx=nd, ndy=nd, ndz=nd, body_centre=centre, rot_axis=ROT_FREE,
                dof_mask=mask, mass=M, inertia=It[0], nu=nu, u_in=0.05, dp=0.0, bc=bc, kappa_max=kappa_max, q=0.1,
                weight_kind=wk, n_steps=nt, n_itr=n_itr, obj_weights=obj, field_precision=precision,
                inertia_tensor=It, design_radius=radius)
    return P, g


def rotvec_matrix(v):
    """Rotation matrix of the rotation vector v (angle |v| about v), by scipy's Rotation."""
    from scipy.spatial.transform import Rotation
    return Rotation.from_rotvec(np.asarray(v, dtype=float)).as_matrix()


def perturbed_state6(P, seed=1, amp=0.01, ug=(0.01, 0.0, 0.005), rotvec=(0.3, -0.2, 0.5), h=(0.5, -0.3, 0.8),
                     omega=(0.002, 0.003, -0.001)):
    """Impulsive-start state plus seeded noise, with a rotated, moving, spinning free body."""
    p0, u0, s0 = initial_state(P)
    rng = np.random.default_rng(seed)
    p0 = p0 + amp * rng.standard_normal(p0.shape)
    u0 = u0 + amp * rng.standard_normal(u0.shape)
    s0[3:6] = ug
    s0[6:9] = h
    s0[9:12] = omega
    s0[12:21] = rotvec_matrix(rotvec).reshape(-1)
    return p0, u0, s0
