"""Seeded synthetic inputs shaped like the paper's 2D and 3D moving-body problems.

The paper's own geometries (2D sail, 2D/3D turbine, Sec. 4) are given only as figures, so the
workloads here are synthetic stand-ins with the sizes listed in ``config``:

* random numbers come from splitmix64 (Steele, Lea and Flood 2014), doubles from the top 53 bits;
* 2D design fields: gamma ~ U[0,1] i.i.d. on the design grid, then a 3x3 box filter applied twice
  (each pass averages over the in-bounds neighbours);
* 3D design fields: U[0,1] on a coarse lattice of ceil(n/8)+1 points per axis, trilinearly
  interpolated to n^3; rotating 3D bodies are multiplied by the inscribed-sphere mask;
* mass M = 2 * sum(gamma) (unit design-cell volume), inertia I = 2 * sum(gamma * |r_perp|^2),
  both computed once and held constant (Sec. 2.1 states M and I_z are constant).

Array layouts: design fields are flat with x fastest (m = i + ndx*(j + ndy*k)); analysis fields
are flat planes with x fastest, one plane per velocity component.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

# Boundary kinds per axis.
BC_PERIODIC = 0
BC_INFLOW_OUTFLOW = 1
BC_WALL = 2
BC_PRESSURE = 3
# Design-to-analysis weight kernels.
W_COS4 = 0
W_BILINEAR = 1
# Motion degrees of freedom.
DOF_TX = 1
DOF_TY = 2
DOF_TZ = 4
DOF_ROT = 8
# rot_axis value of a freely rotating 3D body (six DOFs)
ROT_FREE = -1
# Checkpoint policies and storage formats.
CKPT_STORE_ALL = 0
CKPT_UNIFORM = 1
CKPT_BINOMIAL = 2
CKPT_FP32 = 0
CKPT_BF16 = 1
CKPT_FP16 = 2

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_uniform(seed: int, n: int) -> np.ndarray:
    """First n outputs of splitmix64 seeded with ``seed``, mapped to doubles in [0, 1)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + _GOLDEN * k
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _box3_2d(g: np.ndarray) -> np.ndarray:
    ny, nx = g.shape
    out = np.empty_like(g)
    for j in range(ny):
        j0, j1 = max(j - 1, 0), min(j + 2, ny)
        for i in range(nx):
            i0, i1 = max(i - 1, 0), min(i + 2, nx)
            out[j, i] = g[j0:j1, i0:i1].mean()
    return out


def gamma_2d(nd: int, seed: int, smooth_passes: int = 2) -> np.ndarray:
    """Design field on an nd x nd grid: U[0,1] i.i.d., then 3x3 box filtered ``smooth_passes`` times."""
    g = splitmix64_uniform(seed, nd * nd).reshape(nd, nd)
    for _ in range(smooth_passes):
        g = _box3_2d(g)
    return np.ascontiguousarray(g.reshape(-1))


def gamma_3d(nd: int, seed: int, sphere_mask: bool = False) -> np.ndarray:
    """Design field on an nd^3 grid: coarse U[0,1] lattice trilinearly refined, optional sphere mask."""
    nc = int(math.ceil(nd / 8)) + 1
    coarse = splitmix64_uniform(seed, nc ** 3).reshape(nc, nc, nc)  # [k][j][i]
    s = np.arange(nd) * (nc - 1) / max(nd - 1, 1)
    i0 = np.minimum(np.floor(s).astype(int), nc - 2)
    fr = s - i0
    # trilinear interpolation, separable along the three axes
    a = coarse[:, :, i0] * (1 - fr) + coarse[:, :, i0 + 1] * fr            # refine x
    a = a[:, i0, :] * (1 - fr)[None, :, None] + a[:, i0 + 1, :] * fr[None, :, None]  # refine y
    a = a[i0, :, :] * (1 - fr)[:, None, None] + a[i0 + 1, :, :] * fr[:, None, None]  # refine z
    if sphere_mask:
        c = (nd - 1) / 2.0
        rad = nd / 2.0 - 2.0
        k, j, i = np.meshgrid(np.arange(nd), np.arange(nd), np.arange(nd), indexing="ij")
        r2 = (i - c) ** 2 + (j - c) ** 2 + (k - c) ** 2
        a = a * (r2 <= rad * rad)
    return np.ascontiguousarray(a.reshape(-1))


def design_offsets(nd: tuple, dim: int) -> np.ndarray:
    """r_m = xi_m - xi^G for every design point, shape [N_D, 3] (pivot at the grid centre)."""
    ndx, ndy, ndz = nd
    k, j, i = np.meshgrid(np.arange(ndz), np.arange(ndy), np.arange(ndx), indexing="ij")
    r = np.stack([i - (ndx - 1) / 2.0, j - (ndy - 1) / 2.0, k - (ndz - 1) / 2.0], axis=-1).reshape(-1, 3)
    if dim == 2:
        r[:, 2] = 0.0
    return r.astype(np.float64)


def inertia_tensor(gamma: np.ndarray, nd: tuple) -> tuple:
    """Body-frame inertia tensor about the pivot, 2 sum(gamma (|r|^2 1 - r r^T)), row-major (9)."""
    r = design_offsets(nd, 3)
    w = 2.0 * gamma
    r2 = (r ** 2).sum(axis=1)
    I = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            I[i, j] = float((w * ((r2 if i == j else 0.0) - r[:, i] * r[:, j])).sum())
    return tuple(I.reshape(-1))


def mass_properties(gamma: np.ndarray, nd: tuple, dim: int, rot_axis: int) -> tuple:
    """M = 2 sum(gamma), I = 2 sum(gamma |r_perp|^2) about ``rot_axis`` (held constant)."""
    r = design_offsets(nd, dim)
    r_perp2 = (r ** 2).sum(axis=1) - r[:, rot_axis] ** 2
    return 2.0 * float(gamma.sum()), 2.0 * float((gamma * r_perp2).sum())


@dataclasses.dataclass
class Problem:
    """Problem statement shared by every consumer (grid, velocity set, body, fluid, run)."""

    dim: int
    nx: int
    ny: int
    nz: int
    ndx: int
    ndy: int
    ndz: int
    body_centre: tuple
    rot_axis: int
    dof_mask: int
    mass: float
    inertia: float
    nu: float
    u_in: float
    dp: float
    bc: tuple                 # (bc_x, bc_y, bc_z)
    kappa_max: float
    q: float
    weight_kind: int
    n_steps: int
    n_itr: int
    obj_weights: tuple        # one weight per DOF: 8 over (xG[3], uG[3], theta, omega), or 21 with free
                              # rotation over (xG[3], uG[3], h[3], omega[3], R[9] row-major)
    field_precision: int = 64  # 32 or 64
    ckpt_policy: int = CKPT_STORE_ALL
    ckpt_every: int = 0
    ckpt_format: int = CKPT_FP32
    name: str = ""
    seed: int = 0
    inertia_tensor: tuple = (0.0,) * 9  # free rotation: body-frame inertia about the pivot
    design_radius: float = 0.0          # > 0: ball-shaped design domain |r_m| <= design_radius
    filter_radius: float = 0.0          # density filter radius (0: no filter)
    proj_beta: float = 0.0              # Heaviside projection steepness (0: no projection)
    proj_eta: float = 0.5               # Heaviside projection threshold
    v_min: float = 0.25                 # minimum volume ratio of the constraint
    cyclic_order: int = 1               # cyclic expansion of the design about the rotation axis: 1, 2, 4
    hbm_budget_bytes: int = 0           # workspace limit (0: none); binomial with ckpt_every 0 fills it

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_design(self) -> int:
        return self.ndx * self.ndy * self.ndz

    @property
    def n_dof(self) -> int:
        return 21 if self.rot_axis == ROT_FREE else 8

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def initial_state(P: Problem, p0: float = 0.0, u0: Optional[tuple] = None) -> tuple:
    """Impulsive start: p = p0, u = (U_in, 0, 0) everywhere, body at rest at its centre."""
    N = P.n_cells
    if u0 is None:
        u0 = (P.u_in, 0.0, 0.0)
    p = np.full(N, p0, dtype=np.float64)
    u = np.zeros((P.dim, N), dtype=np.float64)
    for a in range(P.dim):
        u[a, :] = u0[a]
    dof = np.zeros(P.n_dof, dtype=np.float64)
    dof[0:3] = P.body_centre
    if P.n_dof == 21:
        dof[12:21] = np.eye(3).reshape(-1)  # R = identity
    return p, u, dof


def _nu_from_re(u_in: float, length: float, re: float) -> float:
    return u_in * length / re


def _obj(index: int, n: int = 8) -> tuple:
    w = [0.0] * n
    w[index] = 1.0
    return tuple(w)


# name -> (builder) ; seeds are 20260118 + config index as stated in the workload recipe
def _cfg1(**kw) -> tuple:
    nd, seed = 16, 20260118 + 1
    g = gamma_2d(nd, seed)
    M, I = mass_properties(g, (nd, nd, 1), 2, 2)
    P = Problem(dim=2, nx=80, ny=40, nz=1, ndx=nd, ndy=nd, ndz=1, body_centre=(20.0, 20.0, 0.0),
                rot_axis=2, dof_mask=DOF_TX, mass=M, inertia=I, nu=_nu_from_re(0.05, 16, 100),
                u_in=0.05, dp=0.0, bc=(BC_INFLOW_OUTFLOW, BC_PERIODIC, BC_PERIODIC), kappa_max=1.0,
                q=0.1, weight_kind=W_BILINEAR, n_steps=400, n_itr=5, obj_weights=_obj(0),
                field_precision=64, ckpt_policy=CKPT_STORE_ALL, name="sail2d_80x40_d16", seed=seed)
    return P, g


def _cfg2(**kw) -> tuple:
    nd, seed = 128, 20260118 + 2
    g = gamma_2d(nd, seed)
    M, I = mass_properties(g, (nd, nd, 1), 2, 2)
    P = Problem(dim=2, nx=512, ny=256, nz=1, ndx=nd, ndy=nd, ndz=1, body_centre=(128.0, 128.0, 0.0),
                rot_axis=2, dof_mask=DOF_ROT, mass=M, inertia=I, nu=_nu_from_re(0.05, nd, 200),
                u_in=0.05, dp=0.0, bc=(BC_INFLOW_OUTFLOW, BC_PERIODIC, BC_PERIODIC), kappa_max=1.0,
                q=0.1, weight_kind=W_COS4, n_steps=5000, n_itr=5, obj_weights=_obj(6),
                field_precision=32, ckpt_policy=CKPT_UNIFORM, ckpt_every=100, ckpt_format=CKPT_FP32,
                name="turbine2d_512x256_d128", seed=seed)
    return P, g


def _cfg3(**kw) -> tuple:
    nd, seed = 256, 20260118 + 3
    g = gamma_2d(nd, seed)
    M, I = mass_properties(g, (nd, nd, 1), 2, 2)
    P = Problem(dim=2, nx=1024, ny=512, nz=1, ndx=nd, ndy=nd, ndz=1, body_centre=(256.0, 256.0, 0.0),
                rot_axis=2, dof_mask=DOF_TX | DOF_TY | DOF_ROT, mass=M, inertia=I,
                nu=_nu_from_re(0.05, nd, 500), u_in=0.05, dp=0.0,
                bc=(BC_INFLOW_OUTFLOW, BC_PERIODIC, BC_PERIODIC), kappa_max=1.0, q=0.1,
                weight_kind=W_COS4, n_steps=20000, n_itr=5, obj_weights=_obj(6), field_precision=32,
                ckpt_policy=CKPT_UNIFORM, ckpt_every=100, ckpt_format=CKPT_BF16,
                name="sailturbine2d_1024x512_d256", seed=seed)
    return P, g


def _cfg4(**kw) -> tuple:
    nd, seed = 48, 20260118 + 4
    g = gamma_3d(nd, seed)
    M, I = mass_properties(g, (nd, nd, nd), 3, 2)
    P = Problem(dim=3, nx=128, ny=64, nz=64, ndx=nd, ndy=nd, ndz=nd, body_centre=(32.0, 32.0, 32.0),
                rot_axis=2, dof_mask=DOF_TX | DOF_TY | DOF_TZ, mass=M, inertia=I,
                nu=_nu_from_re(0.05, nd, 100), u_in=0.05, dp=0.0,
                bc=(BC_INFLOW_OUTFLOW, BC_PERIODIC, BC_PERIODIC), kappa_max=1.0, q=0.1,
                weight_kind=W_COS4, n_steps=2000, n_itr=5, obj_weights=_obj(0), field_precision=32,
                ckpt_policy=CKPT_UNIFORM, ckpt_every=100, ckpt_format=CKPT_FP32,
                name="body3d_128x64x64_d48", seed=seed)
    return P, g


def _cfg5(**kw) -> tuple:
    nd, seed = 96, 20260118 + 5
    g = gamma_3d(nd, seed, sphere_mask=True)
    M, _ = mass_properties(g, (nd, nd, nd), 3, 0)
    It = inertia_tensor(g, (nd, nd, nd))
    # six DOFs (free rotation); the design domain is the ball of the sphere mask, radius nd/2 - 2;
    # J = h_x(N_t), the angular momentum about the flow axis. The x axis is periodic (the body is
    # released in a uniform periodic stream): with an inflow/outflow x axis the free body is carried
    # out of the 256-cell channel before step 7000 of the 10000-step march
    P = Problem(dim=3, nx=256, ny=128, nz=128, ndx=nd, ndy=nd, ndz=nd, body_centre=(96.0, 64.0, 64.0),
                rot_axis=ROT_FREE, dof_mask=DOF_TX | DOF_TY | DOF_TZ | DOF_ROT, mass=M, inertia=It[0],
                nu=_nu_from_re(0.05, nd, 300), u_in=0.05, dp=0.0,
                bc=(BC_PERIODIC, BC_PERIODIC, BC_PERIODIC), kappa_max=1.0, q=0.1,
                weight_kind=W_COS4, n_steps=10000, n_itr=5, obj_weights=_obj(6, 21), field_precision=32,
                ckpt_policy=CKPT_BINOMIAL, ckpt_every=0, ckpt_format=CKPT_BF16, hbm_budget_bytes=150 * 10**9,
                name="turbine3d_256x128x128_d96_6dof", seed=seed, inertia_tensor=It,
                design_radius=nd / 2.0 - 2.0)
    return P, g


_CONFIGS = {1: _cfg1, 2: _cfg2, 3: _cfg3, 4: _cfg4, 5: _cfg5}


def verification(kind: str) -> tuple:
    """(Problem, gamma) of the sensitivity checks of Appendix B with the paper's parameters and a
    geometry of our own (the paper draws it only in a figure): a pressure-driven channel of 600x100
    cells (inlet pressure dp, outlet 0, no-slip walls in y) and a 20x20 design grid, FP64, every
    state stored.
      translation: x-translation only, J = x^G_x(N_t); N_t = 3000, nu = 0.1, M = 1e3, dp = 1e-2,
                   kappa_max = 300, q = 1e-2
      rotation:    rotation only, J = theta(N_t); N_t = 10000, nu = 0.1, I = 1e6, dp = 1e-2,
                   kappa_max = 200, q = 1e-2"""
    nd, seed = 20, 20260118 + (11 if kind == "translation" else 12)
    g = gamma_2d(nd, seed)
    common = dict(dim=2, nx=600, ny=100, nz=1, ndx=nd, ndy=nd, ndz=1, rot_axis=2, nu=0.1, u_in=0.0, dp=1e-2,
                  bc=(BC_PRESSURE, BC_WALL, BC_PERIODIC), weight_kind=W_COS4, n_itr=5, field_precision=64,
                  ckpt_policy=CKPT_STORE_ALL, seed=seed)
    if kind == "translation":
        P = Problem(body_centre=(150.0, 50.0, 0.0), dof_mask=DOF_TX, mass=1e3, inertia=1.0, kappa_max=300.0, q=1e-2,
                    n_steps=3000, obj_weights=_obj(0), name="verify_translation_600x100_d20", **common)
    elif kind == "rotation":
        P = Problem(body_centre=(150.0, 50.0, 0.0), dof_mask=DOF_ROT, mass=1.0, inertia=1e6, kappa_max=200.0,
                    q=1e-2, n_steps=10000, obj_weights=_obj(6), name="verify_rotation_600x100_d20", **common)
    else:
        raise ValueError(kind)
    return P, g


def config_names() -> dict:
    return {k: v()[0].name for k, v in _CONFIGS.items() if k <= 2}


def config(index: int) -> tuple:
    """(Problem, gamma) for workload ``index`` (1..5); gamma is float64 [N_D], x fastest."""
    return _CONFIGS[index]()
