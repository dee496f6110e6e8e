"""ctypes wrapper around the oracle library (oracle/lks_oracle.cpp).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg call it. It takes a ``workloads.Problem`` and numpy float64 arrays.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build


class OracleProblem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("ndx", ctypes.c_int), ("ndy", ctypes.c_int), ("ndz", ctypes.c_int),
        ("rot_axis", ctypes.c_int),
        ("dof_mask", ctypes.c_int),
        ("bc", ctypes.c_int * 3),
        ("weight_kind", ctypes.c_int),
        ("n_steps", ctypes.c_int),
        ("n_itr", ctypes.c_int),
        ("mass", ctypes.c_double),
        ("inertia", ctypes.c_double),
        ("nu", ctypes.c_double),
        ("u_in", ctypes.c_double),
        ("dp", ctypes.c_double),
        ("kappa_max", ctypes.c_double),
        ("q", ctypes.c_double),
        ("obj_w", ctypes.c_double * 21),
        ("inertia_tensor", ctypes.c_double * 9),
        ("design_radius", ctypes.c_double),
        ("filter_radius", ctypes.c_double),
        ("proj_beta", ctypes.c_double),
        ("proj_eta", ctypes.c_double),
        ("v_min", ctypes.c_double),
        ("cyclic_order", ctypes.c_int),
    ]


ERRORS = {0: "ok", 1: "bad argument", 2: "body outside the domain", 3: "non-finite state", 4: "unstable (nu <= 0)"}

_lib = None
_libs = {}
_variant = "serial"


def set_variant(name: str) -> bool:
    """Select the build later calls use: "serial" (the oracle), or "openmp" (the timing build: the same
    arithmetic over the host's cores, bitwise the same results). Returns False if that build is absent."""
    global _variant, _lib
    _build.build()
    path = _build.LIB_OMP if name == "openmp" else _build.LIB
    if not os.path.exists(path):
        return False
    _variant = name
    _lib = _libs.get(name)
    return True


def set_alks_outlet_rule(rule: int) -> int:
    """Test hook: plant another outlet rule in the paper-form adjoint (0 restores the reading)."""
    return int(lib().oracle_set_alks_outlet_rule(int(rule)))


def threads() -> int:
    """Threads of the selected build's per-node loops."""
    return int(lib().oracle_threads())


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        if _variant == "openmp":
            path = _build.LIB_OMP
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        pp = ctypes.POINTER(OracleProblem)
        L.oracle_forward.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp, dp]
        L.oracle_gradient.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
        L.oracle_forward_cs.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp, dp, ctypes.c_double, dp, dp]
        L.oracle_stencil.argtypes = [pp, dp, dp, dp, dp]
        L.oracle_stencil_jvp.argtypes = [pp, dp, dp, dp, dp, ctypes.c_double, dp, dp]
        L.oracle_stencil_vjp.argtypes = [pp, dp, dp, dp, dp, dp, dp]
        L.oracle_step.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp, dp]
        L.oracle_spread.argtypes = [pp, dp, dp, dp, dp, ip]
        L.oracle_interp.argtypes = [pp, dp, dp, dp]
        L.oracle_support_sets.argtypes = [pp, dp, ctypes.c_void_p]
        L.oracle_weight.argtypes = [ctypes.c_int, ctypes.c_double, dp]
        L.oracle_weight.restype = ctypes.c_double
        L.oracle_lattice.argtypes = [ctypes.c_int, ip, dp]
        L.oracle_dof_count.argtypes = [pp]
        L.oracle_design_chain.argtypes = [pp, dp, dp]
        L.oracle_design_chain_vjp.argtypes = [pp, dp, dp, dp]
        L.oracle_design_chain_jvp.argtypes = [pp, dp, dp, ctypes.c_double, dp]
        L.oracle_constraint.argtypes = [pp, dp, dp, dp]
        L.oracle_gradient_terminal.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
        L.oracle_forward_cs_terminal.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp, dp, ctypes.c_double, dp]
        L.oracle_gradient_alks.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
        L.oracle_alks_feq.argtypes = [pp, dp, dp, dp, dp, dp]
        L.oracle_feq_adjoint_cs.argtypes = [pp, dp, dp, dp, ctypes.c_double, dp]
        L.oracle_alks_gather.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp]
        L.oracle_alks_parts.argtypes = [pp, dp, dp, dp, dp, dp, ctypes.c_double, dp, dp, dp]
        L.oracle_alks_lambda_cs.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp, dp, ctypes.c_double, ctypes.c_double, dp]
        L.oracle_alks_body_step.argtypes = [pp, dp, dp, dp, dp, dp, ctypes.c_int, dp, dp, dp]
        L.oracle_threads.argtypes = []
        L.oracle_set_alks_outlet_rule.argtypes = [ctypes.c_int]
        if L.oracle_sizeof_problem() != ctypes.sizeof(OracleProblem):
            raise RuntimeError("oracle problem record layout mismatch")
        _lib = L
        _libs[_variant] = L
    return _lib


class OracleError(RuntimeError):
    pass


def _check(rc: int):
    if rc != 0:
        raise OracleError(f"oracle error {rc}: {ERRORS.get(rc, '?')}")


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def problem_record(P, n_steps: Optional[int] = None) -> OracleProblem:
    r = OracleProblem()
    r.dim = P.dim
    r.nx, r.ny, r.nz = P.nx, P.ny, P.nz
    r.ndx, r.ndy, r.ndz = P.ndx, P.ndy, P.ndz
    r.rot_axis = P.rot_axis
    r.dof_mask = P.dof_mask
    for a in range(3):
        r.bc[a] = P.bc[a]
    r.weight_kind = P.weight_kind
    r.n_steps = P.n_steps if n_steps is None else n_steps
    r.n_itr = P.n_itr
    r.mass, r.inertia, r.nu, r.u_in, r.dp = P.mass, P.inertia, P.nu, P.u_in, P.dp
    r.kappa_max, r.q = P.kappa_max, P.q
    for a in range(len(P.obj_weights)):
        r.obj_w[a] = P.obj_weights[a]
    for a in range(9):
        r.inertia_tensor[a] = P.inertia_tensor[a]
    r.design_radius = P.design_radius
    r.filter_radius = P.filter_radius
    r.proj_beta, r.proj_eta = P.proj_beta, P.proj_eta
    r.v_min = P.v_min
    r.cyclic_order = P.cyclic_order
    return r


def dof_count(P) -> int:
    """Length of the DOF vector: 8 for a single rotation axis, 21 for free rotation."""
    n = lib().oracle_dof_count(ctypes.byref(problem_record(P)))
    if n <= 0:
        raise OracleError("invalid problem")
    return n


def forward(P, gamma, p0, u0, dof0, n_steps: Optional[int] = None, check: bool = True):
    """Forward march. Returns (p, u [dim, N], dof history [(n_steps+1), ns], J)."""
    rec = problem_record(P, n_steps)
    N = P.n_cells
    p = np.zeros(N)
    u = np.zeros((P.dim, N))
    hist = np.zeros((rec.n_steps + 1, dof_count(P)))
    J = ctypes.c_double(0.0)
    rc = lib().oracle_forward(ctypes.byref(rec), _ptr(_f64(gamma)), _ptr(_f64(p0)), _ptr(_f64(u0)), _ptr(_f64(dof0)),
                              _ptr(p), _ptr(u), _ptr(hist), ctypes.byref(J))
    if check:
        _check(rc)
    return p, u, hist, J.value


def gradient(P, gamma, p0, u0, dof0, n_steps: Optional[int] = None):
    """Forward + exact discrete adjoint. Returns dict with J, dJdgamma, dJdkref, lam_p0, lam_u0, lam_dof0."""
    rec = problem_record(P, n_steps)
    N, ND = P.n_cells, P.n_design
    out = {"dJdgamma": np.zeros(ND), "dJdkref": np.zeros(ND), "lam_p0": np.zeros(N),
           "lam_u0": np.zeros((P.dim, N)), "lam_dof0": np.zeros(dof_count(P))}
    J = ctypes.c_double(0.0)
    rc = lib().oracle_gradient(ctypes.byref(rec), _ptr(_f64(gamma)), _ptr(_f64(p0)), _ptr(_f64(u0)), _ptr(_f64(dof0)),
                               ctypes.byref(J), _ptr(out["dJdgamma"]), _ptr(out["lam_p0"]), _ptr(out["lam_u0"]),
                               _ptr(out["lam_dof0"]), _ptr(out["dJdkref"]))
    _check(rc)
    out["J"] = J.value
    return out


def forward_cs(P, gamma, p0, u0, dof0, dgamma=None, dp0=None, du0=None, ddof0=None, h: float = 1e-30,
               n_steps: Optional[int] = None):
    """Complex-step directional derivative of J. Returns (J, dJ)."""
    rec = problem_record(P, n_steps)
    J = ctypes.c_double(0.0)
    dJ = ctypes.c_double(0.0)
    rc = lib().oracle_forward_cs(ctypes.byref(rec), _ptr(_f64(gamma)), _ptr(None if dgamma is None else _f64(dgamma)),
                                 _ptr(_f64(p0)), _ptr(None if dp0 is None else _f64(dp0)), _ptr(_f64(u0)),
                                 _ptr(None if du0 is None else _f64(du0)), _ptr(_f64(dof0)),
                                 _ptr(None if ddof0 is None else _f64(ddof0)), h, ctypes.byref(J), ctypes.byref(dJ))
    _check(rc)
    return J.value, dJ.value


def stencil(P, p, u):
    rec = problem_record(P)
    ps = np.zeros(P.n_cells)
    us = np.zeros((P.dim, P.n_cells))
    _check(lib().oracle_stencil(ctypes.byref(rec), _ptr(_f64(p)), _ptr(_f64(u)), _ptr(ps), _ptr(us)))
    return ps, us


def stencil_jvp(P, p, u, dp, du, h: float = 1e-30):
    rec = problem_record(P)
    dps = np.zeros(P.n_cells)
    dus = np.zeros((P.dim, P.n_cells))
    _check(lib().oracle_stencil_jvp(ctypes.byref(rec), _ptr(_f64(p)), _ptr(_f64(dp)), _ptr(_f64(u)), _ptr(_f64(du)), h,
                                    _ptr(dps), _ptr(dus)))
    return dps, dus


def stencil_vjp(P, p, u, lps, lus):
    rec = problem_record(P)
    lp = np.zeros(P.n_cells)
    lu = np.zeros((P.dim, P.n_cells))
    _check(lib().oracle_stencil_vjp(ctypes.byref(rec), _ptr(_f64(p)), _ptr(_f64(u)), _ptr(_f64(lps)), _ptr(_f64(lus)),
                                    _ptr(lp), _ptr(lu)))
    return lp, lu


def step(P, gamma, p, u, s):
    """One forward step. Returns (p, u, s_next, iterates [(n_itr+1), ns])."""
    rec = problem_record(P)
    ns = dof_count(P)
    po = np.zeros(P.n_cells)
    uo = np.zeros((P.dim, P.n_cells))
    so = np.zeros(ns)
    it = np.zeros((P.n_itr + 1, ns))
    _check(lib().oracle_step(ctypes.byref(rec), _ptr(_f64(gamma)), _ptr(_f64(p)), _ptr(_f64(u)), _ptr(_f64(s)),
                             _ptr(po), _ptr(uo), _ptr(so), _ptr(it)))
    return po, uo, so, it


def spread(P, gamma, s):
    """Returns (kappa [N], u^S [dim, N], count [N] of design points with non-zero weight)."""
    rec = problem_record(P)
    k = np.zeros(P.n_cells)
    us = np.zeros((P.dim, P.n_cells))
    cnt = np.zeros(P.n_cells, dtype=np.int32)
    rc = lib().oracle_spread(ctypes.byref(rec), _ptr(_f64(gamma)), _ptr(_f64(s)), _ptr(k), _ptr(us),
                             cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    _check(rc)
    return k, us, cnt


def support_sets(P, s):
    """Per analysis node, the design points whose support window holds it under the DOF vector s:
    int64 [N, 5] = (count, least index or -1, largest index, sum of indices, sum of squares)."""
    rec = problem_record(P)
    out = np.zeros((P.n_cells, 5), dtype=np.int64)
    _check(lib().oracle_support_sets(ctypes.byref(rec), _ptr(_f64(s)), out.ctypes.data))
    return out


def interp(P, s, u):
    rec = problem_record(P)
    uref = np.zeros((P.n_design, 3))
    _check(lib().oracle_interp(ctypes.byref(rec), _ptr(_f64(s)), _ptr(_f64(u)), _ptr(uref)))
    return uref


def weight(kind: int, r: float):
    dw = ctypes.c_double(0.0)
    w = lib().oracle_weight(kind, r, ctypes.byref(dw))
    return w, dw.value


def lattice(dim: int):
    """(c [Q,3] int, w [Q]) of the oracle's velocity set."""
    c = np.zeros((15, 3), dtype=np.int32)
    w = np.zeros(15)
    Q = lib().oracle_lattice(dim, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(w))
    return c[:Q].copy(), w[:Q].copy()


def design_chain(P, gamma):
    """gamma-bar [N_D]: cyclic expansion, density filter and Heaviside projection of gamma."""
    out = np.zeros(P.n_design)
    _check(lib().oracle_design_chain(ctypes.byref(problem_record(P)), _ptr(_f64(gamma)), _ptr(out)))
    return out


def design_chain_vjp(P, gamma, v):
    """(d gamma-bar / d gamma)^T v at gamma."""
    out = np.zeros(P.n_design)
    _check(lib().oracle_design_chain_vjp(ctypes.byref(problem_record(P)), _ptr(_f64(gamma)), _ptr(_f64(v)),
                                         _ptr(out)))
    return out


def design_chain_jvp(P, gamma, v, h: float = 1e-30):
    """Complex-step (d gamma-bar / d gamma) v at gamma."""
    out = np.zeros(P.n_design)
    _check(lib().oracle_design_chain_jvp(ctypes.byref(problem_record(P)), _ptr(_f64(gamma)), _ptr(_f64(v)), h,
                                         _ptr(out)))
    return out


def constraint(P, gamma):
    """(G, dG/dgamma) of the volume constraint on gamma-bar."""
    G = ctypes.c_double(0.0)
    d = np.zeros(P.n_design)
    _check(lib().oracle_constraint(ctypes.byref(problem_record(P)), _ptr(_f64(gamma)), ctypes.byref(G), _ptr(d)))
    return G.value, d


def gradient_terminal(P, gamma, p0, u0, dof0, lam_pT, lam_uT, lam_sT, n_steps: Optional[int] = None):
    """Forward + exact adjoint started from a terminal adjoint (the periodic warm start of Sec. 3.4):
    the derivative of J + lam_pT.p(N_t) + lam_uT.u(N_t) + lam_sT.s(N_t)."""
    rec = problem_record(P, n_steps)
    N, ND = P.n_cells, P.n_design
    out = {"dJdgamma": np.zeros(ND), "dJdkref": np.zeros(ND), "lam_p0": np.zeros(N),
           "lam_u0": np.zeros((P.dim, N)), "lam_dof0": np.zeros(dof_count(P))}
    J = ctypes.c_double(0.0)
    rc = lib().oracle_gradient_terminal(ctypes.byref(rec), _ptr(_f64(gamma)), _ptr(_f64(p0)), _ptr(_f64(u0)),
                                        _ptr(_f64(dof0)), _ptr(_f64(lam_pT)), _ptr(_f64(lam_uT)), _ptr(_f64(lam_sT)),
                                        ctypes.byref(J), _ptr(out["dJdgamma"]), _ptr(out["lam_p0"]),
                                        _ptr(out["lam_u0"]), _ptr(out["lam_dof0"]), _ptr(out["dJdkref"]))
    _check(rc)
    out["J"] = J.value
    return out


def forward_cs_terminal(P, gamma, p0, u0, dof0, lam_pT, lam_uT, lam_sT, dgamma, h: float = 1e-30):
    """Complex-step derivative along dgamma of J + lam_pT.p(N_t) + lam_uT.u(N_t) + lam_sT.s(N_t)."""
    dJ = ctypes.c_double(0.0)
    _check(lib().oracle_forward_cs_terminal(ctypes.byref(problem_record(P)), _ptr(_f64(gamma)), _ptr(_f64(dgamma)),
                                            _ptr(_f64(p0)), _ptr(_f64(u0)), _ptr(_f64(dof0)), _ptr(_f64(lam_pT)),
                                            _ptr(_f64(lam_uT)), _ptr(_f64(lam_sT)), h, ctypes.byref(dJ)))
    return dJ.value


# ---- the paper's adjoint (ALKS, Sec. 2.5) ----------------------------------------------------
# Moments: p~ [N], u~ [dim, N], s~ [dim, dim, N]. Body multipliers: 8 values in the DOF-vector
# order (x~G[3], u~G[3], theta~, omega~), the paper's sign (minus the derivatives of J).


def gradient_alks(P, gamma, p0, u0, dof0, n_steps: Optional[int] = None):
    """Forward + the paper's adjoint: J, dJdgamma, dJdkref, the moments at t = 0 (adj_p0, adj_u0,
    adj_s0) and the body multipliers at t = 1 (body1)."""
    rec = problem_record(P, n_steps)
    N, ND, d = P.n_cells, P.n_design, P.dim
    out = {"dJdgamma": np.zeros(ND), "dJdkref": np.zeros(ND), "adj_p0": np.zeros(N), "adj_u0": np.zeros((d, N)),
           "adj_s0": np.zeros((d, d, N)), "body1": np.zeros(8)}
    J = ctypes.c_double(0.0)
    _check(lib().oracle_gradient_alks(ctypes.byref(rec), _ptr(_f64(gamma)), _ptr(_f64(p0)), _ptr(_f64(u0)),
                                      _ptr(_f64(dof0)), ctypes.byref(J), _ptr(out["dJdgamma"]), _ptr(out["dJdkref"]),
                                      _ptr(out["adj_p0"]), _ptr(out["adj_u0"]), _ptr(out["adj_s0"]),
                                      _ptr(out["body1"])))
    out["J"] = J.value
    return out


def alks_feq(P, ap, au, as_, u):
    """The adjoint equilibrium f~eq [Q, N] of the moments at the velocity u."""
    Q = 9 if P.dim == 2 else 15
    F = np.zeros((Q, P.n_cells))
    _check(lib().oracle_alks_feq(ctypes.byref(problem_record(P)), _ptr(_f64(ap)), _ptr(_f64(au)), _ptr(_f64(as_)),
                                 _ptr(_f64(u)), _ptr(F)))
    return F


def feq_adjoint_cs(P, f, df, phi, h: float = 1e-30):
    """d/dh of sum phi_j f^eq_j(moments of f + i h df) / h: the forward equilibrium's derivative."""
    out = ctypes.c_double(0.0)
    _check(lib().oracle_feq_adjoint_cs(ctypes.byref(problem_record(P)), _ptr(_f64(f)), _ptr(_f64(df)),
                                       _ptr(_f64(phi)), h, ctypes.byref(out)))
    return out.value


def alks_gather(P, ap, au, as_, u):
    """Star moments at t - 1 from the moments at t and the velocity u(t), boundary values included."""
    N, d = P.n_cells, P.dim
    op, ou, os_ = np.zeros(N), np.zeros((d, N)), np.zeros((d, d, N))
    _check(lib().oracle_alks_gather(ctypes.byref(problem_record(P)), _ptr(_f64(ap)), _ptr(_f64(au)),
                                    _ptr(_f64(as_)), _ptr(_f64(u)), _ptr(op), _ptr(ou), _ptr(os_)))
    return op, ou, os_


def alks_parts(P, gamma, s, u, ustar, ug, om):
    """Eq. au's fluid multiplier, the coupling terms (X[3], U[3], Th, Om) and the step's design
    sensitivity term, at the DOFs s [8], velocity u, star moment ustar, multipliers ug [3], om."""
    ut = np.zeros((P.dim, P.n_cells))
    terms = np.zeros(8)
    sens = np.zeros(P.n_design)
    _check(lib().oracle_alks_parts(ctypes.byref(problem_record(P)), _ptr(_f64(gamma)), _ptr(_f64(s)), _ptr(_f64(u)),
                                   _ptr(_f64(ustar)), _ptr(_f64(ug)), float(om), _ptr(ut), _ptr(terms), _ptr(sens)))
    return ut, terms, sens


def alks_lambda_cs(P, gamma, s, u, ut, ug, om, dkref=None, ds=None, du=None, h: float = 1e-30):
    """Complex-step derivative of the step Lagrangian along (dkref, ds, du), multipliers fixed."""
    out = ctypes.c_double(0.0)
    _check(lib().oracle_alks_lambda_cs(ctypes.byref(problem_record(P)), _ptr(_f64(gamma)),
                                       _ptr(None if dkref is None else _f64(dkref)), _ptr(_f64(s)),
                                       _ptr(None if ds is None else _f64(ds)), _ptr(_f64(u)),
                                       _ptr(None if du is None else _f64(du)), _ptr(_f64(ut)), _ptr(_f64(ug)),
                                       float(om), h, ctypes.byref(out)))
    return out.value


def alks_body_step(P, gamma, s, u, ustar, nxt, K: int):
    """One step of the paper's adjoint with K fixed-point iterations: (u~ [dim, N], body [8], sens)."""
    ut = np.zeros((P.dim, P.n_cells))
    b = np.zeros(8)
    sens = np.zeros(P.n_design)
    _check(lib().oracle_alks_body_step(ctypes.byref(problem_record(P)), _ptr(_f64(gamma)), _ptr(_f64(s)),
                                       _ptr(_f64(u)), _ptr(_f64(ustar)), _ptr(_f64(nxt)), int(K), _ptr(ut), _ptr(b),
                                       _ptr(sens)))
    return ut, b, sens
