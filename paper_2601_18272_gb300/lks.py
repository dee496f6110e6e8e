"""ctypes binding of the C ABI in include/lks.h (argument marshalling only).

Every step of the forward march, adjoint sweep and sensitivity runs in the CUDA library
``lib/liblks_gb300.so``; this module only converts arguments. If the library cannot be built or
loaded, every call raises: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

LKS_OK = 0
LKS_D2Q9, LKS_D3Q15 = 9, 15
LKS_FP32, LKS_FP64 = 32, 64
LKS_CKPT_STORE_ALL, LKS_CKPT_UNIFORM, LKS_CKPT_BINOMIAL = 0, 1, 2
LKS_CKPT_NATIVE, LKS_CKPT_BF16, LKS_CKPT_FP16 = 0, 1, 2
LKS_BIN_FWD_SNAPSHOT, LKS_BIN_RESTORE, LKS_BIN_ADVANCE, LKS_BIN_STORE, LKS_BIN_REVERSE = 0, 1, 2, 3, 4
LKS_ROT_FREE = -1
LKS_NDOF_AXIS, LKS_NDOF_FREE, LKS_MAX_DOF = 8, 21, 21
STATUS = {0: "LKS_OK", 1: "LKS_ERR_ARG", 2: "LKS_ERR_OOM", 3: "LKS_ERR_BUDGET", 4: "LKS_ERR_UNSTABLE",
          5: "LKS_ERR_BODY_OUTSIDE", 6: "LKS_ERR_NONFINITE", 7: "LKS_ERR_ORDER", 8: "LKS_ERR_CUDA",
          9: "LKS_ERR_UNSUPPORTED", 10: "LKS_ERR_TIMEOUT"}


class lks_problem(ctypes.Structure):  # noqa: N801  (mirrors the C struct name)
    _fields_ = [
        ("dim", ctypes.c_int),
        ("velocity_set", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("ndx", ctypes.c_int), ("ndy", ctypes.c_int), ("ndz", ctypes.c_int),
        ("body_centre", ctypes.c_double * 3),
        ("rot_axis", ctypes.c_int),
        ("dof_mask", ctypes.c_uint),
        ("mass", ctypes.c_double),
        ("inertia", ctypes.c_double),
        ("inertia_tensor", ctypes.c_double * 9),
        ("design_radius", ctypes.c_double),
        ("filter_radius", ctypes.c_double),
        ("proj_beta", ctypes.c_double),
        ("proj_eta", ctypes.c_double),
        ("v_min", ctypes.c_double),
        ("cyclic_order", ctypes.c_int),
        ("nu", ctypes.c_double),
        ("u_in", ctypes.c_double),
        ("dp", ctypes.c_double),
        ("bc", ctypes.c_int * 3),
        ("kappa_max", ctypes.c_double),
        ("q", ctypes.c_double),
        ("weight_kind", ctypes.c_int),
        ("n_steps", ctypes.c_int),
        ("n_itr", ctypes.c_int),
        ("obj_weights", ctypes.c_double * LKS_MAX_DOF),
        ("field_precision", ctypes.c_int),
        ("ckpt_policy", ctypes.c_int),
        ("ckpt_every", ctypes.c_int),
        ("ckpt_format", ctypes.c_int),
        ("hbm_budget_bytes", ctypes.c_size_t),
    ]


class LksError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        detail = ""
        if code == 8 and _lib is not None:
            detail = f" (cudaError {_lib.lks_last_cuda_error()})"
        super().__init__(f"{where}: {STATUS.get(code, code)}{detail}")


_lib = None


def library_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load (building first if needed) the CUDA library. Raises if it cannot be built or loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    L = ctypes.CDLL(path)
    vp, dp, sz = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t
    hp = ctypes.c_void_p
    L.lks_create.argtypes = [ctypes.POINTER(lks_problem), ctypes.POINTER(ctypes.c_void_p)]
    L.lks_set_initial_state.argtypes = [hp, dp, dp, dp]
    L.lks_forward.argtypes = [hp, vp, dp, vp]
    L.lks_adjoint.argtypes = [hp, ctypes.c_double, vp]
    L.lks_sensitivity.argtypes = [hp, vp, vp]
    L.lks_gradient_host.argtypes = [hp, dp, dp, dp, vp]
    L.lks_get_dof_history.argtypes = [hp, dp, sz]
    L.lks_get_state.argtypes = [hp, dp, dp]
    L.lks_get_initial_adjoint.argtypes = [hp, dp, dp, dp]
    L.lks_adjoint_alks.argtypes = [hp, ctypes.c_double, vp]
    L.lks_set_continuation.argtypes = [hp, ctypes.c_double, ctypes.c_double]
    L.lks_get_alks_adjoint.argtypes = [hp, dp, dp, dp, dp]
    L.lks_launch_count.argtypes = [hp]
    L.lks_launch_count.restype = ctypes.c_longlong
    L.lks_set_kernel_timing.argtypes = [hp, ctypes.c_int]
    L.lks_kernel_time.argtypes = [hp, ctypes.c_char_p, dp, ctypes.POINTER(ctypes.c_longlong)]
    L.lks_workspace_bytes.argtypes = [hp]
    L.lks_workspace_bytes.restype = ctypes.c_size_t
    L.lks_destroy.argtypes = [hp]
    L.lks_destroy.restype = None
    L.lks_status_string.argtypes = [ctypes.c_int]
    L.lks_status_string.restype = ctypes.c_char_p
    L.lks_last_cuda_error.argtypes = []
    L.lks_step_noalloc.argtypes = [ctypes.POINTER(lks_problem), vp, vp, ctypes.c_int, dp, vp]
    L.lks_dof_count.argtypes = [ctypes.POINTER(lks_problem)]
    L.lks_support_sets.argtypes = [hp, dp, vp, vp, sz]
    L.lks_debug_sync_skip.argtypes = [hp, ctypes.c_int]
    L.lks_debug_copy_skip.argtypes = [hp, ctypes.c_int]
    L.lks_persistent_coupling.argtypes = [hp, ctypes.c_int]
    L.lks_checkpoint_slots.argtypes = [hp]
    L.lks_stencil_form.argtypes = [hp]
    L.lks_constraint.argtypes = [hp, vp, dp, vp, vp]
    L.lks_warm_start.argtypes = [hp, ctypes.c_int, vp]
    L.lks_binomial_plan.argtypes = [ctypes.c_int, ctypes.c_int, vp, ctypes.c_longlong]
    L.lks_binomial_plan.restype = ctypes.c_longlong
    L.lks_problem_size.argtypes = []
    L.lks_problem_size.restype = ctypes.c_size_t
    if L.lks_problem_size() != ctypes.sizeof(lks_problem):
        raise RuntimeError("lks_problem layout of the binding does not match the library")
    _lib = L
    return L


def _check(code: int, where: str):
    if code != LKS_OK:
        raise LksError(code, where)


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    if a.dtype != np.float64 or not a.flags.c_contiguous:
        raise TypeError("host arrays passed to the library must be contiguous float64")
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def check_design_tensor(t, n_design: int, name: str = "gamma"):
    """Raise unless t is a contiguous float64 CUDA tensor of n_design values: the library reads or
    writes exactly that many doubles at its address."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if t.numel() != n_design:
        raise ValueError(f"{name}: {t.numel()} values, expected {n_design}")


def problem_struct(P, precision: Optional[int] = None, ckpt_policy: Optional[int] = None,
                   ckpt_every: Optional[int] = None, ckpt_format: Optional[int] = None,
                   n_steps: Optional[int] = None, hbm_budget_bytes: Optional[int] = None) -> lks_problem:
    """lks_problem from a ``workloads.Problem`` (optionally overriding the run controls)."""
    s = lks_problem()
    s.dim = P.dim
    s.velocity_set = LKS_D2Q9 if P.dim == 2 else LKS_D3Q15
    s.nx, s.ny, s.nz = P.nx, P.ny, P.nz
    s.ndx, s.ndy, s.ndz = P.ndx, P.ndy, P.ndz
    for a in range(3):
        s.body_centre[a] = P.body_centre[a]
        s.bc[a] = P.bc[a]
    s.rot_axis = P.rot_axis
    s.dof_mask = P.dof_mask
    s.mass, s.inertia, s.nu, s.u_in, s.dp = P.mass, P.inertia, P.nu, P.u_in, P.dp
    for a in range(9):
        s.inertia_tensor[a] = P.inertia_tensor[a]
    s.design_radius = P.design_radius
    s.filter_radius = P.filter_radius
    s.proj_beta, s.proj_eta = P.proj_beta, P.proj_eta
    s.v_min = P.v_min
    s.cyclic_order = P.cyclic_order
    s.kappa_max, s.q = P.kappa_max, P.q
    s.weight_kind = P.weight_kind
    s.n_steps = P.n_steps if n_steps is None else n_steps
    s.n_itr = P.n_itr
    for a in range(len(P.obj_weights)):
        s.obj_weights[a] = P.obj_weights[a]
    s.field_precision = P.field_precision if precision is None else precision
    s.ckpt_policy = P.ckpt_policy if ckpt_policy is None else ckpt_policy
    s.ckpt_every = P.ckpt_every if ckpt_every is None else ckpt_every
    s.ckpt_format = P.ckpt_format if ckpt_format is None else ckpt_format
    if s.ckpt_format != LKS_CKPT_NATIVE and s.field_precision == LKS_FP64:
        s.ckpt_format = LKS_CKPT_NATIVE
    s.hbm_budget_bytes = int(getattr(P, "hbm_budget_bytes", 0) if hbm_budget_bytes is None else hbm_budget_bytes)
    return s


# ---- the C ABI, one Python function per entry point --------------------------------------
def lks_create(problem: lks_problem) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().lks_create(ctypes.byref(problem), ctypes.byref(h)), "lks_create")
    return h


def lks_set_initial_state(h, p: Optional[np.ndarray] = None, u: Optional[np.ndarray] = None,
                          s: Optional[np.ndarray] = None):
    conv = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
    p, u, s = conv(p), conv(u), conv(s)
    _check(load().lks_set_initial_state(h, _dptr(p), _dptr(u), _dptr(s)), "lks_set_initial_state")


def check_initial_state(n_cells: int, dim: int, n_dof: int, p=None, u=None, s=None):
    """Raise ValueError unless each given array holds exactly the values lks_set_initial_state
    reads: p [N], u [dim][N], s [n_dof] (the library reads that many, whatever the array holds)."""
    for name, a, n in (("p", p, n_cells), ("u", u, dim * n_cells), ("s", s, n_dof)):
        if a is not None and np.size(a) != n:
            raise ValueError(f"initial state {name}: {np.size(a)} values, expected {n}")


def lks_forward(h, gamma_dev_ptr: int, stream: int = 0) -> float:
    J = ctypes.c_double(0.0)
    _check(load().lks_forward(h, ctypes.c_void_p(gamma_dev_ptr), ctypes.byref(J), ctypes.c_void_p(stream)),
           "lks_forward")
    return J.value


def lks_adjoint(h, seed: float = 1.0, stream: int = 0):
    _check(load().lks_adjoint(h, float(seed), ctypes.c_void_p(stream)), "lks_adjoint")


def lks_set_continuation(h, q: float, proj_beta: float):
    _check(load().lks_set_continuation(h, float(q), float(proj_beta)), "lks_set_continuation")


def lks_adjoint_alks(h, seed: float = 1.0, stream: int = 0):
    _check(load().lks_adjoint_alks(h, float(seed), ctypes.c_void_p(stream)), "lks_adjoint_alks")


def lks_get_alks_adjoint(h, n_cells: int, dim: int):
    p = np.zeros(n_cells)
    u = np.zeros((dim, n_cells))
    s = np.zeros((dim, dim, n_cells))
    body = np.zeros(8)
    _check(load().lks_get_alks_adjoint(h, _dptr(p), _dptr(u), _dptr(s), _dptr(body)), "lks_get_alks_adjoint")
    return p, u, s, body


def lks_sensitivity(h, out_dev_ptr: int, stream: int = 0):
    _check(load().lks_sensitivity(h, ctypes.c_void_p(out_dev_ptr), ctypes.c_void_p(stream)), "lks_sensitivity")


def lks_gradient_host(h, gamma: np.ndarray, out: np.ndarray, stream: int = 0) -> float:
    J = ctypes.c_double(0.0)
    _check(load().lks_gradient_host(h, _dptr(gamma), ctypes.byref(J), _dptr(out), ctypes.c_void_p(stream)),
           "lks_gradient_host")
    return J.value


def lks_constraint(h, gamma_dev_ptr: int, dG_dev_ptr: int = 0, stream: int = 0) -> float:
    G = ctypes.c_double(0.0)
    _check(load().lks_constraint(h, ctypes.c_void_p(gamma_dev_ptr), ctypes.byref(G),
                                 ctypes.c_void_p(dG_dev_ptr) if dG_dev_ptr else None, ctypes.c_void_p(stream)),
           "lks_constraint")
    return G.value


def lks_warm_start(h, with_adjoint: bool = True, stream: int = 0):
    _check(load().lks_warm_start(h, int(bool(with_adjoint)), ctypes.c_void_p(stream)), "lks_warm_start")


def lks_binomial_plan(n_steps: int, snapshots: int) -> np.ndarray:
    """The binomial checkpoint schedule as rows (kind, a, b, c), kinds LKS_BIN_* (host only)."""
    L = load()
    n = L.lks_binomial_plan(int(n_steps), int(snapshots), None, 0)
    if n < 0:
        raise LksError(int(-n), "lks_binomial_plan")
    ops = np.zeros((n, 4), dtype=np.int32)
    if n:
        L.lks_binomial_plan(int(n_steps), int(snapshots), ops.ctypes.data, n)
    return ops


def lks_dof_count(problem: lks_problem) -> int:
    return int(load().lks_dof_count(ctypes.byref(problem)))


def lks_get_dof_history(h, n_steps: int, n_dof: int = LKS_NDOF_AXIS) -> np.ndarray:
    buf = np.zeros((n_steps + 1, n_dof))
    _check(load().lks_get_dof_history(h, _dptr(buf), buf.size), "lks_get_dof_history")
    return buf


def lks_get_state(h, n_cells: int, dim: int):
    p = np.zeros(n_cells)
    u = np.zeros((dim, n_cells))
    _check(load().lks_get_state(h, _dptr(p), _dptr(u)), "lks_get_state")
    return p, u


def lks_get_initial_adjoint(h, n_cells: int, dim: int, n_dof: int = LKS_NDOF_AXIS):
    lp = np.zeros(n_cells)
    lu = np.zeros((dim, n_cells))
    ls = np.zeros(n_dof)
    _check(load().lks_get_initial_adjoint(h, _dptr(lp), _dptr(lu), _dptr(ls)), "lks_get_initial_adjoint")
    return lp, lu, ls


def lks_launch_count(h) -> int:
    return int(load().lks_launch_count(h))


def lks_set_kernel_timing(h, enable: bool):
    _check(load().lks_set_kernel_timing(h, int(bool(enable))), "lks_set_kernel_timing")


def lks_kernel_time(h, family: str):
    ms = ctypes.c_double(0.0)
    n = ctypes.c_longlong(0)
    _check(load().lks_kernel_time(h, family.encode(), ctypes.byref(ms), ctypes.byref(n)), "lks_kernel_time")
    return ms.value, n.value


def lks_workspace_bytes(h) -> int:
    return int(load().lks_workspace_bytes(h))


def lks_checkpoint_slots(h) -> int:
    r = int(load().lks_checkpoint_slots(h))
    if r < 0:
        raise LksError(-r, "lks_checkpoint_slots")
    return r


def lks_stencil_form(h) -> int:
    r = int(load().lks_stencil_form(h))
    if r < 0:
        raise LksError(-r, "lks_stencil_form")
    return r


def lks_destroy(h):
    if h:
        load().lks_destroy(h)


def lks_step_noalloc(problem: lks_problem, gamma_dev_ptr: int, state_dev_ptr: int, t: int, s: np.ndarray,
                     stream: int = 0) -> np.ndarray:
    """One time step without device allocation; s (8 doubles) is s(t-1) in and s(t) out."""
    s = np.ascontiguousarray(s, dtype=np.float64).copy()
    _check(load().lks_step_noalloc(ctypes.byref(problem), ctypes.c_void_p(gamma_dev_ptr),
                                   ctypes.c_void_p(state_dev_ptr), int(t), _dptr(s), ctypes.c_void_p(stream)),
           "lks_step_noalloc")
    return s


def lks_support_sets(h, s: np.ndarray):
    """Test export: (box origin [3], box extent [3], int64 stats [box cells, 5]) of the design points
    the coupling's gather accepts for each box cell under the DOF vector s."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    box = np.zeros(6, dtype=np.int32)
    L = load()
    _check(L.lks_support_sets(h, _dptr(s), box.ctypes.data, None, 0), "lks_support_sets")
    n = int(np.prod(box[3:]))
    stats = np.zeros((n, 5), dtype=np.int64)
    _check(L.lks_support_sets(h, _dptr(s), box.ctypes.data, stats.ctypes.data, stats.size), "lks_support_sets")
    return box[:3].copy(), box[3:].copy(), stats


def lks_debug_sync_skip(h, skip: bool):
    """Test hook: the persistent kernels' first CTA skips its grid-barrier arrivals (waits time out)."""
    _check(load().lks_debug_sync_skip(h, int(bool(skip))), "lks_debug_sync_skip")


def lks_debug_copy_skip(h, skip: bool):
    """Test hook: withhold one plane's tile copy in the row-streamed 3D stencils (the waits time out)."""
    _check(load().lks_debug_copy_skip(h, int(bool(skip))), "lks_debug_copy_skip")


def lks_persistent_coupling(h, mode: int = -1) -> bool:
    """Set (1 on, 0 off, 2 automatic) or ask (-1) whether each step's coupling runs as one persistent
    launch; returns whether it does after the call."""
    r = int(load().lks_persistent_coupling(h, int(mode)))
    if r < 0:
        raise LksError(-r, "lks_persistent_coupling")
    return r == 1


def lks_status_string(code: int) -> str:
    return load().lks_status_string(code).decode()


class Solver:
    """Owns one lks_handle for a ``workloads.Problem``; torch supplies device memory and streams."""

    def __init__(self, P, **overrides):
        self.P = P
        self.struct = problem_struct(P, **overrides)
        self.handle = lks_create(self.struct)
        self.forward_count = 0  # forwards run so far: a reverse sweep belongs to the latest one

    @property
    def n_steps(self) -> int:
        return self.struct.n_steps

    def set_initial_state(self, p=None, u=None, s=None):
        check_initial_state(self.P.n_cells, self.P.dim, self.n_dof, p, u, s)
        lks_set_initial_state(self.handle, p, u, s)

    def forward(self, gamma, stream=None) -> float:
        import torch
        check_design_tensor(gamma, self.P.n_design)
        st = torch.cuda.current_stream(gamma.device) if stream is None else stream
        self.forward_count += 1
        return lks_forward(self.handle, gamma.data_ptr(), st.cuda_stream)

    def adjoint(self, seed: float = 1.0, stream=None):
        import torch
        st = torch.cuda.current_stream() if stream is None else stream
        lks_adjoint(self.handle, seed, st.cuda_stream)

    def set_continuation(self, q: float, proj_beta: float):
        """Continuation step (Sec. 3.3): new q and Heaviside beta for the following calls."""
        lks_set_continuation(self.handle, q, proj_beta)

    def adjoint_alks(self, seed: float = 1.0, stream=None):
        """The paper's adjoint (ALKS) in place of the exact one; sensitivity() then gives its dJ/dgamma."""
        import torch
        st = torch.cuda.current_stream() if stream is None else stream
        lks_adjoint_alks(self.handle, seed, st.cuda_stream)

    def alks_adjoint(self):
        """(p~, u~, s~) at t = 0 and the body multipliers at t = 1 of the last adjoint_alks."""
        return lks_get_alks_adjoint(self.handle, self.P.n_cells, self.P.dim)

    def sensitivity(self, out, stream=None):
        import torch
        check_design_tensor(out, self.P.n_design, "out")
        st = torch.cuda.current_stream(out.device) if stream is None else stream
        lks_sensitivity(self.handle, out.data_ptr(), st.cuda_stream)
        return out

    def gradient_host(self, gamma: np.ndarray, stream=None):
        import torch
        st = torch.cuda.current_stream() if stream is None else stream
        out = np.zeros(self.P.n_design)
        if np.size(gamma) != self.P.n_design:
            raise ValueError(f"gamma: {np.size(gamma)} values, expected {self.P.n_design}")
        J = lks_gradient_host(self.handle, np.ascontiguousarray(gamma, dtype=np.float64), out, st.cuda_stream)
        return J, out

    @property
    def n_dof(self) -> int:
        return lks_dof_count(self.struct)

    def warm_start(self, with_adjoint: bool = True, stream=None):
        import torch
        st = torch.cuda.current_stream() if stream is None else stream
        lks_warm_start(self.handle, with_adjoint, st.cuda_stream)

    def constraint(self, gamma, dG=None, stream=None) -> float:
        import torch
        check_design_tensor(gamma, self.P.n_design)
        if dG is not None:
            check_design_tensor(dG, self.P.n_design, "dG")
        st = torch.cuda.current_stream(gamma.device) if stream is None else stream
        return lks_constraint(self.handle, gamma.data_ptr(), 0 if dG is None else dG.data_ptr(), st.cuda_stream)

    def dof_history(self) -> np.ndarray:
        return lks_get_dof_history(self.handle, self.n_steps, self.n_dof)

    def state(self):
        return lks_get_state(self.handle, self.P.n_cells, self.P.dim)

    def initial_adjoint(self):
        return lks_get_initial_adjoint(self.handle, self.P.n_cells, self.P.dim, self.n_dof)

    def launches(self) -> int:
        return lks_launch_count(self.handle)

    def close(self):
        if self.handle:
            lks_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # pragma: no cover
            pass
