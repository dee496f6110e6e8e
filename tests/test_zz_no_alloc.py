"""The allocation-free single-step entry point.

lks_step_noalloc serves callers that cannot let a library allocate device memory (fixed-memory
real-time loops, frameworks that own all allocations); its scratch is a fixed device array shared
by every call. Checked here through the C ABI:
  - two calls in a row (steps 1 and 2, which also reuses the shared scratch) against lks_forward
    over one and two steps, with the FP64 tolerance of the other parity tests, and step 1 against
    the oracle's step;
  - a third call leaves the free device memory unchanged (it allocates nothing);
  - what the step does not do is refused before any device work: the design chain, 3D and FP32
    fields (LKS_ERR_UNSUPPORTED), sizes beyond the fixed array (LKS_ERR_BUDGET), a non-finite DOF
    vector (LKS_ERR_NONFINITE).
This file is collected last, so a run that stops at the first failure has run everything else.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from tests.problems import body2d, body3d, perturbed_state

pytestmark = pytest.mark.gpu

ERR_BUDGET, ERR_NONFINITE, ERR_UNSUPPORTED = 3, 6, 9


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _state(P, p0, u0):
    import torch
    state = torch.zeros((2, P.dim + 1, P.n_cells), dtype=torch.float64, device="cuda")
    state[0, 0] = torch.tensor(p0, device="cuda")
    state[0, 1:] = torch.tensor(u0, device="cuda")
    return state


def test_step_noalloc_matches_forward_two_calls():
    import torch
    from paper_2601_18272_gb300 import lks
    from paper_2601_18272_gb300.lks import Solver, problem_struct

    P, g = body2d(nt=2)
    p0, u0, s0 = perturbed_state(P)
    ref = {}
    for n in (1, 2):
        S = Solver(P, precision=64, ckpt_policy=0, n_steps=n)
        try:
            S.set_initial_state(p0, u0, s0)
            S.forward(torch.tensor(g, device="cuda"))
            ref[n] = (S.state(), S.dof_history()[-1])
        finally:
            S.close()

    prob = problem_struct(P, precision=64, ckpt_policy=0)
    state = _state(P, p0, u0)
    gam = torch.tensor(g, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    s = s0.copy()
    for t in (1, 2):
        s = lks.lks_step_noalloc(prob, gam.data_ptr(), state.data_ptr(), t, s, stream)
        out = state[t % 2].cpu().numpy()
        (p_ref, u_ref), s_ref = ref[t]
        assert _rel(out[0], p_ref) < 1e-12
        assert _rel(out[1:], u_ref) < 1e-12
        np.testing.assert_allclose(s, s_ref, rtol=1e-12, atol=1e-14)


def test_step_noalloc_matches_oracle_step():
    """One step of a translating and rotating body against the oracle's step (FP64)."""
    import torch
    from paper_2601_18272_gb300 import lks
    from paper_2601_18272_gb300.lks import problem_struct

    P, g = body2d(nx=30, ny=18, nd=7, centre=(12.4, 9.1), nt=1)
    p0, u0, s0 = perturbed_state(P, seed=3)
    po, uo, so, _ = O.step(P, g, p0, u0, s0)
    prob = problem_struct(P, precision=64, ckpt_policy=0)
    state = _state(P, p0, u0)
    gam = torch.tensor(g, device="cuda")
    s = lks.lks_step_noalloc(prob, gam.data_ptr(), state.data_ptr(), 1, s0, torch.cuda.current_stream().cuda_stream)
    out = state[1].cpu().numpy()
    assert _rel(out[0], po) < 1e-10
    assert _rel(out[1:], uo) < 1e-10
    np.testing.assert_allclose(s, so, rtol=1e-11, atol=1e-13)


def test_step_noalloc_allocates_nothing():
    """After a first call, further calls leave the device's free memory unchanged."""
    import torch
    from paper_2601_18272_gb300 import lks
    from paper_2601_18272_gb300.lks import problem_struct

    P, g = body2d(nt=3)
    p0, u0, s0 = perturbed_state(P)
    prob = problem_struct(P, precision=64, ckpt_policy=0)
    state = _state(P, p0, u0)
    gam = torch.tensor(g, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    s = lks.lks_step_noalloc(prob, gam.data_ptr(), state.data_ptr(), 1, s0, stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for t in (2, 3):
        s = lks.lks_step_noalloc(prob, gam.data_ptr(), state.data_ptr(), t, s, stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def _refused(prob, P, s0, code):
    import torch
    from paper_2601_18272_gb300 import lks
    state = torch.zeros((2, P.dim + 1, P.n_cells), dtype=torch.float64, device="cuda")
    gam = torch.zeros(P.n_design, dtype=torch.float64, device="cuda")
    with pytest.raises(lks.LksError) as e:
        lks.lks_step_noalloc(prob, gam.data_ptr(), state.data_ptr(), 1, s0, torch.cuda.current_stream().cuda_stream)
    assert e.value.code == code


@pytest.mark.parametrize("field,value", [("filter_radius", 1.5), ("proj_beta", 4.0), ("cyclic_order", 2)])
def test_step_noalloc_refuses_the_design_chain(field, value):
    from paper_2601_18272_gb300.lks import problem_struct
    P, _ = body2d(nt=1)
    _, _, s0 = perturbed_state(P)
    prob = problem_struct(P, precision=64, ckpt_policy=0)
    setattr(prob, field, value)
    if field == "proj_beta":
        prob.proj_eta = 0.5
    _refused(prob, P, s0, ERR_UNSUPPORTED)


def test_step_noalloc_refuses_3d_fp32_and_oversize():
    from paper_2601_18272_gb300.lks import problem_struct
    P3, _ = body3d(nt=1)
    _, _, s3 = perturbed_state(P3)
    _refused(problem_struct(P3, precision=64, ckpt_policy=0), P3, s3, ERR_UNSUPPORTED)
    P, _ = body2d(nt=1)
    _, _, s0 = perturbed_state(P)
    _refused(problem_struct(P, precision=32, ckpt_policy=0), P, s0, ERR_UNSUPPORTED)
    prob = problem_struct(P.replace(n_itr=17), precision=64, ckpt_policy=0)
    _refused(prob, P, s0, ERR_BUDGET)
    bad = s0.copy()
    bad[3] = np.nan
    _refused(problem_struct(P, precision=64, ckpt_policy=0), P, bad, ERR_NONFINITE)
