"""The allocation-free single-step entry point against the handle-based forward march.

lks_step_noalloc serves callers that cannot allocate device memory (graph capture in relaxed
mode, fixed-memory real-time loops, frameworks that own all allocations); its scratch is a fixed
device array shared by every call. This checks it through the C ABI on two calls in a row (steps
1 and 2, which also exercises reuse of the shared scratch) against lks_forward over one and two
steps, with the FP64 tolerance of the other parity tests.
"""
from __future__ import annotations

import numpy as np
import pytest

from tests.problems import body2d, perturbed_state

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


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
    N = P.n_cells
    state = torch.zeros((2, 3, N), dtype=torch.float64, device="cuda")
    state[0, 0] = torch.tensor(p0, device="cuda")
    state[0, 1:] = torch.tensor(u0, device="cuda")
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
