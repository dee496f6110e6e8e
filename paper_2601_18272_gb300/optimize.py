"""The outer optimisation loop (Algorithm 1): continuation in q and beta (Sec. 3.3), the stopping
criterion (Eq. stopping_criterion), the periodic warm start (Sec. 3.4) and the method of moving
asymptotes (Svanberg 1987) as the optimiser.

The forward, the adjoint, the design chain and the constraint run in the CUDA library (``Solver``);
this module only updates the design variables on the host, once per gradient.

Readings: the objective is maximised (the paper's J_1 and J_2 are the distance travelled and the
angle turned); the text asks for a minimum solid volume, while the printed G <= 0 of Eq. constraint
would bound the volume from above (gamma = 1 is solid in Eq. brinkman_coefficient), so the loop
imposes G >= 0 by default (``min_volume=False`` takes the printed inequality); the stopping
criterion ends a continuation step only at a feasible design.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Optional, Sequence

import numpy as np


class MMA:
    """Method of moving asymptotes (K. Svanberg, Int. J. Numer. Methods Eng. 24 (1987) 359-373) for
    min f0(x) subject to f1(x) <= 0 and xmin <= x <= xmax.

    Each iteration replaces f0 and f1 by convex separable approximations
        f~(x) = r + sum_j p_j / (U_j - x_j) + q_j / (x_j - L_j)
    around the current point, with the asymptotes L < x < U moved by the usual rule (closer after an
    oscillation, farther after steady progress), and solves the subproblem through its dual, a
    concave function of one multiplier lambda >= 0, by bisection on its derivative. An artificial
    variable y >= 0 with cost c y + y^2 / 2 keeps the subproblem feasible from an infeasible start.
    """

    def __init__(self, n: int, xmin=0.0, xmax=1.0, move: float = 0.2, asyinit: float = 0.5, asyincr: float = 1.2,
                 asydecr: float = 0.7, c: float = 1000.0):
        self.n = n
        self.xmin = np.broadcast_to(np.asarray(xmin, dtype=np.float64), (n,)).copy()
        self.xmax = np.broadcast_to(np.asarray(xmax, dtype=np.float64), (n,)).copy()
        self.move, self.asyinit, self.asyincr, self.asydecr, self.c = move, asyinit, asyincr, asydecr, c
        self.k = 0
        self.xold1 = self.xold2 = self.low = self.upp = None

    def step(self, x, f0: float, df0, f1: float, df1):
        """One iteration from x with f0, df/dx0, f1, df1/dx; returns (x_new, lambda)."""
        x = np.asarray(x, dtype=np.float64)
        df0 = np.asarray(df0, dtype=np.float64)
        df1 = np.asarray(df1, dtype=np.float64)
        span = self.xmax - self.xmin
        self.k += 1
        if self.k <= 2:
            low = x - self.asyinit * span
            upp = x + self.asyinit * span
        else:
            trend = (x - self.xold1) * (self.xold1 - self.xold2)
            fac = np.where(trend > 0, self.asyincr, np.where(trend < 0, self.asydecr, 1.0))
            low = x - fac * (self.xold1 - self.low)
            upp = x + fac * (self.upp - self.xold1)
            low = np.clip(low, x - 10.0 * span, x - 0.01 * span)
            upp = np.clip(upp, x + 0.01 * span, x + 10.0 * span)
        alpha = np.maximum(np.maximum(self.xmin, low + 0.1 * (x - low)), x - self.move * span)
        beta = np.minimum(np.minimum(self.xmax, upp - 0.1 * (upp - x)), x + self.move * span)
        ux2, xl2 = (upp - x) ** 2, (x - low) ** 2
        eps = 1e-5 / span

        def coeffs(df):
            a = np.abs(df)
            return ux2 * (np.maximum(df, 0.0) + 1e-3 * a + eps), xl2 * (np.maximum(-df, 0.0) + 1e-3 * a + eps)

        p0, q0 = coeffs(df0)
        p1, q1 = coeffs(df1)
        r1 = f1 - np.sum(p1 / (upp - x) + q1 / (x - low))

        def x_of(lam):  # minimiser of the Lagrangian of the subproblem, separable in x_j
            sp, sq = np.sqrt(p0 + lam * p1), np.sqrt(q0 + lam * q1)
            return np.clip((sp * low + sq * upp) / (sp + sq), alpha, beta)

        def dual_slope(lam):  # derivative of the dual: the approximated constraint minus y(lambda)
            xx = x_of(lam)
            return np.sum(p1 / (upp - xx) + q1 / (xx - low)) + r1 - max(0.0, lam - self.c)

        lam = 0.0
        if dual_slope(0.0) > 0.0:
            lo, hi = 0.0, 1.0
            while dual_slope(hi) > 0.0:
                lo, hi = hi, 2.0 * hi
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                if dual_slope(mid) > 0.0:
                    lo = mid
                else:
                    hi = mid
            lam = 0.5 * (lo + hi)
        xnew = x_of(lam)
        self.xold2, self.xold1 = self.xold1, x.copy()
        self.low, self.upp = low, upp
        return xnew, lam


@dataclass
class Record:
    step: int          # continuation step l
    it: int            # optimisation iteration k within the step
    q: float
    beta: float
    J: float
    G: float
    feasible: bool
    lam: float = 0.0


@dataclass
class Result:
    gamma: np.ndarray
    history: list = field(default_factory=list)


def optimize(solver, gamma0, q_steps: Sequence[float] = (0.1,), beta_steps: Sequence[float] = (0.0,),
             n_opt: int = 50, tol: float = 1e-6, maximize: bool = True, min_volume: bool = True,
             warm_start: bool = False, move: float = 0.2, objective_scale: float = 10.0,
             callback: Optional[Callable[[Record], None]] = None) -> Result:
    """Algorithm 1 on a ``Solver``: for each continuation step l with (q^l, beta^l), up to n_opt
    iterations of design chain + forward (J), constraint (G, dG/dgamma), the stopping criterion
    |J^k - J^(k-1)| / |J^(k-1)| <= tol at a feasible design, adjoint + sensitivity (dJ/dgamma) and an
    MMA update of gamma in [0, 1]. With warm_start, each forward and reverse sweep starts from the
    previous one's final state and initial adjoint (periodic problems). The objective enters MMA
    scaled to objective_scale at the first design."""
    import torch
    x = np.array(gamma0, dtype=np.float64)
    g = torch.tensor(x, dtype=torch.float64, device="cuda")
    dJ, dG = torch.empty_like(g), torch.empty_like(g)
    sgn = -1.0 if maximize else 1.0
    csgn = -1.0 if min_volume else 1.0
    scale = None
    res = Result(gamma=x)
    for l, (q, beta) in enumerate(zip(q_steps, beta_steps)):
        solver.set_continuation(q, beta)
        mma = MMA(x.size, move=move)
        J_prev = None
        for k in range(n_opt):
            g.copy_(torch.from_numpy(x))
            J = solver.forward(g)
            G = solver.constraint(g, dG)
            rec = Record(step=l, it=k, q=q, beta=beta, J=J, G=G, feasible=csgn * G <= 0.0)
            res.history.append(rec)
            if callback:
                callback(rec)
            if J_prev is not None and rec.feasible and abs((J - J_prev) / J_prev) <= tol:
                break
            solver.adjoint(1.0)
            solver.sensitivity(dJ)
            torch.cuda.synchronize()
            if scale is None:
                scale = objective_scale / max(abs(J), 1e-300)
            x, rec.lam = mma.step(x, sgn * scale * J, sgn * scale * dJ.cpu().numpy(), csgn * G,
                                  csgn * dG.cpu().numpy())
            if warm_start:
                solver.warm_start(True)
            J_prev = J
    res.gamma = x
    return res
