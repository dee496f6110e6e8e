"""The binomial checkpoint schedule (host logic, no GPU): lks_binomial_plan returns the actions the
library runs for LKS_CKPT_BINOMIAL. A replay on a model of the working state and the snapshot slots
checks that every step is reversed once, in the order N_t .. 1, from the right state, and that no
slot is read after it was overwritten; the number of re-advanced steps is compared with an
exhaustive search over every split of the recursion (itself pinned to Griewank's closed form
r n - beta(c + 1, r - 1) for c restart states)."""
from __future__ import annotations

import sys
from functools import lru_cache
from math import comb

import pytest

from paper_2601_18272_gb300.lks import (LKS_BIN_ADVANCE, LKS_BIN_FWD_SNAPSHOT, LKS_BIN_RESTORE, LKS_BIN_REVERSE,
                                        LKS_BIN_STORE, LksError, lks_binomial_plan)

sys.setrecursionlimit(20000)


def replay(n_steps: int, snapshots: int):
    """Run the plan on a model machine; return (re-advanced steps, snapshot slots used)."""
    ops = lks_binomial_plan(n_steps, snapshots)
    slot = {}          # snapshot slot -> the state index it holds
    working = None     # state index in the working pair (None: undefined)
    base = None        # state index of the last restore
    advanced = 0
    reversed_steps = []
    k = 0
    last_fwd = 0
    while k < len(ops) and ops[k][0] == LKS_BIN_FWD_SNAPSHOT:   # the forward's snapshots come first
        _, a, b, _ = ops[k]
        assert b > last_fwd and b < n_steps and a not in slot
        slot[a] = b
        last_fwd = b
        k += 1
    for kind, a, b, c in ops[k:]:
        if kind == LKS_BIN_RESTORE:
            held = 0 if a < 0 else slot[a]
            assert held == b
            working = base = held
        elif kind == LKS_BIN_ADVANCE:
            assert working == a and b >= 1
            working += b
            advanced += b
        elif kind == LKS_BIN_STORE:
            assert working == b and c == working - base and a >= 0
            slot[a] = b
        elif kind == LKS_BIN_REVERSE:
            assert working == a - 1 and base == b
            reversed_steps.append(a)
            working = None          # the recompute's state is not kept: the next action restores
        else:
            raise AssertionError(f"unexpected action {kind} after the forward's snapshots")
    assert reversed_steps == list(range(n_steps, 0, -1))
    used = (max(slot) + 1) if slot else 0
    assert used <= snapshots
    return advanced, used


@lru_cache(maxsize=None)
def least_cost(n: int, s: int) -> int:
    """Fewest re-advanced steps to reverse n steps from a restorable state with s free slots, over
    every split m: advance m, store, reverse the last n - m with s - 1 slots, then the first m."""
    if n <= 1:
        return 0
    if s == 0:
        return n * (n - 1) // 2
    return min(m + least_cost(n - m, s - 1) + least_cost(m, s) for m in range(1, n))


@lru_cache(maxsize=None)
def least_cost_after_forward(n: int, s: int) -> int:
    """The same when the snapshots of the first descent come free with the forward."""
    if n <= 1:
        return 0
    if s == 0:
        return n * (n - 1) // 2
    return min(least_cost_after_forward(n - m, s - 1) + least_cost(m, s) for m in range(1, n))


def griewank(n: int, c: int) -> int:
    """Griewank's minimal number of forward steps to reverse n steps with c restart states."""
    r = 0
    while comb(c + r, c) < n:
        r += 1
    return r * n - (comb(c + r, c + 1) if r >= 1 else 0)


def test_exhaustive_search_matches_the_closed_form():
    for s in range(1, 6):
        for n in range(1, 70):
            assert least_cost(n, s) == griewank(n, s + 1), (n, s)


@pytest.mark.parametrize("s", [1, 2, 3, 4, 6, 9])
def test_plan_is_valid_and_optimal(s):
    for n in range(1, 90):
        advanced, used = replay(n, s)
        assert advanced == least_cost_after_forward(n, s), (n, s, advanced)
        assert used <= min(s, max(n - 1, 0))


@pytest.mark.parametrize("n,s", [(11, 1), (11, 2), (23, 3), (40, 5), (7, 9), (5000, 10), (10000, 40), (3000, 1)])
def test_plan_at_the_tested_and_workload_sizes(n, s):
    """The GPU tests' (N_t, snapshots) pairs and long marches: valid, and between Griewank's count less
    the forward's n - 1 steps (every snapshot free) and Griewank's count (no snapshot free)."""
    advanced, _ = replay(n, s)
    assert griewank(n, s + 1) - (n - 1) <= advanced <= griewank(n, s + 1)
    if n <= 120:
        assert advanced == least_cost_after_forward(n, s)


def test_enough_snapshots_need_no_re_advance():
    for n in range(1, 40):
        assert replay(n, n)[0] == 0
        assert replay(n, max(n - 1, 1))[0] == 0


def test_arguments_are_checked():
    with pytest.raises(LksError, match="LKS_ERR_ARG"):
        lks_binomial_plan(0, 2)
    with pytest.raises(LksError, match="LKS_ERR_ARG"):
        lks_binomial_plan(10, -1)
    assert lks_binomial_plan(1, 0).tolist() == [[LKS_BIN_RESTORE, -1, 0, 0], [LKS_BIN_REVERSE, 1, 0, 0]]
    ops = lks_binomial_plan(4, 0)  # no slot: every step re-advanced from the initial state
    assert [o[0] for o in ops].count(LKS_BIN_ADVANCE) == 3
    assert [o[0] for o in ops].count(LKS_BIN_STORE) == 0
