"""Binomial checkpointing schedule of the drag gradient (imb_binomial_schedule, host only).

Replayed on a toy machine whose "state" is the time step it holds:

* valid: the adjoints come in the order T-1, ..., 0, each from the state of its own step;
  a restore reads only a slot that holds a stored state; at most snapshots + 1 slots are used;
* optimal: the number of forward steps equals the least number over all recursive reversal
  schedules with that many snapshots, found by brute force over every first-snapshot position
  (small T), and Griewank's closed form r T - C(s + 2 + r - 1, r - 1) with r the least integer
  for which C(s + 1 + r, r) >= T (large T).
"""
from functools import lru_cache
from math import comb

import pytest

from paper_1809_07008_gb300 import binding as B


def _replay(T, s, ops):
    state, slots, adjoints, advances = None, {}, [], 0
    for kind, v in ops:
        if kind == B.CK_ADVANCE:
            assert state is not None and v >= 1
            state += v
            advances += v
        elif kind == B.CK_STORE:
            assert 0 <= v <= s
            if state is None:      # the first operation stores the start state
                assert v == 0 and not slots
                state = 0
            slots[v] = state
        elif kind == B.CK_RESTORE:
            assert v in slots
            state = slots[v]
        else:
            assert kind == B.CK_ADJOINT and v == state
            adjoints.append(v)
    assert adjoints == list(range(T - 1, -1, -1))
    assert len(slots) <= s + 1
    return advances


@lru_cache(None)
def _least(l, s):
    """Fewest forward steps to reverse l steps with s free snapshots, by brute force."""
    if l == 1:
        return 0
    if s == 0:
        return l * (l - 1) // 2
    return min(j + _least(l - j, s - 1) + _least(j, s) for j in range(1, l))


def _closed_form(T, s):
    if T == 1:
        return 0
    S = s + 1
    r = 0
    while comb(S + r, r) < T:
        r += 1
    return r * T - comb(S + 1 + r - 1, r - 1)


@pytest.mark.parametrize("s", [0, 1, 2, 3, 5, 8])
def test_schedule_is_valid_and_least(s):
    for T in range(1, 90):
        ops, adv = B.binomial_schedule(T, s)
        assert _replay(T, min(s, max(T - 1, 0)), ops) == adv
        assert adv == _least(T, min(s, T - 1)), (T, s)


@pytest.mark.parametrize("T,s", [(4000, 40), (4000, 10), (20000, 30), (1000, 3), (777, 1)])
def test_schedule_matches_closed_form(T, s):
    ops, adv = B.binomial_schedule(T, s)
    assert _replay(T, s, ops) == adv
    assert adv == _closed_form(T, s)


def test_more_snapshots_never_cost_more_and_enough_give_one_pass():
    prev = None
    for s in range(0, 12):
        _, adv = B.binomial_schedule(300, s)
        assert prev is None or adv <= prev
        prev = adv
    # with T - 1 snapshots every state is stored on the way: T - 1 forward steps
    _, adv = B.binomial_schedule(50, 49)
    assert adv == 49


def test_schedule_rejects_bad_arguments():
    L = B.load()
    import ctypes as C
    n = C.c_int(0)
    assert L.imb_binomial_schedule(0, 3, None, 0, C.byref(n), None) != 0
    assert L.imb_binomial_schedule(10, -1, None, 0, C.byref(n), None) != 0
    assert L.imb_binomial_schedule(10, 2, None, 0, None, None) != 0
