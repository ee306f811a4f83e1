"""Oracle for binomial recompute-checkpointing (Griewank & Walther's "revolve").

TEST INFRASTRUCTURE (see oracle/wave.py).

Checkpointing (Sec. 1) keeps a few forward states and recomputes the others from
the nearest stored one while the adjoint runs backward.  Model used here: the
adjoint of step n needs the forward state n; the initial state 0 is always
available; `s` state buffers may hold further states; the first forward pass must
also run the last step (for the final receiver record).

Cost = number of forward steps.  The recursion

    T(l, s) = min_{1<=j<l} [ j + T(l-j, s-1) + T(j, s) ],  T(1, s) = 0,
    T(l, 0) = l (l-1) / 2

counts the forward steps needed to reverse l steps when the first state of the range
is available and s extra buffers are free.  Griewank's closed form, with S = s + 1
snapshots (the range's first state occupies one),

    T = r l - beta(S+1, r-1),  beta(S, r) = C(S+r, S),  beta(S, r-1) < l <= beta(S, r),

solves it; the whole gradient costs T(nt, s) + 1 forward steps (the +1 is the last
step of the first pass).
"""
from __future__ import annotations

from functools import lru_cache
from math import comb


def beta(S: int, r: int) -> int:
    if r < 0:
        return 0
    return comb(S + r, S)


def repetition_number(l: int, S: int) -> int:
    r = 0
    while beta(S, r) < l:
        r += 1
    return r


def closed_form(l: int, s: int) -> int:
    """Griewank & Walther's minimal forward-step count with S = s + 1 snapshots."""
    S = s + 1
    r = repetition_number(l, S)
    return r * l - beta(S + 1, r - 1)


def brute_force(l: int, s: int) -> int:
    """The recursion T(l, s) evaluated by exhaustive minimisation (small l only)."""

    @lru_cache(maxsize=None)
    def T(l, s):
        if l <= 1:
            return 0
        if s == 0:
            return l * (l - 1) // 2
        return min(j + T(l - j, s - 1) + T(j, s) for j in range(1, l))

    return T(l, s)


def gradient_forward_steps(nt: int, s: int) -> int:
    """Forward steps of one checkpointed gradient: T(nt, s) + 1."""
    return closed_form(nt, s) + 1


def simulate(actions, nt: int, s: int):
    """Replay an action list and check it.

    actions: sequence of (op, a) with op in
        'advance' (a steps), 'store' (slot a), 'restore' (slot a, or -1 for the
        zero initial state), 'final' (the last step nt-1 -> nt, run once for its
        receiver record; the live state stays nt-1), 'reverse' (adjoint step a;
        needs live state == a).
    Returns the number of forward steps; raises AssertionError on any violation
    (wrong state reversed, reversal out of order, slot out of range).
    """
    live = 0
    slots = {}
    fwd = 0
    expect = nt - 1
    final_done = False
    for op, a in actions:
        if op == "advance":
            assert a >= 1
            live += a
            fwd += a
            assert live <= nt - 1, "advanced past state nt-1"
        elif op == "final":
            assert live == nt - 1 and not final_done
            final_done = True
            fwd += 1
        elif op == "store":
            assert 0 <= a < s, f"slot {a} out of range"
            slots[a] = live
        elif op == "restore":
            if a == -1:
                live = 0
            else:
                assert a in slots, f"slot {a} empty"
                live = slots[a]
        elif op == "reverse":
            assert final_done, "reverse before the final step"
            assert a == expect, f"reverse {a}, expected {expect}"
            assert live == a, f"reverse {a} with live state {live}"
            expect -= 1
        else:
            raise AssertionError(op)
    assert expect == -1, "not every step reversed"
    assert final_done
    return fwd
