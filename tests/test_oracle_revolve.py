"""Pins of the checkpointing oracle: Griewank's closed form against exhaustive
minimisation of the recursion, and the published example values.  CPU only."""
import pytest

from oracle import revolve as R


@pytest.mark.parametrize("s", [0, 1, 2, 3, 4])
def test_closed_form_equals_brute_force(s):
    for l in range(1, 41):
        assert R.closed_form(l, s) == R.brute_force(l, s), (l, s)


def test_published_values():
    # Griewank & Walther with S snapshots: S = 20, l = 1000 -> r = 3, t = 2747
    assert R.repetition_number(1000, 20) == 3
    assert 3 * 1000 - R.beta(21, 2) == 2747
    # S = 20, l = 2000 -> r = 4
    assert R.repetition_number(2000, 20) == 4
    # no buffers: quadratic; enough buffers: one forward pass
    assert R.closed_form(10, 0) == 45
    assert R.closed_form(10, 9) == 9


def test_simulator_rejects_bad_schedules():
    good = [("advance", 1), ("final", 2), ("reverse", 1), ("restore", -1), ("reverse", 0)]
    assert R.simulate(good, 2, 1) == 2
    with pytest.raises(AssertionError):
        R.simulate([("advance", 1), ("final", 2), ("reverse", 0)], 2, 1)
    with pytest.raises(AssertionError):
        R.simulate([("advance", 1), ("reverse", 1), ("restore", -1), ("reverse", 0)], 2, 1)
