"""The library's binomial checkpoint schedule attains the minimum number of forward steps:
it equals a brute-force dynamic program over all split points and the closed form of
Griewank and Walther, r l - beta(c + 1, r - 1) with beta(c, r) = C(c + r, c), for c stored
states including the initial one; 2000 steps with 40 states need 5097 forward steps."""
from functools import lru_cache
from math import comb

import pytest

from paper_2302_05164_gb300 import pbf


@lru_cache(None)
def brute(l, s):
    if l <= 1:
        return 0
    if s == 0:
        return l * (l - 1) // 2
    return min(m + brute(l - m, s - 1) + brute(m, s) for m in range(1, l))


def closed(l, c):
    r = 0
    while comb(c + r, c) < l:
        r += 1
    return r * l - comb(c + r, c + 1) if r > 0 else 0


@pytest.mark.parametrize("c", [1, 2, 3, 5])
def test_schedule_cost_is_minimal(c):
    for l in range(1, 41):
        got = pbf.pbf_revolve_cost(l, c)
        assert got == brute(l, c - 1) == closed(l, c), (l, c)


def test_configuration_four_schedule():
    assert pbf.pbf_revolve_cost(2000, 40) == 5097
    with pytest.raises(pbf.PbfError):
        pbf.pbf_revolve_cost(0, 4)
