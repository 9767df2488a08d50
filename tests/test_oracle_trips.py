"""Pins of the round-trip (tunnelling-time) counters of Sec. 2.3.

With temperatures 1 + k 1e-14 every proposed swap is accepted (|delta| < 1e-12, so
exp(delta) exceeds every u 2^-32 < 1 - 2^-32), and the ascending pass then rotates the
chain: the replica at the lowest slot climbs to the top and every other replica steps
down one slot.  Replica j is therefore at the lowest slot after pass t iff
t = j (mod T): its first arrival is pass j (pass T for replica 0, which starts with a
climb), and it completes a trip of exactly T passes every T passes after that.
"""
import numpy as np
import pytest

from paper_2003_04621_gb300.observables import tunnelling_time


@pytest.mark.parametrize("T,n", [(2, 9), (5, 23), (12, 40), (31, 100)])
def test_rotating_chain_trip_counts(oracle_mod, T, n):
    temps = [1.0 + k * 1e-14 for k in range(T)]
    o = oracle_mod.Oracle(oracle_mod.OracleParams(2, (4, 6), 3, 2, temps, sim_seed=3))
    for _ in range(n):
        o.exchange()
    acc, tries = o.pt_stats()
    np.testing.assert_array_equal(acc, tries)  # every swap accepted
    first = [T if j == 0 else j for j in range(T)]
    expect = sum(max(0, (n - t0) // T) for t0 in first)
    got, total = o.trips()
    np.testing.assert_array_equal(got, expect)
    np.testing.assert_array_equal(total, T * expect)
    if expect:
        assert tunnelling_time(got, total) == T


def test_single_temperature_has_no_trips(oracle_mod):
    o = oracle_mod.Oracle(oracle_mod.OracleParams(2, (4, 4), 2, 2, [1.0], sim_seed=3))
    o.mcs(20)
    n, total = o.trips()
    assert (n == 0).all() and (total == 0).all()
    assert np.isnan(tunnelling_time(n, total))
