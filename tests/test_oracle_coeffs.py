"""Pins for the oracle's Eq. 3 weights (oracle.fd2_weights).

The weights are pinned three independent ways: against a published table
(tests/golden/fd2_central_weights.txt), against the closed form for centred
second-derivative weights, and by the moment conditions they must satisfy.
"""
import math
from fractions import Fraction

import pytest

import oracle
from conftest import read_golden


@pytest.mark.parametrize("R", [1, 2, 3, 4])
def test_weights_match_published_table(R):
    row = next(r for r in read_golden("fd2_central_weights.txt") if int(r[0]) == R)
    expect = tuple(Fraction(x) for x in row[1:])
    assert oracle.fd2_weights(R) == expect


def test_radius4_is_the_25_point_set():
    assert oracle.fd2_weights(4) == (Fraction(-205, 72), Fraction(8, 5), Fraction(-1, 5),
                                     Fraction(8, 315), Fraction(-1, 560))


@pytest.mark.parametrize("R", range(1, 9))
def test_closed_form(R):
    # c_m = 2 (-1)^(m+1) (R!)^2 / (m^2 (R-m)! (R+m)!),  c_0 = -2 sum_m c_m
    c = [Fraction(2 * (-1) ** (m + 1) * math.factorial(R) ** 2,
                  m * m * math.factorial(R - m) * math.factorial(R + m)) for m in range(1, R + 1)]
    assert oracle.fd2_weights(R) == tuple([-2 * sum(c)] + c)


@pytest.mark.parametrize("R", range(1, 9))
def test_moment_conditions(R):
    w = oracle.fd2_weights(R)
    full = {0: w[0]}
    for m in range(1, R + 1):
        full[m] = full[-m] = w[m]
    for k in range(0, 2 * R + 2):
        moment = sum(c * Fraction(m) ** k for m, c in full.items())
        assert moment == (2 if k == 2 else 0), (R, k)
    # and the next even moment is NOT zero: the order is exactly 2R
    assert sum(c * Fraction(m) ** (2 * R + 2) for m, c in full.items()) != 0


def test_float_coeffs_round_the_rationals():
    for R in range(1, 5):
        c = oracle.fd2_coeffs(R)
        assert all(float(x) == y for x, y in zip(oracle.fd2_weights(R), c))
