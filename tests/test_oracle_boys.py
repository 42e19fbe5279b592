"""Pins for the oracle's Boys function F_m(T) = int_0^1 t^2m exp(-T t^2) dt
against the confluent hypergeometric function, closed forms and identities."""
import math

import numpy as np
import pytest
import scipy.special

from oracle import oracle as O

T_GRID = np.concatenate([[0.0], np.logspace(-8, np.log10(200.0), 120)])


@pytest.mark.parametrize("m", range(0, 9))
def test_boys_matches_hyp1f1(m):
    # F_m(T) = 1F1(m+1/2; m+3/2; -T) / (2m+1); scipy's 1F1 is itself only good
    # to ~1e-13 relative in places, hence the looser bound here.
    for T in T_GRID:
        F = O.boys(8, T)
        ref = scipy.special.hyp1f1(m + 0.5, m + 1.5, -T) / (2 * m + 1)
        assert abs(F[m] - ref) <= 5e-13 * abs(ref), (m, T, F[m], ref)


@pytest.mark.parametrize("m", [0, 1, 3, 6, 8])
def test_boys_matches_hyp1f1_40_digits(m):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    for T in T_GRID[::3]:
        F = O.boys(8, T)
        ref = float(mpmath.hyp1f1(m + 0.5, m + 1.5, -mpmath.mpf(T)) / (2 * m + 1))
        assert abs(F[m] - ref) <= 3e-15 * abs(ref), (m, T, F[m], ref)


def test_boys_at_zero():
    F = O.boys(8, 0.0)
    for m in range(9):
        assert F[m] == pytest.approx(1.0 / (2 * m + 1), rel=1e-15)


def test_boys_f0_erf_closed_form():
    for T in T_GRID[1:]:
        ref = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
        assert O.boys(0, T)[0] == pytest.approx(ref, rel=1e-14)


def test_boys_large_T_asymptote():
    T = 200.0
    F = O.boys(6, T)
    for m in range(7):
        dfact = 1.0
        for k in range(2 * m - 1, 1, -2):
            dfact *= k
        ref = dfact / 2 ** (m + 1) * math.sqrt(math.pi / T ** (2 * m + 1))
        assert F[m] == pytest.approx(ref, rel=1e-14)


def test_boys_downward_identity():
    # F_m = (2T F_{m+1} + e^-T) / (2m+1), on both sides of the series/erf switch
    for T in [1e-3, 0.7, 5.0, 29.9, 30.1, 45.0, 120.0]:
        F = O.boys(8, T)
        for m in range(8):
            rhs = (2 * T * F[m + 1] + math.exp(-T)) / (2 * m + 1)
            assert F[m] == pytest.approx(rhs, rel=1e-13)
