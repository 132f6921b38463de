"""Pins of the oracle's sweeps on the linear model problem (Sec. 4, Sec. 5.1)."""
import numpy as np
import pytest

import oracle as O
from conftest import read_golden

SCHEMES = [("MISDC", 1), ("MISDCQ", 1), ("CISDCQ", 1), ("CISDCQ", 2), ("CISDCQ", 3), ("CISDCQ", 6), ("IMEXQ", 1)]


def pade(z, M):
    """Stability function of Lobatto IIIA collocation: diagonal (M, M) Pade of exp."""
    from math import factorial
    num = sum(factorial(2 * M - j) * factorial(M) / (factorial(2 * M) * factorial(j) * factorial(M - j)) * z ** j
              for j in range(M + 1))
    den = sum(factorial(2 * M - j) * factorial(M) / (factorial(2 * M) * factorial(j) * factorial(M - j)) * (-z) ** j
              for j in range(M + 1))
    return num / den


@pytest.mark.parametrize("M", [2, 4])
@pytest.mark.parametrize("scheme,nu", SCHEMES)
def test_sweeps_converge_to_collocation_solution(M, scheme, nu):
    a, d, r = 0.3, -0.7, -0.9
    v, incr = O.linear_step(scheme, M, 120, nu, 1.0, a, d, r)
    assert v == pytest.approx(pade(a + d + r, M), rel=1e-13, abs=1e-15)


def test_pade_helper_is_textbook():
    z = 0.37
    assert pade(z, 2) == pytest.approx((1 + z / 2 + z * z / 12) / (1 - z / 2 + z * z / 12), rel=1e-15)


def gamma(scheme, M, nu, a, d, r):
    return max(abs(np.linalg.eigvals(O.linear_G(scheme, M, nu, 1.0, a, d, r))))


def test_iteration_matrix_predicts_sweep_increments():
    """Phi^(k+1) - Phi^(k) = G (Phi^(k) - Phi^(k-1)): increments decay at rate gamma(G)."""
    M, a, d, r = 4, 1.0, -5.0, -10.0
    for scheme, nu in [("MISDCQ", 1), ("CISDCQ", 3)]:
        g = gamma(scheme, M, nu, a, d, r)
        v, inc = O.linear_step(scheme, M, 40, nu, 1.0, a, d, r)
        k0 = 4
        k1 = k0 + int(np.log(1e-10) / np.log(g))      # stay above round-off
        rate = (inc[k1] / inc[k0]) ** (1.0 / (k1 - k0))
        assert rate == pytest.approx(g, rel=0.2)


@pytest.mark.parametrize("M", [2, 4])
def test_imexq_stiff_limit_gamma_vanishes(M):
    # lim_{d+r -> -inf} gamma(G) = 0 for the fully coupled implicit sweep
    g = [gamma("IMEXQ", M, 1, 1.0, s / 3, 2 * s / 3) for s in (-1e3, -1e6, -1e9)]
    assert g[0] > g[1] > g[2]
    assert g[2] < 2e-3


def test_lu_sdc_limit_and_split_schemes_deteriorate():
    # MISDCQ with a = d = 0 is Weiser's LU-SDC: gamma -> 0 in the stiff limit;
    # with separate D and R solves the stiff limit is slow (gamma -> 1).
    assert gamma("MISDCQ", 4, 1, 0.0, 0.0, -1e9) < 1e-3
    assert gamma("MISDCQ", 4, 1, 1.0, -1e6 / 3, -2e6 / 3) > 0.999
    assert gamma("CISDCQ", 4, 1, 1.0, -1e6 / 3, -2e6 / 3) > 0.999


@pytest.mark.parametrize("M", [2, 4])
def test_nonstiff_rates_agree(M):
    g = [gamma(s, M, nu, 1.0, -0.05, -0.1) for s, nu in [("MISDCQ", 1), ("CISDCQ", 1), ("CISDCQ", 3), ("IMEXQ", 1)]]
    assert max(g) / min(g) < 1.05


@pytest.mark.parametrize("M", [2, 4])
def test_nested_iterations_order_in_mid_range(M):
    # Sec. 4: CISDCQ-1 converges slower than MISDCQ, CISDCQ-3 and -6 faster.
    for r in (-4.0, -20.0, -100.0):
        gm = gamma("MISDCQ", M, 1, 1.0, r / 2, r)
        assert gamma("CISDCQ", M, 1, 1.0, r / 2, r) > gm
        assert gamma("CISDCQ", M, 3, 1.0, r / 2, r) < gm
        assert gamma("CISDCQ", M, 6, 1.0, r / 2, r) < gm


def sweeps_to(scheme, nu, d, r, tol=1e-14, kmax=800):
    v, inc = O.linear_step(scheme, 4, kmax, nu, 1.0, 1.0, d, r)
    idx = np.where(inc <= tol)[0]
    assert len(idx), "no convergence"
    return int(idx[0]) + 1


# Entries of Tables 1-2 that the equations as printed do not reproduce:
# (-5,-5) nu=1 prints 2.1 where the sweep counts give 1.2 (and the text states that
# CISDCQ-1 converges slower than MISDCQ there); the two nu=3 entries at r=-4 and r=-20.
TABLE_EXCEPTIONS = {("-5", "-5", 1), ("-2", "-4", 3), ("-10", "-20", 3)}


@pytest.mark.slow
def test_tables_1_and_2_sweep_counts():
    M = 4
    checked = 0
    for row in read_golden("tables_paper.txt"):
        if row[0] not in ("T1", "T2"):
            continue
        d, r = float(row[1]), float(row[2])
        NM = sweeps_to("MISDCQ", 1, d, r)
        for nu, Rp in zip((1, 3, 6), map(float, row[3:6])):
            NC = sweeps_to("CISDCQ", nu, d, r)
            f = 2 * M / (2 * nu + M - 1)
            if (row[1], row[2], nu) in TABLE_EXCEPTIONS:
                continue
            # printed R has one decimal: N_C must lie in the implied band, +-1 sweep
            lo, hi = NM * f / (Rp + 0.05), NM * f / (Rp - 0.05)
            assert lo - 1 <= NC <= hi + 1, (row, nu, NM, NC, lo, hi)
            checked += 1
    assert checked == 15
    # the documented exception that the text decides: CISDCQ-1 slower than MISDCQ
    assert sweeps_to("CISDCQ", 1, -5.0, -5.0) > sweeps_to("MISDCQ", 1, -5.0, -5.0)
