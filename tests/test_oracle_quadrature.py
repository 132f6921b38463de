"""Pins of the oracle's Gauss-Lobatto tables (Sec. 3.1, eq. "weights", LU trick)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from conftest import read_golden


def golden_m2():
    out = {}
    for row in read_golden("lobatto_m2.txt"):
        out[row[0]] = np.array([float(Fraction(v)) for v in row[1:]])
    return out


def test_three_node_tables_match_hand_worked_values():
    g = golden_m2()
    tau, Q, S, QI, QE = O.lobatto(2)
    np.testing.assert_allclose(tau, g["tau"], atol=1e-15)
    np.testing.assert_allclose(Q.ravel(), g["Q"], atol=1e-15)
    np.testing.assert_allclose(S.ravel(), g["S"], atol=1e-15)
    np.testing.assert_allclose(QI.ravel(), g["QI"], atol=1e-15)
    np.testing.assert_allclose(QE.ravel(), g["QE"], atol=1e-15)


def test_five_nodes_closed_form():
    tau = O.lobatto(4)[0]
    r = np.sqrt(3.0 / 7.0)
    np.testing.assert_allclose(tau, [0, (1 - r) / 2, 0.5, (1 + r) / 2, 1], atol=1e-15)


@pytest.mark.parametrize("M", [2, 3, 4, 5, 6])
def test_nodes_are_roots_of_legendre_derivative(M):
    tau = O.lobatto(M)[0]
    dP = np.polynomial.legendre.Legendre.basis(M).deriv()
    x = 2 * tau[1:-1] - 1
    assert np.max(np.abs(dP(x))) < 1e-12
    assert tau[0] == 0.0 and tau[-1] == 1.0


@pytest.mark.parametrize("M", [2, 3, 4, 6])
def test_Q_integrates_polynomials_of_degree_M_exactly(M):
    tau, Q, S, QI, QE = O.lobatto(M)
    for p in range(M + 1):
        exact = tau[1:] ** (p + 1) / (p + 1)
        np.testing.assert_allclose(Q @ tau ** p, exact, atol=1e-14)
        exact_s = (tau[1:] ** (p + 1) - tau[:-1] ** (p + 1)) / (p + 1)
        np.testing.assert_allclose(S @ tau ** p, exact_s, atol=1e-14)
    np.testing.assert_allclose(np.cumsum(S, axis=0), Q, atol=1e-14)


@pytest.mark.parametrize("M", [2, 3, 4, 5])
def test_QI_is_U_transpose_of_unit_lower_LU(M):
    tau, Q, S, QI, QE = O.lobatto(M)
    Qt = Q[:, 1:].T
    U = QI.T
    assert np.allclose(np.tril(U, -1), 0.0)
    L = Qt @ np.linalg.inv(U)
    np.testing.assert_allclose(np.diag(L), 1.0, atol=1e-13)
    np.testing.assert_allclose(np.triu(L, 1), 0.0, atol=1e-13)


@pytest.mark.parametrize("M", [2, 4])
def test_QE_is_cumulative_forward_euler(M):
    tau, Q, S, QI, QE = O.lobatto(M)
    for i in range(M):
        for j in range(M):
            want = tau[j + 2] - tau[j + 1] if j < i else 0.0
            assert QE[i, j] == pytest.approx(want, abs=1e-15)
    # forward Euler integrates constants exactly from tau_1: row sums = tau_{m+1} - tau_1
    np.testing.assert_allclose(QE.sum(axis=1), tau[1:] - tau[1], atol=1e-15)
