"""Pins of the oracle's 1D variable-density low-Mach system (Sec. 2: eqs.
species_equation, enthalpy_equation, continuity_equation, p_eos_definition,
divergence_constraint, S_def), open boundaries."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_1801_01201_gb300 import inputs as I

L_DOMAIN = 6.4e-3


@pytest.fixture(scope="module")
def inert():
    """9 species / 21 reactions with negligible rates, and its unburnt / burnt
    compositions."""
    mech = I.make_mechanism(1801, 9, 21, logA_range=(-3.0, -2.0))
    fl = I.flame_1d(mech, 1801, nx=32, dx=1e-4)
    return mech, fl.Y[:, 0].copy(), fl.Y[:, fl.nx // 2].copy()


def front(mech, Yu, Yb, nx, U_in=0.5):
    dx = L_DOMAIN / nx
    x = (np.arange(nx) + 0.5) * dx
    s = 0.5 * (1 + np.tanh((x - L_DOMAIN / 2) / (L_DOMAIN / 16)))
    Y = Yu[:, None] * (1 - s) + Yb[:, None] * s
    T = 300 + 1700 * s
    lm = O.LowMach(mech, nx, dx, U_in, Yu, 300.0)
    return lm, lm.state_from_YT(Y, T)


def test_S_is_the_rate_the_eos_implies(inert):
    """eq. S_def is the Lagrangian rate of ln p_EOS that the species and enthalpy
    equations imply (it is how the constraint is derived, Sec. 2): with U = 0,
    (1/T) dT/dt + W sum_i (1/W_i) dY_i/dt from the discrete right-hand sides
    equals the discrete S up to their O(dx^2) difference. A sign error in one of
    S's terms (e.g. Gamma_i taken as -rho D_i grad Y_i) leaves an O(1) gap."""
    mech, Yu, Yb = inert
    N, W = mech.n_species, np.asarray(mech.W)
    errs = []
    for nx in (64, 128, 256):
        lm, q = front(mech, Yu, Yb, nx)
        FA, FD, FR, S, U, pe, T = lm.terms(q, U_adv=np.zeros(nx + 1))
        rho = q[0]
        Y = q[1:N + 1] / rho
        dY = (FD[1:N + 1] + FR[1:N + 1]) / rho
        dh = (FD[N + 1] + FA[N + 1]) / rho   # FA holds only the differential diffusion at U = 0
        hs = np.array([[O.lib().or_species_h(C.byref(lm.m), i, t) for t in T] for i in range(N)])
        cps = np.array([[O.lib().or_species_cp(C.byref(lm.m), i, t) for t in T] for i in range(N)])
        dT = (dh - np.sum(hs * dY, axis=0)) / np.sum(Y * cps, axis=0)
        Wm = 1.0 / np.sum(Y / W[:, None], axis=0)
        rate = dT / T + Wm * np.sum(dY / W[:, None], axis=0)
        errs.append(np.max(np.abs(S - rate)) / np.max(np.abs(S)))
    assert errs[0] < 3e-4, errs
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


def test_uniform_inflow_state_is_steady(inert):
    """A domain filled with the inflow state, chemistry off: no flux divergence,
    S = 0, U = U_in on every face, p_EOS = p0."""
    _, Yu, _ = inert
    mech = I.make_mechanism(1801, 9, 21, logA_range=(-30.0, -29.0))
    nx = 40
    lm = O.LowMach(mech, nx, L_DOMAIN / nx, 0.7, Yu, 300.0)
    q = lm.state_from_YT(np.repeat(Yu[:, None], nx, axis=1), np.full(nx, 300.0))
    FA, FD, FR, S, U, pe, T = lm.terms(q)
    scale = np.abs(q).max(axis=1, keepdims=True)
    assert np.max(np.abs(FA) / scale) < 1e-9 and np.max(np.abs(FD) / scale) < 1e-9
    assert np.max(np.abs(S)) < 1e-9
    assert np.max(np.abs(U - 0.7)) < 1e-12
    assert np.max(np.abs(pe / 101325.0 - 1.0)) < 1e-13


def test_velocity_integrates_the_constraint(inert):
    """I4, S6: div U = S + delta_chi cell by cell, U = U_in on the inflow face; the
    front expands the flow (S > 0 where the temperature rises)."""
    mech, Yu, Yb = inert
    nx = 64
    lm, q = front(mech, Yu, Yb, nx)
    dchi = np.linspace(-3.0, 3.0, nx)
    FA, FD, FR, S, U, pe, T = lm.terms(q, dchi=dchi)
    assert U[0] == 0.5
    np.testing.assert_allclose(np.diff(U) / (L_DOMAIN / nx), S + dchi, rtol=1e-12, atol=1e-9)
    assert np.sum(S) > 0.0
