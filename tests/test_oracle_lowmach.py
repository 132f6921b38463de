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


def test_uniform_state_is_steady_through_a_step(inert):
    """A full CISDCQ step (S2-S6) keeps the inert inflow state unchanged."""
    _, Yu, _ = inert
    mech = I.make_mechanism(1801, 9, 21, logA_range=(-30.0, -29.0))
    nx = 32
    lm = O.LowMach(mech, nx, L_DOMAIN / nx, 0.5, Yu, 300.0)
    q0 = lm.state_from_YT(np.repeat(Yu[:, None], nx, axis=1), np.full(nx, 300.0))
    q1, pe = lm.step(q0, 1e-5, n_sweeps=3, nu=2)
    assert np.max(np.abs(q1 - q0) / np.abs(q0).max(axis=1, keepdims=True)) < 1e-14
    assert np.max(np.abs(pe / 101325.0 - 1.0)) < 1e-14


def _front_inert(Yu, Yb, dchi):
    mech = I.make_mechanism(1801, 9, 21, logA_range=(-30.0, -29.0))
    nx = 32
    lm = O.LowMach(mech, nx, L_DOMAIN / nx, 0.5, Yu, 300.0, dchi=dchi)
    x = (np.arange(nx) + 0.5) * L_DOMAIN / nx
    s = 0.5 * (1 + np.tanh((x - L_DOMAIN / 2) / (L_DOMAIN / 16)))
    return lm, lm.state_from_YT(Yu[:, None] * (1 - s) + Yb[:, None] * s, 300 + 1700 * s)


@pytest.mark.parametrize("scheme", ["CISDCQ", "MISDCQ"])
def test_each_sweep_adds_one_order_without_the_correction(inert, scheme):
    """Without delta_chi (S6 solves div U = S), 1-4 sweeps give temporal orders
    1-4 on a front with variable density and velocity (against 8 CISDCQ sweeps
    at 1/8 of the smallest step), for the concurrent and the serial scheme."""
    _, Yu, Yb = inert
    lm, q = _front_inert(Yu, Yb, dchi=False)
    t_end = 2e-5
    ref, _ = lm.step(q, t_end / 64, n_sweeps=8, nu=2, n_steps=64)
    for sweeps in (1, 2, 3, 4):
        err = []
        for k in (2, 4, 8):
            got, _ = lm.step(q, t_end / k, n_sweeps=sweeps, nu=2, n_steps=k, scheme=scheme)
            err.append(np.max(np.abs(got[-1] - ref[-1])) / np.max(np.abs(ref[-1])))
        orders = [np.log2(err[i] / err[i + 1]) for i in range(2)]
        assert all(abs(o - sweeps) < 0.25 for o in orders), (sweeps, err, orders)


def test_correction_drives_the_thermodynamic_pressure_to_p0(inert):
    """S6: with delta_chi the sweeps drive p_EOS to p0 (2 -> 16 sweeps: more than
    1e5 times closer); without it p_EOS drifts by the discretisation error."""
    _, Yu, Yb = inert
    lm, q = _front_inert(Yu, Yb, dchi=True)
    dev = []
    for sweeps in (2, 8, 16):
        _, pe = lm.step(q, 5e-6, n_sweeps=sweeps, nu=2, n_steps=2)
        dev.append(np.max(np.abs(pe / 101325.0 - 1.0)))
    assert dev[0] > 30 * dev[1] > 30 * 30 * dev[2] and dev[2] < 1e-11, dev
    lm0, q0 = _front_inert(Yu, Yb, dchi=False)
    _, pe0 = lm0.step(q0, 5e-6, n_sweeps=16, nu=2, n_steps=2)
    assert np.max(np.abs(pe0 / 101325.0 - 1.0)) > 1e4 * dev[2]


@pytest.mark.parametrize("dchi,bounds", [(False, (2e-10, 2e-11)), (True, (1e-8, 5e-10))])
def test_uniform_reacting_mixture_is_a_constant_pressure_reactor(inert, dchi, bounds):
    """A uniform reacting mixture (no inflow through the inflow face: U_in = 0)
    must follow the textbook constant-pressure adiabatic reactor, dY/dt =
    wdot(rho, Y, T)/rho with h fixed and rho = p0 W/(R T): in the low-Mach system
    that takes S (its reaction term), the velocity it induces, the density
    advection and delta_chi together. Reference: scipy's BDF at rtol 1e-12 on
    the reactor ODE; cells next to the inflow face (whose Dirichlet state keeps
    diffusing in) are left out. delta_chi adds the error of its own unconverged
    iteration; without it the match is closer, and a missing S term shows at once."""
    from scipy.integrate import solve_ivp
    _, Yu, _ = inert
    mech = I.make_mechanism(1801, 9, 21, logA_range=(3.0, 5.0))
    N, W, p0, T0, nx = mech.n_species, np.asarray(mech.W), 101325.0, 1000.0, 24
    lm = O.LowMach(mech, nx, 2e-4, 0.0, Yu, T0, dchi=dchi)
    q0 = lm.state_from_YT(np.repeat(Yu[:, None], nx, axis=1), np.full(nx, T0))
    h0 = q0[N + 1, 0] / q0[0, 0]

    def temp(Y):
        T = np.zeros(1)
        O.lib().or_T_from_h(C.byref(lm.m), 1, O._p(np.ascontiguousarray(Y)), O._p(np.array([h0])), O._p(T))
        return T[0]

    def rhs(t, Y):
        T = temp(Y)
        rho = p0 / (O.R_U * T * np.sum(Y / W))
        w = np.zeros(N)
        O.lib().or_wdot(C.byref(lm.m), rho, O._p(np.ascontiguousarray(Y)), T, O._p(w), None)
        return w / rho

    t_end = 6e-8
    sol = solve_ivp(rhs, (0.0, t_end), Yu.copy(), method="BDF", rtol=1e-12, atol=1e-15)
    Yref = sol.y[:, -1]
    assert np.max(np.abs(Yref - Yu)) > 1e-2   # the mixture reacts noticeably
    rho_ref = p0 / (O.R_U * temp(Yref) * np.sum(Yref / W))
    errs = []
    for n_steps, sweeps in ((8, 6), (16, 8)):
        q, pe = lm.step(q0, t_end / n_steps, n_sweeps=sweeps, nu=2, n_steps=n_steps)
        Y = q[1:N + 1] / q[0]
        errs.append(max(np.max(np.abs(Y[:, 6:] - Yref[:, None])) / np.max(Yref),
                        np.max(np.abs(q[0, 6:] / rho_ref - 1.0))))
    assert errs[0] < bounds[0] and errs[1] < bounds[1], errs


@pytest.mark.parametrize("dchi", [False, True])
def test_serial_and_concurrent_sweeps_share_the_fixed_point(inert, dchi):
    """MISDCQ and CISDCQ-2 iterate to the same solution of the node equations (the
    collocation solution; with delta_chi, the one whose nodes satisfy the EOS)."""
    _, Yu, Yb = inert
    lm, q = _front_inert(Yu, Yb, dchi=dchi)
    a, _ = lm.step(q, 1e-5, n_sweeps=30, nu=2, scheme="CISDCQ")
    b, _ = lm.step(q, 1e-5, n_sweeps=30, scheme="MISDCQ")
    assert np.max(np.abs(a - b) / np.abs(a).max(axis=1, keepdims=True)) < 1e-12
