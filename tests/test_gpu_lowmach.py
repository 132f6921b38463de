"""GPU tests of the variable-density low-Mach step (misdc_lowmach_step) through
the C ABI: parity with the oracle's or_lm_step_ex on the same inputs (CISDCQ-2
and MISDCQ, with and without delta_chi, inert and reacting), the oracle's pins
reproduced on the device (a uniform inflow state is steady; with delta_chi the
sweeps drive p_EOS to p0; a uniform reacting mixture follows the
constant-pressure adiabatic reactor), and several flames in one call equal to
one call each, bit for bit.

Bound: 1e-10 relative per field (max|a - b| / max|b|) where the oracle's own
sensitivity to one-ulp input perturbations is far below it (inert fronts,
mild chemistry); the reacting front is held to max(1e-10, 2 S) like the
periodic steps.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_1801_01201_gb300 import inputs as I
from parity_util import TOL, record, relerr, tol_from

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

L_DOMAIN = 6.4e-3


def S():
    from paper_1801_01201_gb300 import solver
    return solver


@pytest.fixture(scope="module")
def comps():
    mech = I.make_mechanism(1801, 9, 21, logA_range=(-3.0, -2.0))
    fl = I.flame_1d(mech, 1801, nx=32, dx=1e-4)
    return fl.Y[:, 0].copy(), fl.Y[:, fl.nx // 2].copy()


def _solver(mech, nx, dx, scheme="CISDCQ", sweeps=4, nu=2, i0=None, Y_in=None):
    """A 1D solver (its grid, mechanism and time-integration options) for the
    low-Mach step; the periodic face velocity it is created with is unused."""
    fl = I.flame_1d(mech, 0, nx=nx, dx=dx)
    if i0 is not None:
        fl.dominant = i0
    return S().Solver(mech, fl, scheme=scheme, n_sweeps=sweeps, nu=nu)


def _front(mech, Yu, Yb, nx, U_in=0.5, dchi=True):
    dx = L_DOMAIN / nx
    x = (np.arange(nx) + 0.5) * dx
    s = 0.5 * (1 + np.tanh((x - L_DOMAIN / 2) / (L_DOMAIN / 16)))
    lm = O.LowMach(mech, nx, dx, U_in, Yu, 300.0, dchi=dchi)
    q = lm.state_from_YT(Yu[:, None] * (1 - s) + Yb[:, None] * s, 300 + 1700 * s)
    return lm, q, dx


@pytest.mark.parametrize("scheme", ["CISDCQ", "MISDCQ"])
@pytest.mark.parametrize("dchi", [False, True])
def test_inert_front_matches_oracle(comps, scheme, dchi):
    Yu, Yb = comps
    mech = I.make_mechanism(1801, 9, 21, logA_range=(-30.0, -29.0))
    nx = 48   # not a multiple of the block's warps
    lm, q, dx = _front(mech, Yu, Yb, nx, dchi=dchi)
    want, pe_want = lm.step(q, 5e-6, n_sweeps=4, nu=2, n_steps=2, scheme=scheme)
    sv = _solver(mech, nx, dx, scheme=scheme, i0=lm.cfg.i0)
    got, pe, status = sv.lowmach_step(q, 5e-6, Yu, 300.0, 0.5, dchi=dchi, n_steps=2)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    err = relerr(got.cpu().numpy(), want)
    record("lowmach_inert_%s_dchi%d" % (scheme, dchi), err=err)
    assert np.all(err < TOL), err
    assert relerr(pe.cpu().numpy(), pe_want) < TOL


@pytest.mark.parametrize("scheme", ["CISDCQ", "MISDCQ"])
def test_reacting_front_matches_oracle(comps, scheme):
    """A front with chemistry (pre-exponential factors 1e2..1e4 in cm-mol-s: the
    reaction moves the mass fractions by up to 14 % per step; stronger rates make
    the EOS-density front, whose synthetic equilibria are anchored for the
    constant-density system, react faster than these steps resolve), with
    delta_chi."""
    Yu, Yb = comps
    mech = I.make_mechanism(1801, 9, 21, logA_range=(2.0, 4.0))
    nx = 40
    lm, q, dx = _front(mech, Yu, Yb, nx)
    want, _ = lm.step(q, 2e-6, n_sweeps=4, nu=2, n_steps=2, scheme=scheme)
    sens = np.zeros(q.shape[0])
    for r in range(4):
        rng = np.random.default_rng(100 + r)
        other, _ = lm.step(q * (1 + 1e-16 * rng.standard_normal(q.shape)), 2e-6, n_sweeps=4, nu=2,
                           n_steps=2, scheme=scheme)
        sens = np.maximum(sens, relerr(other, want))
    sv = _solver(mech, nx, dx, scheme=scheme, i0=lm.cfg.i0)
    got, pe, status = sv.lowmach_step(q, 2e-6, Yu, 300.0, 0.5, n_steps=2)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    err = relerr(got.cpu().numpy(), want)
    record("lowmach_reacting_%s" % scheme, err=err, S=sens)
    assert np.all(err <= tol_from(sens)), (err, sens)


def test_uniform_inflow_state_is_steady_on_the_device(comps):
    Yu, _ = comps
    mech = I.make_mechanism(1801, 9, 21, logA_range=(-30.0, -29.0))
    nx = 32
    lm = O.LowMach(mech, nx, L_DOMAIN / nx, 0.5, Yu, 300.0)
    q0 = lm.state_from_YT(np.repeat(Yu[:, None], nx, axis=1), np.full(nx, 300.0))
    sv = _solver(mech, nx, L_DOMAIN / nx, sweeps=3, i0=lm.cfg.i0)
    q1, pe, status = sv.lowmach_step(q0, 1e-5, Yu, 300.0, 0.5)
    q1 = q1.cpu().numpy()
    assert int(status.item()) == 0
    assert np.max(np.abs(q1 - q0) / np.abs(q0).max(axis=1, keepdims=True)) < 1e-14
    assert np.max(np.abs(pe.cpu().numpy() / 101325.0 - 1.0)) < 1e-14


def test_correction_drives_the_thermodynamic_pressure_to_p0_on_the_device(comps):
    Yu, Yb = comps
    mech = I.make_mechanism(1801, 9, 21, logA_range=(-30.0, -29.0))
    nx = 32
    lm, q, dx = _front(mech, Yu, Yb, nx)
    dev = []
    for sweeps in (2, 8, 16):
        sv = _solver(mech, nx, dx, sweeps=sweeps, i0=lm.cfg.i0)
        _, pe, status = sv.lowmach_step(q, 5e-6, Yu, 300.0, 0.5, n_steps=2)
        assert int(status.item()) == 0
        dev.append(float(np.max(np.abs(pe.cpu().numpy() / 101325.0 - 1.0))))
    record("lowmach_peos_deviation", dev=dev)
    assert dev[0] > 30 * dev[1] > 30 * 30 * dev[2] and dev[2] < 1e-11, dev


def test_uniform_reacting_mixture_is_a_constant_pressure_reactor_on_the_device(comps):
    """The constant-pressure adiabatic reactor (scipy BDF at rtol 1e-12 on
    dY/dt = wdot/rho with h fixed and rho = p0 W/(R T)) against the device's
    low-Mach steps of a uniform mixture with U_in = 0, with delta_chi; cells next
    to the inflow face are left out (its Dirichlet state diffuses in)."""
    from scipy.integrate import solve_ivp
    Yu, _ = comps
    mech = I.make_mechanism(1801, 9, 21, logA_range=(3.0, 5.0))
    N, W, p0, T0, nx = mech.n_species, np.asarray(mech.W), 101325.0, 1000.0, 24
    lm = O.LowMach(mech, nx, 2e-4, 0.0, Yu, T0)
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
    rho_ref = p0 / (O.R_U * temp(Yref) * np.sum(Yref / W))
    sv = _solver(mech, nx, 2e-4, sweeps=8, i0=lm.cfg.i0)
    q, _, status = sv.lowmach_step(q0, t_end / 16, Yu, T0, 0.0, n_steps=16)
    assert int(status.item()) == 0
    q = q.cpu().numpy()
    Y = q[1:N + 1] / q[0]
    err = max(np.max(np.abs(Y[:, 6:] - Yref[:, None])) / np.max(Yref),
              np.max(np.abs(q[0, 6:] / rho_ref - 1.0)))
    record("lowmach_reactor", err=err)
    assert err < 5e-10, err


def test_several_flames_in_one_call_equal_one_call_each(comps):
    Yu, Yb = comps
    mech = I.make_mechanism(1801, 9, 21, logA_range=(2.0, 4.0))
    nx = 40
    states = []
    for k in range(5):
        lm, q, dx = _front(mech, Yu, Yb, nx, U_in=0.3 + 0.1 * k)
        states.append(q * (1 + 0.01 * k))
    sv = _solver(mech, nx, dx, i0=lm.cfg.i0)
    qs = torch.as_tensor(np.stack(states), device="cuda")
    allq, allpe, st = sv.lowmach_step(qs, 2e-6, Yu, 300.0, 0.5)
    assert int(st.abs().sum().item()) == 0
    for k in range(5):
        one, pe, s1 = sv.lowmach_step(torch.as_tensor(states[k], device="cuda"), 2e-6, Yu, 300.0, 0.5)
        assert torch.equal(one, allq[k]) and torch.equal(pe, allpe[k])


def test_lowmach_rejects_bad_input(comps):
    from paper_1801_01201_gb300 import _lib as L
    Yu, _ = comps
    mech = I.make_mechanism(1801, 9, 21)
    two_d = S().Solver(mech, I.flame_2d(mech, 0, n=8, dx=4e-5, radius=1e-4, delta=4e-5))
    q = torch.zeros((mech.n_species + 2, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(L.MisdcError):
        two_d.lowmach_step(q, 1e-6, Yu, 300.0, 0.5)
    sv = _solver(mech, 16, 1e-4)
    with pytest.raises(L.MisdcError):
        sv.lowmach_step(q[:, :16], -1.0, Yu, 300.0, 0.5)
