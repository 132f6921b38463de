"""Python access to the plain serial FP64 CPU oracle (misdc_oracle.c).

TEST INFRASTRUCTURE ONLY. The oracle is the independent checker of the CUDA
library: only the tests, the smoke check and the benchmark's CPU-baseline leg
may import it. It shares no code with the CUDA path; the two meet only in the
seeded input generator (paper_1801_01201_gb300.inputs), which holds none of the
method's arithmetic.

The C library is compiled in-tree with gcc on first use (or by build()).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "misdc_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

MISDC, MISDCQ, CISDCQ, IMEXQ = 0, 1, 2, 3
SCHEMES = {"MISDC": MISDC, "MISDCQ": MISDCQ, "CISDCQ": CISDCQ, "IMEXQ": IMEXQ}

_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (plain gcc, portable flags)."""
    deps = [SRC, os.path.join(HERE, "misdc_oracle.h")]
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(d) for d in deps):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"])
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


dp = C.POINTER(C.c_double)
ip = C.POINTER(C.c_int)


class Mech(C.Structure):
    _fields_ = [("N", C.c_int), ("R", C.c_int), ("W", dp), ("nasa7", dp), ("A", dp),
                ("beta", dp), ("Ea", dp), ("nu_f", ip), ("nu_r", ip), ("D0", dp),
                ("alpha0", C.c_double), ("T_ref", C.c_double), ("theta_exp", C.c_double),
                ("p_ref", C.c_double)]


class AdrCfg(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("vel", dp), ("rho", C.c_double), ("i0", C.c_int),
                ("newton_rtol", C.c_double), ("newton_maxit", C.c_int),
                ("lin_rtol", C.c_double), ("lin_maxit", C.c_int)]


class NuRule(C.Structure):
    """Adaptive nested iterations (see or_nu_rule): eta <= 0 runs all nu."""
    _fields_ = [("eta", C.c_double), ("rho_stall", C.c_double)]


class AdrStats(C.Structure):
    _fields_ = [("newton_solves", C.c_long), ("newton_iters", C.c_long), ("newton_fail", C.c_long),
                ("newton_maxit_seen", C.c_long), ("lin_solves", C.c_long), ("lin_iters", C.c_long),
                ("lin_fail", C.c_long), ("tdiag_fail", C.c_long), ("newton_floor", C.c_long)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _declare(L):
    L.or_lobatto.argtypes = [C.c_int, dp, dp, dp, dp, dp]
    L.or_linear_step.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                 C.c_double, C.c_double, C.c_double, dp, dp]
    L.or_linear_G.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                              C.c_double, dp]
    L.or_pde_step.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.c_double,
                              C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, dp, dp, dp]
    L.or_adr_step.argtypes = [C.POINTER(Mech), C.POINTER(AdrCfg), C.c_int, C.c_int, C.c_int, C.c_int,
                              C.c_double, dp, dp, dp, C.POINTER(AdrStats)]
    L.or_linear_step_ex.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(NuRule), C.c_double,
                                    C.c_double, C.c_double, C.c_double, C.c_double, dp, dp, ip]
    L.or_adr_step_ex.argtypes = [C.POINTER(Mech), C.POINTER(AdrCfg), C.c_int, C.c_int, C.c_int, C.c_int,
                                 C.POINTER(NuRule), C.c_double, dp, dp, dp, ip, C.POINTER(AdrStats)]
    L.or_species_h.restype = C.c_double
    L.or_species_h.argtypes = [C.POINTER(Mech), C.c_int, C.c_double]
    L.or_species_cp.restype = C.c_double
    L.or_species_cp.argtypes = [C.POINTER(Mech), C.c_int, C.c_double]
    L.or_species_s_R.restype = C.c_double
    L.or_species_s_R.argtypes = [C.POINTER(Mech), C.c_int, C.c_double]
    L.or_h_from_T.argtypes = [C.POINTER(Mech), C.c_int, dp, dp, dp]
    L.or_T_from_h.argtypes = [C.POINTER(Mech), C.c_int, dp, dp, dp]
    L.or_wdot.argtypes = [C.POINTER(Mech), C.c_double, dp, C.c_double, dp, dp]
    L.or_wdot_jac.argtypes = [C.POINTER(Mech), C.c_double, dp, C.c_double, dp]
    L.or_reaction_newton.argtypes = [C.POINTER(Mech), C.c_double, C.c_double, dp, C.c_double, dp,
                                     C.c_double, C.c_int]
    L.or_reaction_newton_ex.argtypes = [C.POINTER(Mech), C.c_double, C.c_double, dp, C.c_double, dp,
                                        C.c_double, C.c_int, C.POINTER(C.c_int)]
    L.or_adr_operators.argtypes = [C.POINTER(Mech), C.POINTER(AdrCfg), dp, dp, dp, dp]
    L.or_adr_solve_diff.argtypes = [C.POINTER(Mech), C.POINTER(AdrCfg), C.c_double, dp, dp, dp]
    L.or_lm_terms.argtypes = [C.POINTER(Mech), C.POINTER(LmCfg), dp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
    L.or_lm_step.argtypes = [C.POINTER(Mech), C.POINTER(LmCfg), C.c_int, C.c_int, C.c_int, C.c_double, dp, dp, dp, dp]
    L.or_lm_step_ex.argtypes = [C.POINTER(Mech), C.POINTER(LmCfg), C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, dp, dp, dp, dp]


def _p(a):
    return a.ctypes.data_as(dp) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
def lobatto(M):
    """tau, Q (M x M+1), S (M x M+1), QI (M x M), QE (M x M)."""
    tau = np.zeros(M + 1)
    Q = np.zeros((M, M + 1))
    S = np.zeros((M, M + 1))
    QI = np.zeros((M, M))
    QE = np.zeros((M, M))
    if lib().or_lobatto(M, _p(tau), _p(Q), _p(S), _p(QI), _p(QE)):
        raise ValueError("bad M")
    return tau, Q, S, QI, QE


def linear_step(scheme, M, n_sweeps, nu, dt, a, d, r, phi0=1.0, nu_rule=None):
    """One step of the linear model problem; with nu_rule = (eta, rho_stall) the
    nested iterations are adaptive and (phi, incr, nu_used per sweep) is returned."""
    out = np.zeros(1)
    incr = np.zeros(max(n_sweeps, 1))
    if nu_rule is None:
        rc = lib().or_linear_step(SCHEMES.get(scheme, scheme), M, n_sweeps, nu, dt, a, d, r, phi0,
                                  _p(out), _p(incr))
        if rc:
            raise RuntimeError("linear step failed")
        return out[0], incr[:n_sweeps]
    used = np.zeros(max(n_sweeps, 1), dtype=np.int32)
    rule = NuRule(*nu_rule)
    rc = lib().or_linear_step_ex(SCHEMES.get(scheme, scheme), M, n_sweeps, nu, C.byref(rule), dt, a, d,
                                 r, phi0, _p(out), _p(incr), used.ctypes.data_as(C.POINTER(C.c_int)))
    if rc:
        raise RuntimeError("linear step failed")
    return out[0], incr[:n_sweeps], used[:n_sweeps]


def linear_G(scheme, M, nu, dt, a, d, r):
    G = np.zeros((M, M))
    if lib().or_linear_G(SCHEMES.get(scheme, scheme), M, nu, dt, a, d, r, _p(G)):
        raise RuntimeError("G failed")
    return G


def pde_step(scheme, M, n_sweeps, nu, dt, phi_n, Lx=20.0, a=1.0, d=2.0, r=4.0, left=1.0, right=0.0):
    phi_n = _f64(phi_n)
    out = np.zeros_like(phi_n)
    incr = np.zeros(max(n_sweeps, 1))
    rc = lib().or_pde_step(SCHEMES.get(scheme, scheme), M, n_sweeps, nu, dt, len(phi_n), Lx, a, d, r,
                           left, right, _p(phi_n), _p(out), _p(incr))
    if rc:
        raise RuntimeError("pde step failed")
    return out, incr[:n_sweeps]


class ADR:
    """Oracle handle for one mechanism + flame (keeps the ctypes arrays alive)."""

    def __init__(self, mech, flame, newton_rtol=1e-12, newton_maxit=50, lin_rtol=1e-14, lin_maxit=2000):
        self.mech_py = mech
        self.flame = flame
        self._keep = dict(
            W=_f64(mech.W), nasa7=_f64(mech.nasa7), A=_f64(mech.A), beta=_f64(mech.beta),
            Ea=_f64(mech.Ea), nu_f=np.ascontiguousarray(mech.nu_f, dtype=np.int32),
            nu_r=np.ascontiguousarray(mech.nu_r, dtype=np.int32), D0=_f64(mech.D0),
            vel=_f64(flame.vel))
        k = self._keep
        self.m = Mech(mech.n_species, mech.n_reactions, _p(k["W"]), _p(k["nasa7"]), _p(k["A"]),
                      _p(k["beta"]), _p(k["Ea"]), k["nu_f"].ctypes.data_as(ip),
                      k["nu_r"].ctypes.data_as(ip), _p(k["D0"]), mech.alpha0, mech.T_ref,
                      mech.theta_exp, mech.p_ref)
        self.cfg = AdrCfg(flame.dim, flame.nx, flame.ny, flame.nz, flame.dx, _p(k["vel"]), flame.rho,
                          flame.dominant, newton_rtol, newton_maxit, lin_rtol, lin_maxit)
        self.N = mech.n_species
        self.cells = flame.cells

    # thermo -------------------------------------------------------------
    def h_from_T(self, Y, T):
        Y = _f64(Y); T = _f64(T)
        h = np.zeros(self.cells if T.size == self.cells else T.size)
        lib().or_h_from_T(C.byref(self.m), T.size, _p(Y), _p(T), _p(h))
        return h

    def T_from_h(self, Y, h):
        Y = _f64(Y); h = _f64(h)
        T = np.zeros(h.size)
        lib().or_T_from_h(C.byref(self.m), h.size, _p(Y), _p(h), _p(T))
        return T

    def state_from_YT(self, Y, T):
        """phi = [Y_1..Y_N, h] with h from T by the oracle's thermo."""
        return np.concatenate([_f64(Y), self.h_from_T(Y, T)[None, :]], axis=0)

    def species_h(self, i, T):
        return lib().or_species_h(C.byref(self.m), i, T)

    def species_cp(self, i, T):
        return lib().or_species_cp(C.byref(self.m), i, T)

    def species_s_R(self, i, T):
        return lib().or_species_s_R(C.byref(self.m), i, T)

    def wdot(self, Y, T, rho=None):
        Y = _f64(Y)
        w = np.zeros(self.N)
        q = np.zeros(self.mech_py.n_reactions)
        lib().or_wdot(C.byref(self.m), self.flame.rho if rho is None else rho, _p(Y), T, _p(w), _p(q))
        return w, q

    def wdot_jac(self, Y, T, rho=None):
        Y = _f64(Y)
        J = np.zeros((self.N, self.N + 1))
        lib().or_wdot_jac(C.byref(self.m), self.flame.rho if rho is None else rho, _p(Y), T, _p(J))
        return J

    def reaction_newton(self, wdt, b, hstar, x0, rtol=1e-12, maxit=50, rho=None, floor_out=None):
        """Reaction step S5 of one cell; floor_out (a list) receives 1 when the
        solve ended on the round-off-floor test, else 0."""
        x = _f64(x0).copy()
        b = _f64(b)
        fl = C.c_int(0)
        it = lib().or_reaction_newton_ex(C.byref(self.m), self.flame.rho if rho is None else rho, wdt,
                                         _p(b), hstar, _p(x), rtol, maxit, C.byref(fl))
        if floor_out is not None:
            floor_out.append(fl.value)
        return x, it

    # operators ----------------------------------------------------------
    def operators(self, phi):
        phi = _f64(phi)
        FE = np.zeros_like(phi); FD = np.zeros_like(phi); FR = np.zeros_like(phi)
        lib().or_adr_operators(C.byref(self.m), C.byref(self.cfg), _p(phi), _p(FE), _p(FD), _p(FR))
        return FE, FD, FR

    def solve_diff(self, wdt, coef_state, rhs):
        coef_state = _f64(coef_state); rhs = _f64(rhs)
        x = np.zeros_like(rhs)
        rc = lib().or_adr_solve_diff(C.byref(self.m), C.byref(self.cfg), wdt, _p(coef_state), _p(rhs), _p(x))
        return x, rc

    def step(self, phi, dt, scheme="CISDCQ", M=2, n_sweeps=4, nu=2, n_steps=1, incr_out=None,
             nu_rule=None, nu_used_out=None):
        """Advance phi [(N+1) x cells] by n_steps time steps; returns (phi, stats).
        nu_rule = (eta, rho_stall): adaptive nested iterations (or_nu_rule); the
        iterations each sweep ran are appended to nu_used_out (one array per step)."""
        phi = _f64(phi).copy()
        st = AdrStats()
        out = np.zeros_like(phi)
        rule = NuRule(*(nu_rule if nu_rule is not None else (0.0, 0.0)))
        for _ in range(n_steps):
            incr = np.zeros(max(n_sweeps, 1))
            used = np.zeros(max(n_sweeps, 1), dtype=np.int32)
            rc = lib().or_adr_step_ex(C.byref(self.m), C.byref(self.cfg), SCHEMES.get(scheme, scheme), M,
                                      n_sweeps, nu, C.byref(rule), dt, _p(phi), _p(out), _p(incr),
                                      used.ctypes.data_as(C.POINTER(C.c_int)), C.byref(st))
            if incr_out is not None:
                incr_out.append(incr[:n_sweeps].copy())
            if nu_used_out is not None:
                nu_used_out.append(used[:n_sweeps].copy())
            if rc:
                raise RuntimeError("oracle step failed: %r" % st.as_dict())
            phi, out = out, phi
        return phi, st.as_dict()


R_U = 8.314462618   # J/(mol K)


class LmCfg(C.Structure):
    _fields_ = [("nx", C.c_int), ("dx", C.c_double), ("U_in", C.c_double), ("Y_in", dp),
                ("T_in", C.c_double), ("p0", C.c_double), ("i0", C.c_int),
                ("newton_rtol", C.c_double), ("newton_maxit", C.c_int), ("dchi", C.c_int)]


class LowMach:
    """Oracle handle of the 1D variable-density low-Mach system (Sec. 2, Sec. 3.3):
    state q = [rho, rho Y_1..rho Y_N, rho h] per cell, open boundaries (inflow
    Dirichlet state and velocity at x = 0, zero-gradient outflow at x = L)."""

    def __init__(self, mech, nx, dx, U_in, Y_in, T_in, p0=101325.0, i0=None, newton_rtol=1e-12,
                 newton_maxit=50, dchi=True):
        self.mech_py = mech
        self.N, self.nx = mech.n_species, nx
        self._keep = dict(
            W=_f64(mech.W), nasa7=_f64(mech.nasa7), A=_f64(mech.A), beta=_f64(mech.beta),
            Ea=_f64(mech.Ea), nu_f=np.ascontiguousarray(mech.nu_f, dtype=np.int32),
            nu_r=np.ascontiguousarray(mech.nu_r, dtype=np.int32), D0=_f64(mech.D0), Y_in=_f64(Y_in))
        k = self._keep
        self.m = Mech(mech.n_species, mech.n_reactions, _p(k["W"]), _p(k["nasa7"]), _p(k["A"]),
                      _p(k["beta"]), _p(k["Ea"]), k["nu_f"].ctypes.data_as(ip),
                      k["nu_r"].ctypes.data_as(ip), _p(k["D0"]), mech.alpha0, mech.T_ref,
                      mech.theta_exp, mech.p_ref)
        if i0 is None:
            i0 = int(np.argmax(k["Y_in"]))
        self.cfg = LmCfg(nx, dx, U_in, _p(k["Y_in"]), T_in, p0, i0, newton_rtol, newton_maxit,
                         1 if dchi else 0)
        self.p0 = p0

    def state_from_YT(self, Y, T):
        """q from mass fractions and temperature, with rho from the EOS at p0."""
        Y = _f64(Y)
        T = _f64(T)
        W = _f64(self.mech_py.W)
        rho = self.p0 / (R_U * T * np.sum(Y / W[:, None], axis=0))
        h = np.zeros(T.size)
        lib().or_h_from_T(C.byref(self.m), T.size, _p(np.ascontiguousarray(Y)), _p(T), _p(h))
        return np.concatenate([rho[None], rho[None] * Y, (rho * h)[None]], axis=0)

    def terms(self, q, dchi=None, U_adv=None, T_guess=None):
        """(FA, FD, FR, S, U, p_eos, T) of state q (or_lm_terms)."""
        q = _f64(q)
        nx, F = self.nx, self.N + 2
        FA = np.zeros((F, nx)); FD = np.zeros((F, nx)); FR = np.zeros((F, nx))
        S = np.zeros(nx); U = np.zeros(nx + 1); pe = np.zeros(nx)
        T = _f64(T_guess).copy() if T_guess is not None else np.full(nx, 1000.0)
        rc = lib().or_lm_terms(C.byref(self.m), C.byref(self.cfg), _p(q),
                               _p(_f64(dchi)) if dchi is not None else None,
                               _p(_f64(U_adv)) if U_adv is not None else None,
                               _p(FA), _p(FD), _p(FR), _p(S), _p(U), _p(pe), _p(T))
        if rc:
            raise RuntimeError("temperature diagnosis failed")
        return FA, FD, FR, S, U, pe, T

    def step(self, q, dt, M=2, n_sweeps=4, nu=2, n_steps=1, incr_out=None, scheme="CISDCQ"):
        """Advance q by n_steps steps of CISDCQ-nu or MISDCQ (or_lm_step_ex); returns
        (q, p_eos)."""
        q = _f64(q).copy()
        out = np.zeros_like(q)
        pe = np.zeros(self.nx)
        for _ in range(n_steps):
            incr = np.zeros(max(n_sweeps, 1))
            rc = lib().or_lm_step_ex(C.byref(self.m), C.byref(self.cfg), SCHEMES.get(scheme, scheme), M,
                                     n_sweeps, nu, dt, _p(q), _p(out), _p(incr), _p(pe))
            if incr_out is not None:
                incr_out.append(incr[:n_sweeps].copy())
            if rc:
                raise RuntimeError("low-Mach oracle step failed (%d)" % rc)
            q, out = out, q
        return q, pe
