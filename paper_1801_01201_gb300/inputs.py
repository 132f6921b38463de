"""Seeded synthetic inputs: mechanisms, flames and velocity fields.

This module only draws and lays out input data. It evaluates none of the
method's arithmetic (no rates, no thermodynamic state, no operators): the CPU
oracle and the CUDA library each turn these arrays into enthalpies, rates and
updates with their own code. Everything here is deterministic in its seed.

Units on output are SI: W in kg/mol, A in (m^3/mol)^(order-1)/s, Ea in J/mol,
diffusivities in m^2/s, lengths in m, velocities in m/s, T in K.

The mechanism recipe (element-balanced stoichiometry, W in [1, 40] g/mol,
A log-uniform in [1e8, 1e14] in cm-mol-s units, beta in [-1, 1], Ea in
[0, 200] kJ/mol, NASA-7 polynomials on one range) is the synthetic stand-in
for the detailed mechanism of the paper's Section 5.3 flame, which is not
available.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

R_U = 8.314462618          # J/(mol K)
P_ATM = 101325.0           # Pa
ELEMENT_MASS = (1.008, 12.011, 14.007, 15.999)   # g/mol, four pseudo-elements
MAX_ATOMS = 8


@dataclass
class Mechanism:
    n_species: int
    n_reactions: int
    W: np.ndarray          # [N] kg/mol
    elem: np.ndarray       # [E][N] atoms of element k in species i
    nasa7: np.ndarray      # [N][7] a1..a7 (one temperature range)
    A: np.ndarray          # [R] SI pre-exponential factor
    beta: np.ndarray       # [R]
    Ea: np.ndarray         # [R] J/mol
    nu_f: np.ndarray       # [R][N] int32 reactant stoichiometry (nu')
    nu_r: np.ndarray       # [R][N] int32 product stoichiometry (nu'')
    D0: np.ndarray         # [N] species diffusivity at T_ref, m^2/s
    alpha0: float          # thermal diffusivity lambda/(rho cp) at T_ref, m^2/s
    T_ref: float = 2000.0
    theta_exp: float = 0.7
    p_ref: float = P_ATM
    seed: int = 0
    Y_u: np.ndarray = None   # unburnt anchor composition (equilibrium at T_u)
    Y_b: np.ndarray = None   # burnt anchor composition (equilibrium at T_b)
    i0: int = 0              # dominant species (largest unburnt mass fraction)
    rho: float = 1.0         # constant density, p W_mix(Y_u) / (R T_u)
    T_u: float = 300.0
    T_b: float = 2000.0


@dataclass
class Flame:
    dim: int
    nx: int
    ny: int
    nz: int
    dx: float
    Y: np.ndarray          # [N][cells] mass fractions (x fastest)
    T: np.ndarray          # [cells] K
    vel: np.ndarray        # [3][cells] face velocity at the low face of each cell, per direction
    rho: float
    dominant: int          # index of the dominant species i0
    meta: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz


def _candidates(rng):
    out = []
    for comp in itertools.product(range(MAX_ATOMS + 1), repeat=4):
        t = sum(comp)
        if 1 <= t <= MAX_ATOMS:
            w = sum(a * b for a, b in zip(comp, ELEMENT_MASS))
            if 1.0 <= w <= 40.0:
                out.append(comp)
    return out


def _grow_species(rng, n):
    """Element-closed species set: start from atoms, add sums of two members."""
    cands = set(_candidates(rng))
    atoms = [tuple(1 if k == e else 0 for k in range(4)) for e in range(4)]
    species = [a for a in atoms if a in cands]
    rng.shuffle(species)
    n_start = 1 if n <= 4 else (2 if n < 12 else (3 if n < 30 else 4))
    species = species[:n_start]
    tries = 0
    while len(species) < n:
        tries += 1
        if tries > 100000:
            raise RuntimeError("species growth stalled")
        a = species[rng.integers(len(species))]
        b = species[rng.integers(len(species))]
        s = tuple(x + y for x, y in zip(a, b))
        if s in cands and s not in species:
            species.append(s)
    return species


def _balanced_reactions(species):
    comp = [np.array(s) for s in species]
    n = len(species)
    rx = set()
    # 1 <-> 2 (including X <-> 2Y)
    for x in range(n):
        for y in range(n):
            for z in range(y, n):
                if x in (y, z):
                    continue
                if np.array_equal(comp[x], comp[y] + comp[z]):
                    rx.add(((x,), (y, z)))
    # 2 <-> 2 (no species on both sides)
    pairs = [(i, j) for i in range(n) for j in range(i, n)]
    sums = {}
    for p in pairs:
        key = tuple(comp[p[0]] + comp[p[1]])
        sums.setdefault(key, []).append(p)
    for key, lst in sums.items():
        for a in range(len(lst)):
            for b in range(a + 1, len(lst)):
                L, P = lst[a], lst[b]
                if set(L) & set(P):
                    continue
                rx.add((L, P))
    return sorted(rx)


def _dirichlet(rng, n, alpha=0.3, floor=1e-6):
    y = rng.gamma(alpha, 1.0, n)
    y = np.maximum(y / y.sum(), floor)
    return y / y.sum()


def _anchor_compositions(rng, n):
    """Unburnt (largest raised to 0.7, renormalised) and burnt compositions."""
    yu = _dirichlet(rng, n)
    i0 = int(np.argmax(yu))
    rest = yu.sum() - yu[i0]
    yu = yu * (0.3 / rest)
    yu[i0] = 0.7
    yu = yu / yu.sum()
    yb = _dirichlet(rng, n)
    return yu, yb, i0


def make_mechanism(seed: int, n_species: int, n_reactions: int,
                   T_u: float = 300.0, T_b: float = 2000.0,
                   logA_range: tuple = (8.0, 14.0)) -> Mechanism:
    """Seeded, element-balanced synthetic mechanism with equilibrium-anchored thermo.

    Stoichiometry: reactions drawn from the enumerated balanced forms
    X <-> Y + Z and X + Y <-> Z + W; every species takes part.

    Thermo: each species' NASA-7 coefficients are composed from per-element
    NASA-7 terms (which cancel in every balanced reaction) plus a species term
    chosen so that the unburnt composition at T_u and the burnt composition at
    T_b are exact chemical equilibria of every reaction at the constant
    density rho, with equilibrium compositions in between that interpolate
    log-linearly in w(T) = (1/T_u - 1/T)/(1/T_u - 1/T_b). Only coefficients
    are composed here; no thermodynamic state or rate is evaluated.

    Each reaction is written in the direction whose equilibrium constant is
    larger at its smaller anchor value, which bounds k_r/k_f.
    """
    rng = np.random.default_rng(seed)
    for attempt in range(200):
        species = _grow_species(rng, n_species)
        rxs = _balanced_reactions(species)
        if len(rxs) < n_reactions:
            continue
        order = rng.permutation(len(rxs))
        chosen, covered = [], set()
        for idx in order:                     # greedy cover first
            L, P = rxs[idx]
            if set(L + P) - covered:
                chosen.append(idx)
                covered |= set(L + P)
            if len(covered) == n_species:
                break
        if len(covered) < n_species or len(chosen) > n_reactions:
            continue
        for idx in order:
            if len(chosen) == n_reactions:
                break
            if idx not in chosen:
                chosen.append(idx)
        if len(chosen) == n_reactions:
            break
    else:
        raise RuntimeError("could not build mechanism")

    N, R = n_species, n_reactions
    elem = np.array(species, dtype=np.float64).T.copy()       # [E][N]
    W = (np.array(ELEMENT_MASS) @ elem) * 1e-3                  # kg/mol
    yu, yb, i0 = _anchor_compositions(rng, N)
    rho = P_ATM * (1.0 / float(np.sum(yu / W))) / (R_U * T_u)
    cu = rho * yu / W
    cb = rho * yb / W

    # per-element NASA-7 terms e[k] = (e1..e7): cp/R per atom = e1 + e2 T + e3 T^2
    E = elem.shape[0]
    e = np.zeros((E, 7))
    e[:, 0] = rng.uniform(1.5, 2.0, E)
    e[:, 1] = rng.uniform(0.0, 4e-4, E)
    e[:, 2] = rng.uniform(-4e-8, 0.0, E)
    e[:, 5] = rng.uniform(-3000.0, 3000.0, E)
    e[:, 6] = rng.uniform(-5.0, 5.0, E)
    # species: g/(RT) = -ln(R T/p) - [(1-w) ln c_u + w ln c_b] + sum_k a_k phi_k(T)
    # in the NASA form a1(1 - ln T) - a2 T/2 - ... + a6/T - a7
    D = 1.0 / T_u - 1.0 / T_b
    Lr = np.log(cb) - np.log(cu)
    nasa = elem.T @ e                                           # element parts
    nasa[:, 0] += 1.0
    nasa[:, 5] += Lr / D
    nasa[:, 6] += 1.0 + math.log(R_U / P_ATM) + np.log(cu) + Lr / (T_u * D)

    nu_f = np.zeros((R, N), dtype=np.int32)
    nu_r = np.zeros((R, N), dtype=np.int32)
    for r, idx in enumerate(chosen):
        L, P = rxs[idx]
        lf = np.zeros(N, dtype=np.int32)
        lr = np.zeros(N, dtype=np.int32)
        for s_ in L:
            lf[s_] += 1
        for s_ in P:
            lr[s_] += 1
        dnu = lr - lf
        lnK = min(float(dnu @ np.log(cu)), float(dnu @ np.log(cb)))   # ln Kc at the anchors
        lnK_rev = min(float(-dnu @ np.log(cu)), float(-dnu @ np.log(cb)))
        if lnK_rev > lnK:
            lf, lr = lr, lf
        nu_f[r], nu_r[r] = lf, lr

    order = nu_f.sum(axis=1)
    logA = rng.uniform(logA_range[0], logA_range[1], R)
    A = 10.0 ** logA * (1e-6) ** (order - 1)                   # cm-mol-s -> SI
    beta = rng.uniform(-1.0, 1.0, R)
    Ea = rng.uniform(0.0, 200.0, R) * 1e3
    D0 = rng.uniform(5e-5, 1e-4, N)
    alpha0 = float(rng.uniform(5e-5, 1e-4))
    return Mechanism(N, R, W, elem, nasa, A, beta, Ea, nu_f, nu_r, D0, alpha0,
                     seed=seed, Y_u=yu, Y_b=yb, i0=i0, rho=rho, T_u=T_u, T_b=T_b)


def equilibrium_path_composition(mech: Mechanism, T: np.ndarray) -> np.ndarray:
    """Front composition at temperature T: c_i = alpha^{atoms_i} c_u^{1-w} c_b^w.

    This is the equilibrium composition the thermo was anchored on (any alpha
    keeps every balanced reaction in equilibrium, since atoms balance); alpha is
    the normalisation that makes the mass fractions sum to one (bisection).
    """
    T = np.asarray(T, dtype=np.float64)
    w = (1.0 / mech.T_u - 1.0 / T) / (1.0 / mech.T_u - 1.0 / mech.T_b)
    atoms = mech.elem.sum(axis=0)
    lyu, lyb = np.log(mech.Y_u), np.log(mech.Y_b)
    base = np.exp((1.0 - w)[None, :] * lyu[:, None] + w[None, :] * lyb[:, None])   # [N][cells]
    lo = np.full(T.shape, 1e-3)
    hi = np.full(T.shape, 1e3)
    for _ in range(200):
        mid = np.sqrt(lo * hi)
        s = np.sum(mid[None, :] ** atoms[:, None] * base, axis=0)
        hi = np.where(s > 1.0, mid, hi)
        lo = np.where(s > 1.0, lo, mid)
    a = np.sqrt(lo * hi)
    Y = a[None, :] ** atoms[:, None] * base
    return Y / Y.sum(axis=0)[None, :]


def _centres(n, dx):
    return (np.arange(n) + 0.5) * dx


def _profile(mech: Mechanism, s: np.ndarray):
    """T = T_u + (T_b - T_u) s and the equilibrium-path composition at that T."""
    T = mech.T_u + (mech.T_b - mech.T_u) * s
    return equilibrium_path_composition(mech, T), T


def flame_1d(mech: Mechanism, seed: int, nx=128, dx=1e-4, u=1.0) -> Flame:
    """Periodic 1D slab: s(x) = (tanh((x-L/4)/d) - tanh((x-3L/4)/d))/2, d = 4 dx."""
    L = nx * dx
    x = _centres(nx, dx)
    d = 4 * dx
    s = 0.5 * (np.tanh((x - L / 4) / d) - np.tanh((x - 3 * L / 4) / d))
    Y, T = _profile(mech, s)
    vel = np.zeros((3, nx))
    vel[0, :] = u
    return Flame(1, nx, 1, 1, dx, Y, T, vel, mech.rho, mech.i0, {"kind": "slab_1d", "u": u})


def _taylor_green_faces(nx, ny, dx, amp):
    """Face velocities from a node streamfunction psi = (A/k) sin kx sin ky.

    u = d(psi)/dy and v = -d(psi)/dx as differences of node values, so the
    discrete divergence of every cell telescopes to zero.
    """
    L = nx * dx
    k = 2 * math.pi / L
    xn = np.arange(nx + 1) * dx
    yn = np.arange(ny + 1) * dx
    psi = (amp / k) * np.sin(k * xn)[None, :] * np.sin(k * yn)[:, None]   # [ny+1][nx+1]
    ux = (psi[1:, :nx] - psi[:-1, :nx]) / dx          # face (i-1/2, j): psi(i,j+1)-psi(i,j)
    uy = -(psi[:ny, 1:] - psi[:ny, :-1]) / dx         # face (i, j-1/2): -(psi(i+1,j)-psi(i,j))
    vel = np.zeros((3, ny * nx))
    vel[0] = ux.reshape(-1)
    vel[1] = uy.reshape(-1)
    return vel


def flame_2d(mech: Mechanism, seed: int, n=256, dx=4e-5, amp=2.0, radius=2e-3,
             delta=2e-4, centre=None) -> Flame:
    """Periodic 2D circular kernel s(r) = (1 - tanh((r - r0)/delta))/2 in a Taylor-Green field."""
    L = n * dx
    c = (L / 2, L / 2) if centre is None else centre
    xc = _centres(n, dx)
    X, Yg = np.meshgrid(xc, xc)
    ddx, ddy = X - c[0], Yg - c[1]
    ddx -= L * np.round(ddx / L)          # nearest periodic image
    ddy -= L * np.round(ddy / L)
    r = np.sqrt(ddx ** 2 + ddy ** 2).reshape(-1)
    s = 0.5 * (1.0 - np.tanh((r - radius) / delta))
    Y, T = _profile(mech, s)
    vel = _taylor_green_faces(n, n, dx, amp)
    return Flame(2, n, n, 1, dx, Y, T, vel, mech.rho, mech.i0,
                 {"kind": "kernel_2d", "amp": amp, "radius": radius})


def _solenoidal_3d(rng, n, dx, urms, k0_cells=4):
    """Random-phase field as the discrete curl of an edge vector potential.

    Potential spectrum ~ k^4 exp(-2 (k/k0)^2) / k^2 (so velocity ~ k^4 exp(...)),
    random phases; face fluxes are differences of edge values, hence discretely
    divergence free. Scaled to per-component rms urms.
    """
    L = n * dx
    k = np.fft.fftfreq(n, d=1.0 / n) * (2 * math.pi / L)
    KX, KY, KZ = np.meshgrid(k, k, k, indexing="ij")
    kk = np.sqrt(KX**2 + KY**2 + KZ**2)
    k0 = k0_cells * 2 * math.pi / L
    amp = np.where(kk > 0, kk**4 * np.exp(-2 * (kk / k0) ** 2) / np.maximum(kk, 1e-30) ** 2, 0.0)
    pot = []
    for _ in range(3):
        ph = rng.uniform(0, 2 * math.pi, kk.shape)
        f = amp * np.exp(1j * ph)
        pot.append(np.real(np.fft.ifftn(f)))          # [x][y][z]
    ax, ay, az = [p.transpose(2, 1, 0).copy() for p in pot]   # -> [z][y][x]

    def d(a, axis):   # forward difference a(i+1) - a(i), periodic
        return (np.roll(a, -1, axis=axis) - a) / dx
    # faces: u = dAz/dy - dAy/dz, v = dAx/dz - dAz/dx, w = dAy/dx - dAx/dy
    u = d(az, 1) - d(ay, 0)
    v = d(ax, 0) - d(az, 2)
    w = d(ay, 2) - d(ax, 1)
    s = urms / max(np.sqrt(np.mean(u**2)), np.sqrt(np.mean(v**2)), np.sqrt(np.mean(w**2)))
    return np.stack([u.reshape(-1) * s, v.reshape(-1) * s, w.reshape(-1) * s])


def flame_3d(mech: Mechanism, seed: int, n=128, dx=1e-4, urms=3.0, radius=2e-3,
             delta=2e-4) -> Flame:
    """Periodic 3D spherical kernel in a random-phase solenoidal field."""
    rng = np.random.default_rng(seed)
    L = n * dx
    xc = _centres(n, dx)
    Z, Yg, X = np.meshgrid(xc, xc, xc, indexing="ij")
    r = np.sqrt((X - L / 2) ** 2 + (Yg - L / 2) ** 2 + (Z - L / 2) ** 2).reshape(-1)
    s = 0.5 * (1.0 - np.tanh((r - radius) / delta))
    Y, T = _profile(mech, s)
    vel = _solenoidal_3d(rng, n, dx, urms)
    return Flame(3, n, n, n, dx, Y, T, vel, mech.rho, mech.i0,
                 {"kind": "kernel_3d", "urms": urms})


# ---------------------------------------------------------------------------
# Named workloads (seed = 1801 + workload index)
# ---------------------------------------------------------------------------
WORKLOADS = {
    # name: (mechanism (N, R), builder, kwargs, time integration)
    "flame1d_128_n9": dict(mech=(9, 21), seed=1801, dim=1, grid=dict(nx=128, dx=1e-4, u=1.0),
                           dt=1e-5, steps=20, sweeps=4, nodes=3, nu=2),
    "flame2d_256_n21": dict(mech=(21, 84), seed=1802, dim=2, grid=dict(n=256, dx=4e-5, amp=2.0),
                            dt=5e-6, steps=50, sweeps=4, nodes=3, nu=2),
    "flame2d_512_n53": dict(mech=(53, 325), seed=1803, dim=2, grid=dict(n=512, dx=4e-5, amp=2.0),
                            dt=5e-6, steps=20, sweeps=6, nodes=3, nu=2),
    "flame3d_128_n21": dict(mech=(21, 84), seed=1802, dim=3, grid=dict(n=128, dx=1e-4, urms=3.0),
                            dt=5e-6, steps=10, sweeps=4, nodes=3, nu=2),
}


# Batched form: independent 2D flames of uneven size and mechanism.
BATCHES = {
    "batch64_2d": dict(n_flames=64, seed=1804, side_log2=(5.0, 8.0), dx=4e-5, amp=2.0,
                       mechs=((1801, 9, 21), (1802, 21, 84), (1803, 53, 325)),
                       dt=(1e-6, 1e-5), radius=(1e-3, 3e-3), steps=10, sweeps=4, nodes=3, nu=2),
}


def build_batch(name: str = "batch64_2d", n_flames: int | None = None):
    """List of (mechanism, flame, dt) of a batched workload.

    Grid side n = round(2^U[5,8]) (cells 32^2..256^2, log-uniform side), mechanism
    drawn uniformly from the three, dt ~ U[1e-6, 1e-5] s, kernel centre uniform in
    the periodic box and radius ~ U[1, 3] mm clipped to 0.3 L (so that every
    flame keeps a front), front width min(0.2 mm, L/16).
    """
    b = BATCHES[name]
    rng = np.random.default_rng(b["seed"])
    mechs = [make_mechanism(*m) for m in b["mechs"]]
    out = []
    for f in range(b["n_flames"] if n_flames is None else n_flames):
        side = int(round(2.0 ** rng.uniform(*b["side_log2"])))
        mech = mechs[int(rng.integers(len(mechs)))]
        dt = float(rng.uniform(*b["dt"]))
        L = side * b["dx"]
        radius = min(float(rng.uniform(*b["radius"])), 0.3 * L)
        centre = (float(rng.uniform(0, L)), float(rng.uniform(0, L)))
        fl = flame_2d(mech, b["seed"] + f, n=side, dx=b["dx"], amp=b["amp"], radius=radius,
                      delta=min(2e-4, L / 16), centre=centre)
        out.append((mech, fl, dt))
    return out


def build_workload(name: str, grid_override: dict | None = None):
    """Mechanism and flame of a named workload (optionally on a smaller grid)."""
    w = WORKLOADS[name]
    mech = make_mechanism(w["seed"], *w["mech"])
    g = dict(w["grid"])
    if grid_override:
        g.update(grid_override)
    if w["dim"] == 1:
        fl = flame_1d(mech, w["seed"], **g)
    elif w["dim"] == 2:
        fl = flame_2d(mech, w["seed"], **g)
    else:
        fl = flame_3d(mech, w["seed"], **g)
    return mech, fl, w


def tiny_mechanism(seed=7):
    """3-species, 2-reaction mechanism for brute-force checks."""
    return make_mechanism(seed, 3, 2)
