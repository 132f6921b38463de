"""Python binding of the C ABI: argument marshalling around libmisdc.

Every step of the method runs in the CUDA library; PyTorch only provides
device memory and streams.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(t.ctypes.data)
    raise TypeError("expected a torch tensor or numpy array")


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dev(a, device):
    if isinstance(a, torch.Tensor):
        return a.to(device=device, dtype=torch.float64).contiguous()
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=device)


def lobatto(n_nodes):
    """tau, Q, QI, QE as the CUDA library builds them."""
    lib = L.load()
    M = n_nodes - 1
    tau = np.zeros(M + 1)
    Q = np.zeros((M, M + 1))
    QI = np.zeros((M, M))
    QE = np.zeros((M, M))
    L.check(lib.misdc_lobatto(n_nodes, tau.ctypes.data_as(L.dp), Q.ctypes.data_as(L.dp),
                              QI.ctypes.data_as(L.dp), QE.ctypes.data_as(L.dp)))
    return tau, Q, QI, QE


def exp(x, stream=None):
    """e^x with the FP64 exponential the rate kernels use (misdc_exp); x a device tensor."""
    lib = L.load()
    x = x.to(torch.float64).contiguous()
    y = torch.empty_like(x)
    L.check(lib.misdc_exp(_ptr(x), _ptr(y), x.numel(), _stream(stream)))
    return y


PROBE_KINDS = {"dfma": 0, "dmma": 1, "ffma": 2}


def probe_flops(kind, blocks, iters, stream=None):
    """Launch the arithmetic-throughput probe (misdc_probe_flops) on `stream`;
    returns (the flops the launch performs, its output tensor)."""
    lib = L.load()
    out = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    fl = C.c_double()
    L.check(lib.misdc_probe_flops(PROBE_KINDS[kind], blocks, iters, _ptr(out), C.byref(fl), _stream(stream)))
    return fl.value, out


PDE_STATUS_BITS = {1: "newton_limit", 2: "non_finite", 4: "singular_diffusion"}


def pde_step(phi, params, dt, *, length=20.0, scheme="CISDCQ", n_nodes=5, n_sweeps=4, nu=1,
             n_steps=1, stream=None):
    """Advance n instances of the nonlinear test PDE of Sec. 5.2 (misdc_pde_step).

    phi: [n, nx] or [nx] FP64 device tensor of cell averages; params: [n, 5] or [5]
    (a, d, r, left, right). Returns (phi_out [n, nx], incr [n, n_steps, n_sweeps],
    status [n]) as device tensors (status bits: PDE_STATUS_BITS)."""
    lib = L.load()
    one = phi.dim() == 1
    phi = phi.reshape(1, -1) if one else phi
    n, nx = phi.shape
    dev = phi.device
    phi = _dev(phi, dev)
    params = _dev(params, dev).reshape(-1, 5)
    if params.shape[0] == 1 and n > 1:
        params = params.expand(n, 5).contiguous()
    if params.shape[0] != n:
        raise ValueError("params must have one row per instance")
    out = torch.empty_like(phi)
    incr = torch.empty((n, n_steps, n_sweeps), dtype=torch.float64, device=dev)
    status = torch.zeros(n, dtype=torch.int32, device=dev)
    L.check(lib.misdc_pde_step(L.SCHEMES.get(scheme, scheme), n_nodes, n_sweeps, nu, dt, n_steps,
                               nx, length, n, _ptr(params), _ptr(phi), _ptr(out), _ptr(incr),
                               _ptr(status), _stream(stream)))
    if one:
        return out[0], incr[0], status[0]
    return out, incr, status


def pde_smem_bytes(n_nodes, nx):
    """Shared memory one instance of pde_step needs (bytes)."""
    lib = L.load()
    b = C.c_size_t(0)
    L.check(lib.misdc_pde_smem_bytes(n_nodes, nx, C.byref(b)))
    return b.value


def lincomb(outs, ins, w, n, stream=None):
    """out[o] = sum_k w[o][k] in[k] over n elements (device tensors)."""
    lib = L.load()
    w = np.ascontiguousarray(w, dtype=np.float64)
    op = (C.c_void_p * len(outs))(*[t.data_ptr() for t in outs])
    ip = (C.c_void_p * len(ins))(*[t.data_ptr() for t in ins])
    L.check(lib.misdc_lincomb(len(outs), len(ins), op, ip, w.ctypes.data_as(L.dp), n, _stream(stream)))


class Solver:
    """One flame: mechanism + periodic grid + face velocities + time-integration options."""

    def __init__(self, mech, flame, *, n_nodes=3, n_sweeps=4, nu=2, scheme="CISDCQ",
                 precision="fp64", newton_rtol=1e-12, newton_maxit=50, lin_rtol=1e-14,
                 mg_levels=1, two_streams=True, use_graph=True, profile=False, rates_mma=False,
                 nu_rule=None, lanes=1, lin_rounds=0, device="cuda"):
        self.lib = L.load()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.device = torch.device(device)
        self.mech, self.flame = mech, flame
        self.N = mech.n_species
        self.cells = flame.nx * flame.ny * flame.nz
        k = dict(W=np.ascontiguousarray(mech.W, np.float64), nasa7=np.ascontiguousarray(mech.nasa7, np.float64),
                 A=np.ascontiguousarray(mech.A, np.float64), beta=np.ascontiguousarray(mech.beta, np.float64),
                 Ea=np.ascontiguousarray(mech.Ea, np.float64), nu_f=np.ascontiguousarray(mech.nu_f, np.int32),
                 nu_r=np.ascontiguousarray(mech.nu_r, np.int32), D0=np.ascontiguousarray(mech.D0, np.float64))
        self._keep = k
        md = L.MechDesc(self.N, mech.n_reactions, k["W"].ctypes.data_as(L.dp), k["nasa7"].ctypes.data_as(L.dp),
                        k["A"].ctypes.data_as(L.dp), k["beta"].ctypes.data_as(L.dp),
                        k["Ea"].ctypes.data_as(L.dp), k["nu_f"].ctypes.data_as(L.ip),
                        k["nu_r"].ctypes.data_as(L.ip), k["D0"].ctypes.data_as(L.dp),
                        mech.alpha0, mech.T_ref, mech.theta_exp, mech.p_ref)
        gd = L.GridDesc(flame.dim, flame.nx, flame.ny, flame.nz, flame.dx)
        o = L.Opts()
        self.lib.misdc_default_opts(C.byref(o))
        o.n_nodes, o.n_sweeps, o.nu = n_nodes, n_sweeps, nu
        o.scheme = L.SCHEMES[scheme]
        o.precision = L.PRECISIONS[precision]
        o.dominant_species = flame.dominant
        o.rho = flame.rho
        o.newton_rtol, o.newton_maxit, o.lin_rtol = newton_rtol, newton_maxit, lin_rtol
        o.mg_levels = mg_levels
        o.two_streams, o.use_graph = int(two_streams), int(use_graph)
        o.profile = int(profile)
        o.rates_mma = int(rates_mma)
        o.lanes = int(lanes)
        o.lin_rounds = int(lin_rounds)
        if nu_rule is not None:   # (eta, rho_stall): adaptive nested iterations, nu the cap
            o.nu_eta, o.nu_rho_stall = float(nu_rule[0]), float(nu_rule[1])
        self.opts = o
        vel = _dev(flame.vel, self.device)
        h = C.c_void_p()
        L.check(self.lib.misdc_create(C.byref(md), C.byref(gd), C.byref(o), _ptr(vel), C.byref(h)))
        self.handle = h
        torch.cuda.synchronize()

    def close(self):
        if getattr(self, "handle", None):
            self.lib.misdc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state helpers ------------------------------------------------------
    def enthalpy(self, Y, T, stream=None):
        Y = _dev(Y, self.device)
        T = _dev(T, self.device)
        n = T.numel()
        h = torch.empty(n, dtype=torch.float64, device=self.device)
        L.check(self.lib.misdc_enthalpy(self.handle, _ptr(Y), _ptr(T), _ptr(h), n, _stream(stream)))
        return h

    def temperature(self, Y, h, T_guess=None, stream=None):
        Y = _dev(Y, self.device)
        h = _dev(h, self.device)
        n = h.numel()
        T = (_dev(T_guess, self.device).clone() if T_guess is not None
             else torch.full((n,), -1.0, dtype=torch.float64, device=self.device))
        L.check(self.lib.misdc_temperature(self.handle, _ptr(Y), _ptr(h), _ptr(T), n, _stream(stream)))
        return T

    def state_from_YT(self, Y, T):
        """Device state [N+1, cells] = (Y, h(T)) with h from the library's thermo."""
        Y = _dev(Y, self.device)
        h = self.enthalpy(Y, T)
        return torch.cat([Y, h[None, :]], dim=0).contiguous()

    # -- time stepping ------------------------------------------------------
    def step(self, state, dt, n_steps=1, T=None, stream=None):
        L.check(self.lib.misdc_step(self.handle, _ptr(state), _ptr(T), float(dt), int(n_steps),
                                    _stream(stream)))
        return state

    def step_host(self, state_host, dt, n_steps=1, T_host=None, stream=None):
        L.check(self.lib.misdc_step_host(self.handle, _ptr(state_host), _ptr(T_host), float(dt),
                                         int(n_steps), _stream(stream)))
        return state_host

    def stats(self, reset=True):
        st = L.Stats()
        L.check(self.lib.misdc_get_stats(self.handle, C.byref(st), int(reset)))
        return st.as_dict()

    def stage_times(self):
        tn, td = C.c_double(), C.c_double()
        nn, nd = C.c_int(), C.c_int()
        L.check(self.lib.misdc_stage_times(self.handle, C.byref(tn), C.byref(nn), C.byref(td), C.byref(nd)))
        return dict(newton_ms=tn.value, newton_launches=nn.value, diffusion_ms=td.value,
                    diffusion_launches=nd.value)

    # -- variable-density low-Mach step of independent 1D flames -------------
    def lowmach_step(self, q, dt, Y_in, T_in, U_in, p0=101325.0, dchi=True, n_steps=1, stream=None):
        """Advance the 1D low-Mach states q ([n, N+2, nx] or [N+2, nx], device or
        host) n_steps steps (misdc_lowmach_step, one call per step); returns
        (q, p_eos, status) as device tensors."""
        one = q.dim() == 2 if isinstance(q, torch.Tensor) else np.ndim(q) == 2
        q = _dev(q, self.device)
        if one:
            q = q[None]
        q = q.contiguous().clone()
        n, nx = q.shape[0], q.shape[2]
        y_in = np.ascontiguousarray(Y_in, dtype=np.float64)
        d = L.LowMachDesc(float(U_in), float(T_in), float(p0), y_in.ctypes.data_as(L.dp), 1 if dchi else 0)
        pe = torch.empty((n, nx), dtype=torch.float64, device=self.device)
        status = torch.zeros(n, dtype=torch.int32, device=self.device)
        st = torch.zeros_like(status)
        for _ in range(n_steps):
            L.check(self.lib.misdc_lowmach_step(self.handle, C.byref(d), float(dt), n, _ptr(q), _ptr(q),
                                                _ptr(pe), _ptr(st), _stream(stream)))
            status |= st
        if one:
            return q[0], pe[0], status[0]
        return q, pe, status

    # -- row-level entry points --------------------------------------------
    def production_rates(self, Y, T, stream=None):
        Y = _dev(Y, self.device)
        T = _dev(T, self.device)
        n = T.numel()
        FR = torch.empty((self.N, n), dtype=torch.float64, device=self.device)
        L.check(self.lib.misdc_production_rates(self.handle, _ptr(Y), _ptr(T), _ptr(FR), n, _stream(stream)))
        return FR

    def reaction_solve(self, wdt, b, hstar, x0, stream=None):
        b = _dev(b, self.device)
        hstar = _dev(hstar, self.device)
        x = _dev(x0, self.device).clone()
        n = hstar.numel()
        FR = torch.empty((self.N, n), dtype=torch.float64, device=self.device)
        it = torch.zeros(n, dtype=torch.int32, device=self.device)
        L.check(self.lib.misdc_reaction_solve(self.handle, float(wdt), _ptr(b), _ptr(hstar), _ptr(x),
                                              _ptr(FR), _ptr(it), n, _stream(stream)))
        return x, FR, it

    def operators(self, state, stream=None):
        state = _dev(state, self.device)
        FE = torch.empty_like(state)
        FD = torch.empty_like(state)
        FR = torch.empty_like(state)
        L.check(self.lib.misdc_operators(self.handle, _ptr(state), _ptr(FE), _ptr(FD), _ptr(FR),
                                         _stream(stream)))
        return FE, FD, FR

    def diffusion_solve(self, wdt, coef_state, rhs, stream=None):
        coef_state = _dev(coef_state, self.device)
        rhs = _dev(rhs, self.device)
        x = torch.empty_like(rhs)
        L.check(self.lib.misdc_diffusion_solve(self.handle, float(wdt), _ptr(coef_state), _ptr(rhs),
                                               _ptr(x), _stream(stream)))
        return x

    # -- launch shapes ------------------------------------------------------
    def autotune(self, state, T, dt):
        t = L.Tuning()
        L.check(self.lib.misdc_autotune(self.handle, _ptr(state), _ptr(T), float(dt), C.byref(t)))
        return t.as_dict()

    def get_tuning(self):
        t = L.Tuning()
        L.check(self.lib.misdc_get_tuning(self.handle, C.byref(t)))
        return t.as_dict()

    def set_tuning(self, **kw):
        t = L.Tuning()
        L.check(self.lib.misdc_get_tuning(self.handle, C.byref(t)))
        for k, v in kw.items():
            setattr(t, k, v)
        L.check(self.lib.misdc_set_tuning(self.handle, C.byref(t)))

    # -- learned initial guess of the reaction Newton ------------------------
    def surrogate_dims(self):
        v = [C.c_int() for _ in range(5)]
        n = C.c_size_t()
        L.check(self.lib.misdc_surrogate_dims(self.handle, *[C.byref(x) for x in v], C.byref(n)))
        n_in, ldx, hid, n_out, ldo = (x.value for x in v)
        return dict(n_in=n_in, ldx=ldx, n_hidden=hid, n_out=n_out, ldo=ldo, n_params=n.value)

    def surrogate_init(self, seed=0):
        L.check(self.lib.misdc_surrogate_init(self.handle, int(seed)))

    def surrogate_load(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        L.check(self.lib.misdc_surrogate_load(self.handle, p.ctypes.data_as(C.POINTER(C.c_float)), p.size))

    def surrogate_save(self):
        p = np.zeros(self.surrogate_dims()["n_params"], dtype=np.float32)
        L.check(self.lib.misdc_surrogate_save(self.handle, p.ctypes.data_as(C.POINTER(C.c_float)), p.size))
        return p

    def surrogate_enable(self, on=True, s_min=1e-8):
        L.check(self.lib.misdc_surrogate_enable(self.handle, int(bool(on)), float(s_min)))

    def surrogate_sweeps(self, n_sweeps):
        """Use the learned guess only in the first n_sweeps sweeps of a step (0: all)."""
        L.check(self.lib.misdc_surrogate_sweeps(self.handle, int(n_sweeps)))

    def surrogate_collect(self, capacity):
        L.check(self.lib.misdc_surrogate_collect(self.handle, int(capacity)))

    def surrogate_dataset(self):
        """(rows, X bf16 [rows, ldx] as int16 bits, targets f32 [rows, ldo]) copied to torch."""
        rows = C.c_longlong()
        xp, tp = C.c_void_p(), C.c_void_p()
        L.check(self.lib.misdc_surrogate_dataset(self.handle, C.byref(rows), C.byref(xp), C.byref(tp)))
        d = self.surrogate_dims()
        r = rows.value
        if r == 0:
            return 0, None, None
        X = _wrap_device(xp.value, (r, d["ldx"]), "<i2").clone().view(torch.bfloat16)
        T = _wrap_device(tp.value, (r, d["ldo"]), "<f4").clone()
        return r, X, T

    def surrogate_train(self, steps, batch=4096, lr=1e-3, weight_decay=1e-4, seed=0):
        curve = np.zeros(int(steps), dtype=np.float32)
        L.check(self.lib.misdc_surrogate_train(self.handle, int(steps), int(batch), float(lr),
                                               float(weight_decay), int(seed),
                                               curve.ctypes.data_as(C.POINTER(C.c_float))))
        return curve

    def surrogate_features(self, wdt, b, hstar, Yp, Tp, FRp, hp, stream=None):
        d = self.surrogate_dims()
        b, hstar, Yp, Tp, FRp, hp = (_dev(a, self.device) for a in (b, hstar, Yp, Tp, FRp, hp))
        n = hstar.numel()
        X = torch.empty((n, d["ldx"]), dtype=torch.bfloat16, device=self.device)
        sc = torch.empty(n, dtype=torch.float64, device=self.device)
        L.check(self.lib.misdc_surrogate_features(self.handle, float(wdt), _ptr(b), _ptr(hstar), _ptr(Yp),
                                                  _ptr(Tp), _ptr(FRp), _ptr(hp), n, _ptr(X), _ptr(sc),
                                                  _stream(stream)))
        return X, sc

    def surrogate_forward(self, X, stream=None):
        d = self.surrogate_dims()
        X = X.to(device=self.device, dtype=torch.bfloat16).contiguous()
        out = torch.empty((X.shape[0], d["ldo"]), dtype=torch.float32, device=self.device)
        L.check(self.lib.misdc_surrogate_forward(self.handle, _ptr(X), X.shape[0], _ptr(out), _stream(stream)))
        return out

    def surrogate_forward_layers(self, X, stream=None):
        d = self.surrogate_dims()
        X = X.to(device=self.device, dtype=torch.bfloat16).contiguous()
        out = torch.empty((X.shape[0], d["ldo"]), dtype=torch.float32, device=self.device)
        L.check(self.lib.misdc_surrogate_forward_layers(self.handle, _ptr(X), X.shape[0], _ptr(out),
                                                        _stream(stream)))
        return out

    def surrogate_guess(self, wdt, b, hstar, Yp, Tp, FRp, hp, stream=None):
        d = self.surrogate_dims()
        b, hstar, Yp, Tp, FRp, hp = (_dev(a, self.device) for a in (b, hstar, Yp, Tp, FRp, hp))
        n = hstar.numel()
        out = torch.empty((n, d["ldo"]), dtype=torch.float32, device=self.device)
        sc = torch.empty(n, dtype=torch.float64, device=self.device)
        L.check(self.lib.misdc_surrogate_guess(self.handle, float(wdt), _ptr(b), _ptr(hstar), _ptr(Yp),
                                               _ptr(Tp), _ptr(FRp), _ptr(hp), n, _ptr(out), _ptr(sc),
                                               _stream(stream)))
        return out, sc

    def surrogate_gradient(self, X, targets, stream=None):
        d = self.surrogate_dims()
        X = X.to(device=self.device, dtype=torch.bfloat16).contiguous()
        t = targets.to(device=self.device, dtype=torch.float32).contiguous()
        g = torch.empty(d["n_params"], dtype=torch.float32, device=self.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        L.check(self.lib.misdc_surrogate_gradient(self.handle, _ptr(X), _ptr(t), X.shape[0], _ptr(g),
                                                  _ptr(loss), _stream(stream)))
        return g, loss

    def surrogate_train_batch(self, X, targets, lr, weight_decay=0.0, stream=None):
        X = X.to(device=self.device, dtype=torch.bfloat16).contiguous()
        t = targets.to(device=self.device, dtype=torch.float32).contiguous()
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        L.check(self.lib.misdc_surrogate_train_batch(self.handle, _ptr(X), _ptr(t), X.shape[0], float(lr),
                                                     float(weight_decay), _ptr(loss), _stream(stream)))
        return loss



class Batch:
    """Independent flames advanced together, one CUDA graph launch per step;
    `grouping` (default on) merges the flames' k-th reaction steps of one
    mechanism shape into one load-balanced launch (misdc_batch_set_grouping)."""

    def __init__(self, solvers, grouping=True):
        self.lib = L.load()
        self.solvers = list(solvers)
        arr = (C.c_void_p * len(self.solvers))(*[s.handle.value for s in self.solvers])
        h = C.c_void_p()
        L.check(self.lib.misdc_batch_create(arr, len(self.solvers), C.byref(h)))
        self.handle = h
        if not grouping:
            self.set_grouping(False)

    def set_grouping(self, on):
        L.check(self.lib.misdc_batch_set_grouping(self.handle, 1 if on else 0))

    def grouping(self):
        """(grouped reaction launches per step, per-flame reaction steps they replace)
        of the current graph."""
        a, b = C.c_int(), C.c_int()
        L.check(self.lib.misdc_batch_grouping(self.handle, C.byref(a), C.byref(b)))
        return a.value, b.value

    def close(self):
        if getattr(self, "handle", None):
            self.lib.misdc_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, states, dts, n_steps=1, Ts=None, stream=None):
        n = len(self.solvers)
        sp = (C.c_void_p * n)(*[t.data_ptr() for t in states])
        tp = None if Ts is None else (C.c_void_p * n)(*[(t.data_ptr() if t is not None else None) for t in Ts])
        d = np.ascontiguousarray(dts, dtype=np.float64)
        L.check(self.lib.misdc_batch_step(self.handle, sp, tp, d.ctypes.data_as(L.dp), int(n_steps),
                                          _stream(stream)))
        return states

    def stats(self, reset=True):
        st = L.Stats()
        L.check(self.lib.misdc_batch_stats(self.handle, C.byref(st), int(reset)))
        return st.as_dict()


class _DeviceArray:
    """__cuda_array_interface__ view of library-owned device memory (no copy)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": tuple(shape),
                                         "typestr": typestr, "version": 3}


def _wrap_device(ptr, shape, typestr):
    torch.cuda.synchronize()
    return torch.as_tensor(_DeviceArray(ptr, shape, typestr), device="cuda")
