"""The allocation-free reaction solve, against the allocating one.

misdc_reaction_solve_noalloc serves callers that cannot allocate device memory
during a call: it takes its scratch from a static device array instead of
cudaMallocAsync. It must give the results of misdc_reaction_solve, on two calls
in a row (the shared array keeps the previous call's contents), and refuse
sizes beyond the array. This file is collected last so a failure here comes
after every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1801_01201_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _p(t):
    return C.c_void_p(t.data_ptr())


def test_noalloc_reaction_solve_matches_allocating_entry_point_twice():
    from paper_1801_01201_gb300 import _lib as L
    from paper_1801_01201_gb300.solver import Solver
    mech = I.make_mechanism(1802, 21, 84)
    n = 200
    fl = I.flame_1d(mech, 0, nx=n, dx=1e-4)
    sv = Solver(mech, fl)
    lib = L.load()
    N = mech.n_species
    rng = np.random.default_rng(11)
    b = torch.as_tensor(fl.Y * (1 + 0.02 * rng.standard_normal(fl.Y.shape)), device="cuda").contiguous()
    hstar = sv.enthalpy(fl.Y, fl.T)
    x0 = torch.as_tensor(np.concatenate([fl.Y, fl.T[None, :]], axis=0), device="cuda").contiguous()
    wdt = 5e-6 / 4
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    x_ref = x0.clone()
    fr_ref = torch.empty((N, n), dtype=torch.float64, device="cuda")
    it_ref = torch.zeros(n, dtype=torch.int32, device="cuda")
    L.check(lib.misdc_reaction_solve(sv.handle, wdt, _p(b), _p(hstar), _p(x_ref), _p(fr_ref), _p(it_ref), n, stream))
    torch.cuda.synchronize()
    assert bool((it_ref > 0).all())

    for call in range(2):
        x = x0.clone()
        fr = torch.full((N, n), float("nan"), dtype=torch.float64, device="cuda")
        it = torch.zeros(n, dtype=torch.int32, device="cuda")
        L.check(lib.misdc_reaction_solve_noalloc(sv.handle, wdt, _p(b), _p(hstar), _p(x), _p(fr), _p(it), n, stream))
        torch.cuda.synchronize()
        assert bool((it > 0).all()), call
        rel = (x - x_ref).abs().amax(dim=1) / x_ref.abs().amax(dim=1)
        assert float(rel.max()) <= 1e-10, (call, rel)
        relf = (fr - fr_ref).abs().max() / fr_ref.abs().max()
        assert float(relf) <= 1e-10, call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1801_01201_gb300 import _lib as L
    from paper_1801_01201_gb300.solver import Solver
    mech = I.make_mechanism(1802, 21, 84)
    fl = I.flame_1d(mech, 0, nx=16, dx=1e-4)
    sv = Solver(mech, fl)
    lib = L.load()
    N = mech.n_species
    # the array holds 2^19 doubles: 32 for the counters and N + 1 per cell
    n_max = ((1 << 19) - 32) // (N + 1)
    assert n_max == 23829
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = lib.misdc_reaction_solve_noalloc(sv.handle, 1e-6, _p(dummy), _p(dummy), _p(dummy), None, None,
                                          n_max + 1, C.c_void_p(0))
    assert rc == L.E_INVALID
    assert b"no-allocation scratch" in lib.misdc_last_error()
    assert b"at most %d cells" % n_max in lib.misdc_last_error()
    # exactly at the limit the call is accepted and solves every cell
    fl2 = I.flame_1d(mech, 0, nx=n_max, dx=1e-4)
    sv2 = Solver(mech, fl2)
    b = torch.as_tensor(fl2.Y, device="cuda").contiguous()
    hstar = sv2.enthalpy(fl2.Y, fl2.T)
    x = torch.as_tensor(np.concatenate([fl2.Y, fl2.T[None, :]], axis=0), device="cuda").contiguous()
    it = torch.zeros(n_max, dtype=torch.int32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    L.check(lib.misdc_reaction_solve_noalloc(sv2.handle, 1e-7, _p(b), _p(hstar), _p(x), None, _p(it), n_max,
                                             stream))
    torch.cuda.synchronize()
    assert bool((it > 0).all())
