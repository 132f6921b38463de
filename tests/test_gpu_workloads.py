"""GPU parity at the benchmark workloads' own sizes and shapes.

* The 256^2 flame with the 21-species / 84-reaction mechanism, at full size: one
  time step, FP64 and mixed precision, against the oracle on every cell.
* A 24^3 periodic box of the 3D recipe (the same mechanism and seed, dx = 1e-4 m,
  the random-phase solenoidal field of rms 3 m/s, a spherical kernel with the
  workload's front width), one step, FP64 and mixed.
* Four flames drawn from the 64-flame batch (its four smallest: both 53-species
  flames among them, one of each other mechanism, each with its own dt), stepped
  together as an autotuned batch, FP64 and mixed.

The oracle's runs (reference and four one-ulp perturbed inputs per flame) start
in worker processes when the module's first test asks for them, while the GPU
works. Bounds as in test_gpu_parity: max(1e-10, 2 S_f) per field in FP64; the
mixed bar per species; T to 1e-10 (FP64, or 2 S) and 1e-6 (mixed).
"""
import numpy as np
import pytest

import oracle as O
from oracle.parallel import StepPool
from paper_1801_01201_gb300 import inputs as I
from parity_util import TOL, mixed_bar, record, relerr, tol_from

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BATCH_PICK = 4


def _cases():
    out = {}
    mech, fl, w = I.build_workload("flame2d_256_n21")
    out["flame2d_256_n21"] = [(mech, fl, w["dt"])]
    m3 = I.make_mechanism(1802, 21, 84)
    n = 24
    f3 = I.flame_3d(m3, 1802, n=n, dx=1e-4, urms=3.0, radius=0.3 * n * 1e-4, delta=2e-4)
    out["flame3d_box24_n21"] = [(m3, f3, 5e-6)]
    batch = I.build_batch("batch64_2d")
    order = sorted(range(len(batch)), key=lambda k: batch[k][1].cells)[:BATCH_PICK]
    out["batch64_2d_pick4"] = [batch[k] for k in order]
    return out


@pytest.fixture(scope="module")
def oracle_runs():
    cases = _cases()
    pool = StepPool()
    handles = {}
    for name, entries in cases.items():
        handles[name] = []
        for mech, fl, dt in entries:
            ad = O.ADR(mech, fl)
            phi0 = ad.state_from_YT(fl.Y, fl.T)
            handles[name].append(pool.step(mech, fl, phi0, dt, "CISDCQ", 2, 4, 2, 1, perturb=4))
    results = {}

    def get(name):
        if name not in results:
            results[name] = [pool.sensitivity(h) for h in handles[name]]
        return cases[name], results[name]
    yield get
    pool.close()


def _solver(mech, fl, precision, tune=False, dt=None):
    from paper_1801_01201_gb300.solver import Solver
    sv = Solver(mech, fl, precision=precision)
    x = sv.state_from_YT(fl.Y, fl.T)
    if tune:
        sv.autotune(x, torch.as_tensor(fl.T, device="cuda").contiguous(), dt)
    return sv, x


def _check(name, mech, fl, got, want, sens, precision, st):
    N = mech.n_species
    assert st["status_name"] == "OK", st
    assert st["newton_floor_stops"] == 0, st
    err = relerr(got, want)
    ad = O.ADR(mech, fl)
    T_want = ad.T_from_h(want[:N], want[N])
    T_got = ad.T_from_h(got[:N], got[N])
    eT = relerr(T_got, T_want)
    record(name, precision=precision, err=err, S=sens, errT=eT, scale=np.max(np.abs(want), axis=1),
           cells=fl.cells)
    if precision == "fp64":
        assert np.all(err <= tol_from(sens)), (err, sens)
        assert eT <= max(TOL, 2 * sens.max()), eT
    else:
        mixed_bar(got, want, sens, N)
        assert eT <= 1e-6, eT


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_2d_step_matches_oracle(oracle_runs, precision):
    (entries, res) = oracle_runs("flame2d_256_n21")
    mech, fl, dt = entries[0]
    sv, x = _solver(mech, fl, precision)
    sv.step(x, dt, 1)
    torch.cuda.synchronize()
    st = sv.stats()
    want, _, sens = res[0]
    _check("flame2d_256_n21", mech, fl, x.cpu().numpy(), want, sens, precision, st)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_3d_turbulent_box_step_matches_oracle(oracle_runs, precision):
    (entries, res) = oracle_runs("flame3d_box24_n21")
    mech, fl, dt = entries[0]
    sv, x = _solver(mech, fl, precision)
    sv.step(x, dt, 1)
    torch.cuda.synchronize()
    st = sv.stats()
    want, _, sens = res[0]
    _check("flame3d_box24_n21", mech, fl, x.cpu().numpy(), want, sens, precision, st)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_flames_step_matches_oracle(oracle_runs, precision):
    from paper_1801_01201_gb300.solver import Batch
    (entries, res) = oracle_runs("batch64_2d_pick4")
    solvers, states = [], []
    for mech, fl, dt in entries:
        sv, x = _solver(mech, fl, precision, tune=True, dt=dt)
        solvers.append(sv)
        states.append(x)
    B = Batch(solvers)
    B.step(states, [dt for _, _, dt in entries], 1)
    torch.cuda.synchronize()
    st = B.stats()
    for k, ((mech, fl, dt), (want, _, sens), x) in enumerate(zip(entries, res, states)):
        _check("batch64_2d_pick4[%d:%d species]" % (k, mech.n_species), mech, fl, x.cpu().numpy(), want,
               sens, precision, st)
