"""GPU tests of the adaptive number of nested iterations (opts.nu_eta/nu_rho_stall,
the reading of the future-work rule of Sec. 4 and 5 that the oracle pins):
captured steps take the decision on the device (IF graph nodes nested per
iteration), eager steps on the host; both must match the oracle's decisions and
results, and each other bit for bit."""
import numpy as np
import pytest

import oracle as O
from paper_1801_01201_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MILD = (8.0, 11.0)


def S():
    from paper_1801_01201_gb300 import solver
    return solver


def relerr(a, b):
    return np.max(np.abs(a - b), axis=1) / np.maximum(np.max(np.abs(b), axis=1), 1e-300)


def _flame(n=16):
    mech = I.make_mechanism(1802, 21, 84, logA_range=MILD)
    fl = I.flame_2d(mech, 0, n=n, dx=4e-5, radius=n * 4e-5 / 4, delta=2 * 4e-5)
    return mech, fl


def _gpu(mech, fl, phi0, steps, rule, nu=5, **kw):
    sv = S().Solver(mech, fl, nu=nu, nu_rule=rule, **kw)
    x = torch.as_tensor(phi0, device="cuda").contiguous()
    sv.step(x, 5e-6, steps)
    torch.cuda.synchronize()
    return x.cpu().numpy(), sv.stats()


@pytest.mark.parametrize("rule", [(0.02, 0.9), (1e-3, 0.9), (0.3, 0.5)])
def test_adaptive_nu_matches_oracle(rule):
    mech, fl = _flame()
    ad = O.ADR(mech, fl)
    phi0 = ad.state_from_YT(fl.Y, fl.T)
    used = []
    want, _ = ad.step(phi0, 5e-6, "CISDCQ", 2, 4, 5, n_steps=2, nu_rule=rule, nu_used_out=used)
    got, st = _gpu(mech, fl, phi0, 2, rule)
    assert st["status_name"] == "OK", st
    assert st["nested_iterations"] == int(sum(int(np.sum(u)) for u in used))
    assert np.all(relerr(got, want) < 1e-10)


@pytest.mark.parametrize("two_streams", [True, False])
def test_adaptive_nu_graph_equals_eager(two_streams):
    mech, fl = _flame()
    phi0 = O.ADR(mech, fl).state_from_YT(fl.Y, fl.T)
    a, sa = _gpu(mech, fl, phi0, 2, (0.02, 0.9), use_graph=True, two_streams=two_streams)
    b, sb = _gpu(mech, fl, phi0, 2, (0.02, 0.9), use_graph=False, two_streams=two_streams)
    assert np.array_equal(a, b)
    assert sa["nested_iterations"] == sb["nested_iterations"] > 0
    assert sa["kernel_launches"] > 0


def test_adaptive_nu_with_mixed_precision_and_multigrid():
    """IF bodies holding the multigrid WHILE loops and the mixed-precision
    reaction solves: graph and eager steps agree bit for bit, within the mixed
    bar of the oracle's adaptive result."""
    mech, fl = _flame()
    ad = O.ADR(mech, fl)
    phi0 = ad.state_from_YT(fl.Y, fl.T)
    used = []
    want, _ = ad.step(phi0, 5e-6, "CISDCQ", 2, 4, 5, n_steps=2, nu_rule=(1e-3, 0.9), nu_used_out=used)
    kw = dict(precision="mixed", mg_levels=3)
    a, sa = _gpu(mech, fl, phi0, 2, (1e-3, 0.9), use_graph=True, **kw)
    b, sb = _gpu(mech, fl, phi0, 2, (1e-3, 0.9), use_graph=False, **kw)
    assert sa["status_name"] == "OK", sa
    assert np.array_equal(a, b)
    assert sa["nested_iterations"] == int(sum(int(np.sum(u)) for u in used))
    N = mech.n_species
    assert np.max(np.abs(a[:N] - want[:N])) / np.max(np.abs(want[:N])) < 1e-8


def test_adaptive_nu_in_a_batch_equals_single():
    mech, fl = _flame()
    phi0 = O.ADR(mech, fl).state_from_YT(fl.Y, fl.T)
    single, _ = _gpu(mech, fl, phi0, 2, (0.02, 0.9))
    svs = [S().Solver(mech, fl, nu=5, nu_rule=(0.02, 0.9)), S().Solver(mech, fl)]
    xs = [torch.as_tensor(phi0, device="cuda").contiguous() for _ in svs]
    B = S().Batch(svs)
    B.step(xs, [5e-6, 5e-6], 2)
    torch.cuda.synchronize()
    assert B.stats()["status_name"] == "OK"
    assert np.array_equal(xs[0].cpu().numpy(), single)


def test_adaptive_rule_requires_contraction_bound():
    mech, fl = _flame(8)
    from paper_1801_01201_gb300 import _lib as L
    with pytest.raises(L.MisdcError):
        S().Solver(mech, fl, nu=4, nu_rule=(0.1, 0.0))
