"""GPU tests of the launch-shape autotuner and of batched stepping.

Launch shapes and batching change scheduling only: every cell's Newton solve and
every smoother sweep compute the same operations in the same order, so results
are bitwise identical to the default single-flame path; the batched path is
also checked against the CPU oracle (1e-10 relative per field, mild chemistry).
"""
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


def _flames():
    m9 = I.make_mechanism(1801, 9, 21, logA_range=MILD)
    m21 = I.make_mechanism(1802, 21, 84, logA_range=MILD)
    m53 = I.make_mechanism(1803, 53, 325, logA_range=MILD)
    fl = [
        (m21, I.flame_2d(m21, 0, n=32, dx=4e-5, radius=3.2e-4, delta=8e-5, centre=(3e-4, 1e-4)), 5e-6),
        (m9, I.flame_1d(m9, 1801, nx=96, dx=1e-4), 1e-5),
        (m53, I.flame_2d(m53, 1, n=16, dx=4e-5, radius=1.6e-4, delta=8e-5), 2e-6),
        (m21, I.flame_2d(m21, 2, n=20, dx=4e-5, radius=2.0e-4, delta=8e-5), 7e-6),
    ]
    return fl


def _state(sv, fl):
    return sv.state_from_YT(fl.Y, fl.T)


def test_autotune_keeps_results_bitwise():
    mech, fl, dt = _flames()[0]
    a = S().Solver(mech, fl)
    b = S().Solver(mech, fl)
    s0 = _state(a, fl)
    T0 = torch.as_tensor(fl.T, device="cuda").contiguous()
    t = b.autotune(s0, T0, dt)
    assert 0 <= t["newton_warps_per_block"] <= 4 and t["newton_blocks_per_sm"] in (0, 4, 8, 16)
    assert t["cheb_block"] in (128, 256, 512) and t["newton_ms"] > 0 and t["cheb_ms"] > 0
    assert b.get_tuning()["cheb_block"] == t["cheb_block"]
    for shape in ({}, dict(newton_dynamic=1, newton_warps_per_block=1, newton_blocks_per_sm=16)):
        if shape:
            b.set_tuning(**shape)
        x, y = s0.clone(), s0.clone()
        a.step(x, dt, 2)
        b.step(y, dt, 2)
        assert torch.equal(x, y), shape
        assert b.stats()["status_name"] == "OK"


def test_batch_bitwise_equals_single_flames():
    fl = _flames()
    single = [S().Solver(m, f) for m, f, _ in fl]
    batched = [S().Solver(m, f) for m, f, _ in fl]
    # uneven launch shapes in the batch
    batched[0].set_tuning(newton_dynamic=1, newton_warps_per_block=1, newton_blocks_per_sm=16)
    batched[2].set_tuning(cheb_block=128)
    states = [_state(s, f) for s, (_, f, _) in zip(single, fl)]
    ref = [x.clone() for x in states]
    for s, x, (_, _, dt) in zip(single, ref, fl):
        s.step(x, dt, 3)
    got = [x.clone() for x in states]
    B = S().Batch(batched)
    B.step(got, [dt for _, _, dt in fl], 2)
    B.step(got, [dt for _, _, dt in fl], 1)     # graph replay
    st = B.stats()
    assert st["status_name"] == "OK" and st["kernel_launches"] > 0
    for x, y in zip(ref, got):
        assert torch.equal(x, y)


def test_batch_matches_oracle():
    fl = _flames()[:2]
    solvers = [S().Solver(m, f) for m, f, _ in fl]
    states, want = [], []
    for s, (m, f, dt) in zip(solvers, fl):
        ad = O.ADR(m, f)
        phi0 = ad.state_from_YT(f.Y, f.T)
        w, _ = ad.step(phi0, dt, "CISDCQ", 2, 4, 2, n_steps=2)
        want.append(w)
        states.append(torch.as_tensor(phi0, device="cuda").contiguous())
    B = S().Batch(solvers)
    B.step(states, [dt for _, _, dt in fl], 2)
    torch.cuda.synchronize()
    for x, w in zip(states, want):
        assert np.all(relerr(x.cpu().numpy(), w) < 1e-10)


def test_batch_rejects_bad_input():
    fl = _flames()[:1]
    s = S().Solver(fl[0][0], fl[0][1])
    from paper_1801_01201_gb300 import _lib as L
    with pytest.raises(L.MisdcError):
        S().Batch([s, s])
    B = S().Batch([s])
    x = _state(s, fl[0][1])
    with pytest.raises(L.MisdcError):
        B.step([x], [0.0], 1)


def test_batch_mixed_precision_bitwise_and_accurate():
    """Mixed precision (kept Jacobian factors, learned guess off) in a batch equals
    stepping each flame alone, and stays within the mixed bar of the FP64 oracle."""
    fl = _flames()[:3]
    single = [S().Solver(m, f, precision="mixed") for m, f, _ in fl]
    batched = [S().Solver(m, f, precision="mixed") for m, f, _ in fl]
    states = [_state(s, f) for s, (_, f, _) in zip(single, fl)]
    ref = [x.clone() for x in states]
    for s, x, (_, _, dt) in zip(single, ref, fl):
        s.step(x, dt, 2)
    got = [x.clone() for x in states]
    B = S().Batch(batched)
    B.step(got, [dt for _, _, dt in fl], 2)
    assert B.stats()["status_name"] == "OK"
    for x, y in zip(ref, got):
        assert torch.equal(x, y)
    m, f, dt = fl[0]
    ad = O.ADR(m, f)
    want, _ = ad.step(ad.state_from_YT(f.Y, f.T), dt, "CISDCQ", 2, 4, 2, n_steps=2)
    g = got[0].cpu().numpy()
    N = m.n_species
    assert np.max(np.abs(g[:N] - want[:N])) / np.max(np.abs(want[:N])) < 1e-8


def _small_batch(n_flames=64, seed=4242):
    """64 flames like the benchmark batch but on 16^2..32^2 grids: side
    U{16..32}, the three mechanisms with their full rate ranges (taken in turn),
    dt ~ U[1e-6, 1e-5] s, kernel centre uniform, radius 0.3 L, front width L/8."""
    rng = np.random.default_rng(seed)
    mechs = [I.make_mechanism(*k) for k in ((1801, 9, 21), (1802, 21, 84), (1803, 53, 325))]
    out = []
    for f in range(n_flames):
        side = int(rng.integers(16, 33))
        mech = mechs[f % 3]
        dt = float(rng.uniform(1e-6, 1e-5))
        L = side * 4e-5
        centre = (float(rng.uniform(0, L)), float(rng.uniform(0, L)))
        fl = I.flame_2d(mech, seed + f, n=side, dx=4e-5, amp=2.0, radius=0.3 * L, delta=L / 8, centre=centre)
        out.append((mech, fl, dt))
    return out


def test_batch_of_64_small_flames_autotuned():
    """64 uneven flames (16^2..32^2, 9/21, 21/84 and 53/325 species/reactions,
    each its own dt) in one autotuned batch equal stepping each flame alone with
    default launch shapes bit for bit, and three of them (one per mechanism)
    match the oracle within max(1e-10, 2 S) per field."""
    from oracle.parallel import StepPool
    from parity_util import record, tol_from
    fl = _small_batch()
    picks = [0, 1, 2]
    with StepPool() as pool:
        handles = []
        for k in picks:
            m, f, dt = fl[k]
            ad = O.ADR(m, f)
            handles.append(pool.step(m, f, ad.state_from_YT(f.Y, f.T), dt, "CISDCQ", 2, 4, 2, 1, perturb=4))
        single = [S().Solver(m, f) for m, f, _ in fl]
        batched = [S().Solver(m, f) for m, f, _ in fl]
        states = [_state(s, f) for s, (_, f, _) in zip(single, fl)]
        shapes = set()
        for s, x, (_, f, dt) in zip(batched, states, fl):
            t = s.autotune(x, torch.as_tensor(f.T, device="cuda").contiguous(), dt)
            shapes.add((t["newton_warps_per_block"], t["newton_blocks_per_sm"], t["newton_dynamic"],
                        t["cheb_block"]))
        ref = [x.clone() for x in states]
        for s, x, (_, _, dt) in zip(single, ref, fl):
            s.step(x, dt, 1)
        got = [x.clone() for x in states]
        B = S().Batch(batched)
        B.step(got, [dt for _, _, dt in fl], 1)
        st = B.stats()
        assert st["status_name"] == "OK", st
        assert st["newton_floor_stops"] == 0
        for k, (x, y) in enumerate(zip(ref, got)):
            assert torch.equal(x, y), k
        for k, h in zip(picks, handles):
            want, _, sens = pool.sensitivity(h)
            err = relerr(got[k].cpu().numpy(), want)
            record("batch64_small[%d:%d species]" % (k, fl[k][0].n_species), err=err, S=sens,
                   shapes=len(shapes))
            assert np.all(err <= tol_from(sens)), (k, err, sens)


@pytest.mark.parametrize("precision,learned", [("fp64", False), ("mixed", False), ("mixed", True)])
def test_grouped_reaction_steps_equal_separate_launches(precision, learned):
    """Grouping the flames' reaction steps (one persistent, load-balanced Newton
    launch per stage and mechanism shape) changes scheduling: twelve uneven flames
    (four per mechanism) against the batch with one launch per flame, with fewer
    kernel launches. In FP64 the states and Newton counts are equal bit for bit. In
    mixed precision the grouped kernel and the single-solve kernel are compiled
    separately, so the compiler may fuse a multiply and an add in one and not in
    the other; a certification decision near its threshold can then go the other
    way, and the states agree to the mixed-precision bar instead (every species
    within 1e-8 of its largest value, h within 1e-8; measured 2e-10). The learned
    case runs an untrained (random) network: every guess it makes is vetted, and a
    solve that fails from an accepted guess is repeated from the plain guess, so
    the status stays OK."""
    fl = _small_batch(n_flames=12, seed=777)
    dts = [dt for _, _, dt in fl]
    out, counts, launches = [], [], []
    for grouping in (True, False):
        svs = [S().Solver(m, f, precision=precision) for m, f, _ in fl]
        if learned:
            for s in svs:
                s.surrogate_init(seed=3)
                s.surrogate_enable(True, s_min=1e-4)
        states = [_state(s, f) for s, (_, f, _) in zip(svs, fl)]
        B = S().Batch(svs, grouping=grouping)
        B.step(states, dts, 2)
        B.step(states, dts, 1)   # graph replay
        st = B.stats()
        assert st["status_name"] == "OK", (grouping, st)
        g_launches, g_solves = B.grouping()
        if grouping:
            # 3 mechanism shapes x reaction steps per time step (2 nodes x nu 2 x 4 sweeps)
            assert g_launches == 3 * 16 and g_solves == 12 * 16, (g_launches, g_solves)
        else:
            assert (g_launches, g_solves) == (0, 0)
        out.append(states)
        counts.append((st["newton_solves"], st["newton_iters"], st["newton_jacobians"],
                       st["newton_certified"], st["surrogate_used"]))
        launches.append(st["kernel_launches"])
    if precision == "fp64":
        for k, (x, y) in enumerate(zip(*out)):
            assert torch.equal(x, y), k
        assert counts[0] == counts[1], counts
    else:
        worst = 0.0
        for k, ((m, _, _), x, y) in enumerate(zip(fl, *out)):
            rel = ((x - y).abs().amax(dim=1) / y.abs().amax(dim=1).clamp_min(1e-300)).cpu().numpy()
            worst = max(worst, float(rel.max()))
            assert np.all(rel <= 1e-8), (k, rel)
        print("grouped vs separate, worst per-field relative difference %.2e" % worst)
        assert counts[0][0] == counts[1][0], counts
        assert abs(counts[0][1] - counts[1][1]) <= 1e-3 * counts[1][1], counts
    assert launches[0] < launches[1], launches
