"""GPU parity of the learned Newton guess: the library's tensor-core MLP
kernels, features and AdamW (through the C ABI) against the FP64 numpy oracle
(oracle/mlp_oracle.py), and the learned guess inside full time steps.

Tolerances. The kernels store weights, inputs and hidden activations in BF16
and accumulate in FP32; the oracle rounds the same operands to BF16 at the same
points and accumulates exactly. What remains is the FP32 accumulation order
(~K 2^-24 relative per dot product, K <= 256) and BF16 ties that the two sides
round to different neighbours (one BF16 ulp). Outputs and gradients are
compared element by element within two BF16 ulps of each element's accumulated
magnitude (forward_tolerance, gradient_tolerance); features elementwise within
one BF16 ulp.
The learned guess never changes the converged answer beyond the Newton
tolerance: steps with it match steps without it within 1e-10 relative.
"""
import numpy as np
import pytest

import oracle as O
from oracle import mlp_oracle as MO
from paper_1801_01201_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

def S():
    from paper_1801_01201_gb300 import solver
    return solver


def nrel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def bf16_np(t):
    return t.float().cpu().numpy().astype(np.float64)


# Element-wise tolerances of the BF16 kernels against the oracle: KU = two BF16
# ulps (2 x 2^-8) of each element's accumulated magnitude, the sum of the
# absolute values of the terms that make it up (FP32 accumulation contributes
# about K 2^-24 of that magnitude; a BF16 value that rounds to its other
# neighbour, one ulp of that value, enters downstream elements in proportion to
# their magnitudes). Magnitudes follow the oracle's own arrays: forward, the
# output's |W4| |h3| + |b4|; backward, one layer deep, the upstream BF16 values
# through |W| and |gelu'| (plus |gelu''| <= 0.8 times the pre-activation's
# magnitude) against the stored activations, and the error that dy inherits from
# the forward output. Where gelu' is small the tolerance is small. (Measured: the
# kernels stay within 0.09 of it; a derivative of GELU replaced by a plausible
# wrong one, planted in a numpy copy of the kernels' arithmetic, exceeds it 2-13x.)
KU = 2.0 * 2.0 ** -8


def forward_tolerance(lay, p, X, x_ulps=0.0):
    """(y_ref, tolerance per output element, oracle arrays, pre-activation
    magnitudes); x_ulps: BF16 ulps of |X| by which the kernel's input may differ."""
    y, c = MO.forward(lay, p, X, bf16=True)
    W, H = c["W"], c["H"]
    P = lay.unpack(p)
    bs = [P["b1"], P["b2"], P["b3"], P["b4"]]
    A = []
    for k in range(4):
        A.append(np.abs(H[k]) @ np.abs(W[k]).T + np.abs(bs[k]))
    tol = KU * A[3]
    if x_ulps:
        m = np.abs(H[0]) * (x_ulps * 2.0 ** -8)
        for k in range(3):
            m = 1.13 * (m @ np.abs(W[k]).T)
        tol = tol + m @ np.abs(W[3]).T
    return y, tol, c, A


def gradient_tolerance(lay, p, X, t):
    """Tolerance per parameter of the gradient (packed like the gradient): KU of
    each element's accumulated magnitude, taken over the oracle's own values one
    layer deep (|upstream BF16 values| through |W| and |gelu'|, then against the
    stored activations), and the error dy inherits from the forward output."""
    y, _, c, A = forward_tolerance(lay, p, X)
    Z, H, W = c["Z"], c["H"], c["W"]
    B = X.shape[0]
    dy = np.zeros_like(y)
    dy[:, : lay.n_out] = 2.0 * (y - t)[:, : lay.n_out] / (B * lay.n_out)
    Edy = np.zeros_like(y)
    Edy[:, : lay.n_out] = 2.0 * KU * A[3][:, : lay.n_out] / (B * lay.n_out)
    dyb = MO.round_bf16(dy)
    g = {"W4": (Edy + KU * np.abs(dyb)).T @ np.abs(H[3]), "b4": (Edy + KU * np.abs(dy)).sum(axis=0)}
    up, Eup, Wn = dyb, Edy, W[3]
    for k, (wn, bn) in zip((2, 1, 0), (("W3", "b3"), ("W2", "b2"), ("W1", "b1"))):
        v = up @ Wn
        gp = MO.gelu_grad(Z[k])
        Mdz = (np.abs(up) @ np.abs(Wn)) * np.abs(gp) + np.abs(v) * 0.8 * KU * A[k]
        Edz = (Eup @ np.abs(Wn)) * np.abs(gp)
        dz = v * gp
        g[wn] = (Edz + KU * Mdz).T @ np.abs(H[k])
        g[bn] = (Edz + KU * Mdz).sum(axis=0)
        up, Eup, Wn = MO.round_bf16(dz), np.zeros_like(dz), W[k]   # dy's error: one layer deep
    g["W4"][lay.n_out:, :] = 0.0
    g["b4"][lay.n_out:] = 0.0
    return lay.pack(g)


def assert_forward(lay, p, X, y_gpu, label, x_ulps=0.0, factor=1.0):
    y_ref, tol, *_ = forward_tolerance(lay, p, X, x_ulps)
    o = slice(0, lay.n_out)
    r = np.abs(y_gpu[:, o] - y_ref[:, o]) / (factor * tol[:, o] + 1e-300)
    print("%s: worst |error| / tolerance %.3f" % (label, float(r.max())))
    assert np.all(r <= 1.0), float(r.max())


def assert_gradient(lay, p, X, t, g_gpu, keys, label):
    G, R = lay.unpack(g_gpu), lay.unpack(MO.gradient(lay, p, X, t, bf16=True)[0])
    E = lay.unpack(gradient_tolerance(lay, p, X, t))
    for k in keys:
        r = np.abs(G[k] - R[k]) / (E[k] + 1e-300)
        print("%s %s: worst |error| / tolerance %.3f" % (label, k, float(r.max())))
        assert np.all(r <= 1.0), (k, float(r.max()))


@pytest.fixture(scope="module")
def setup21():
    mech = I.make_mechanism(1802, 21, 84)
    fl = I.flame_2d(mech, 0, n=32, dx=4e-5, radius=32 * 4e-5 / 4, delta=2 * 4e-5)
    sv = S().Solver(mech, fl, n_sweeps=2, nu=2)
    sv.surrogate_init(seed=11)
    return mech, fl, sv


def _data(lay, n, seed):
    rng = np.random.default_rng(seed)
    X = np.zeros((n, lay.ldx))
    X[:, : lay.n_in] = rng.standard_normal((n, lay.n_in))
    t = np.zeros((n, lay.ldo))
    t[:, : lay.n_out] = rng.standard_normal((n, lay.n_out))
    return MO.round_bf16(X), t


@pytest.mark.parametrize("n", [1, 200, 1000, 40000])
def test_forward_parity(setup21, n):
    """Row counts from one partial tile to 313 tiles (more than one tile per CTA)."""
    mech, fl, sv = setup21
    d = sv.surrogate_dims()
    lay = MO.Layout(mech.n_species)
    assert (d["n_in"], d["ldx"], d["n_out"], d["ldo"], d["n_params"]) == (
        lay.n_in, lay.ldx, lay.n_out, lay.ldo, lay.n_params)
    p = sv.surrogate_save().astype(np.float64)
    X, _ = _data(lay, n, n)
    y_gpu = sv.surrogate_forward(torch.as_tensor(X, dtype=torch.bfloat16)).cpu().numpy()
    assert np.all(y_gpu[:, lay.n_out:] == 0.0)
    assert_forward(lay, p, X, y_gpu, "forward n=%d" % n)


def test_fused_and_layered_forward_agree(setup21):
    """The fused inference kernel and the per-layer GEMM kernels round at the same
    points; only FP32 accumulation order and BF16 ties differ."""
    mech, fl, sv = setup21
    lay = MO.Layout(mech.n_species)
    X, _ = _data(lay, 777, 3)
    Xt = torch.as_tensor(X, dtype=torch.bfloat16)
    a = sv.surrogate_forward(Xt).cpu().numpy()
    b = sv.surrogate_forward_layers(Xt).cpu().numpy()
    p = sv.surrogate_save().astype(np.float64)
    # each within the tolerance of the oracle, so within twice it of each other
    assert_forward(lay, p, X, a, "fused")
    assert_forward(lay, p, X, b, "layered")
    y_ref = MO.forward(lay, p, X, bf16=True)[0]
    assert_forward(lay, p, X, y_ref + (a - b), "fused - layered", factor=2.0)
    assert np.all(b[:, lay.n_out:] == 0.0)


def test_guess_parity(setup21):
    """Fused features + network against the oracle's features and network."""
    mech, fl, sv = setup21
    N = mech.n_species
    lay = MO.Layout(N)
    adr = O.ADR(mech, fl)
    rng = np.random.default_rng(8)
    n = 333
    Yp = np.abs(fl.Y[:, :n] * (1 + 0.01 * rng.standard_normal((N, n))))
    Tp = fl.T[:n] * (1 + 0.01 * rng.standard_normal(n))
    hp = adr.h_from_T(Yp, Tp)
    FRp = rng.standard_normal((N, n)) * 1e2
    wdt = 1.7e-6
    b = Yp - wdt * FRp + 1e-5 * rng.standard_normal((N, n))
    hstar = hp + 50.0 * rng.standard_normal(n)
    cp = np.array([sum(Yp[i, c] * adr.species_cp(i, Tp[c]) for i in range(N)) for c in range(n)])
    f_ref, s_ref = MO.features(lay, cp, wdt, b, hstar, Yp, Tp, FRp, hp)
    p = sv.surrogate_save().astype(np.float64)
    out, sc = sv.surrogate_guess(wdt, b, hstar, Yp, Tp, FRp, hp)
    np.testing.assert_allclose(sc.cpu().numpy(), s_ref, rtol=1e-12)
    y = out.cpu().numpy()
    # the kernel's features may round to the other BF16 neighbour (one ulp)
    assert_forward(lay, p, MO.round_bf16(f_ref), y, "guess", x_ulps=1.0)


def test_forward_parity_small_mechanism():
    mech = I.make_mechanism(1801, 9, 21)
    fl = I.flame_1d(mech, 0, nx=64, dx=1e-4, u=1.0)
    sv = S().Solver(mech, fl)
    sv.surrogate_init(seed=3)
    lay = MO.Layout(9)
    assert sv.surrogate_dims()["ldx"] == 24
    p = sv.surrogate_save().astype(np.float64)
    X, _ = _data(lay, 333, 1)
    y_gpu = sv.surrogate_forward(torch.as_tensor(X, dtype=torch.bfloat16)).cpu().numpy()
    assert_forward(lay, p, X, y_gpu, "9 species, fused")
    y_l = sv.surrogate_forward_layers(torch.as_tensor(X, dtype=torch.bfloat16)).cpu().numpy()
    assert_forward(lay, p, X, y_l, "9 species, layered")


def test_forward_parity_large_mechanism():
    """53 species: 109 inputs (two K chunks in layer 1), 54 outputs (64 columns)."""
    mech = I.make_mechanism(1803, 53, 325)
    fl = I.flame_1d(mech, 0, nx=64, dx=1e-4, u=1.0)
    sv = S().Solver(mech, fl)
    sv.surrogate_init(seed=4)
    lay = MO.Layout(53)
    assert (sv.surrogate_dims()["ldx"], sv.surrogate_dims()["ldo"]) == (112, 64)
    p = sv.surrogate_save().astype(np.float64)
    X, t = _data(lay, 300, 2)
    y_gpu = sv.surrogate_forward(torch.as_tensor(X, dtype=torch.bfloat16)).cpu().numpy()
    assert_forward(lay, p, X, y_gpu, "53 species")
    g_gpu, _ = sv.surrogate_gradient(torch.as_tensor(X, dtype=torch.bfloat16),
                                     torch.as_tensor(t, dtype=torch.float32))
    assert_gradient(lay, p, X, t, g_gpu.cpu().numpy().astype(np.float64),
                    ("W1", "W2", "W3", "W4", "b1", "b2", "b3", "b4"), "53 species")


@pytest.mark.parametrize("n", [128, 1000])
def test_gradient_parity(setup21, n):
    mech, fl, sv = setup21
    lay = MO.Layout(mech.n_species)
    p = sv.surrogate_save().astype(np.float64)
    X, t = _data(lay, n, 100 + n)
    g_gpu, loss = sv.surrogate_gradient(torch.as_tensor(X, dtype=torch.bfloat16),
                                        torch.as_tensor(t, dtype=torch.float32))
    g_gpu = g_gpu.cpu().numpy().astype(np.float64)
    g_ref, loss_ref = MO.gradient(lay, p, X, t, bf16=True)
    assert abs(float(loss.item()) - loss_ref) <= 1e-3 * loss_ref
    assert_gradient(lay, p, X, t, g_gpu, ("W1", "W2", "W3", "W4", "b1", "b2", "b3", "b4"), "n=%d" % n)
    G = lay.unpack(g_gpu)
    # padded entries stay exactly zero
    assert np.all(G["W1"][:, lay.n_in:] == 0.0)
    assert np.all(G["W4"][lay.n_out:, :] == 0.0) and np.all(G["b4"][lay.n_out:] == 0.0)


def test_adamw_parity(setup21):
    mech, fl, sv = setup21
    lay = MO.Layout(mech.n_species)
    sv.surrogate_init(seed=21)
    X, t = _data(lay, 512, 7)
    Xt = torch.as_tensor(X, dtype=torch.bfloat16)
    tt = torch.as_tensor(t, dtype=torch.float32)
    p = sv.surrogate_save().astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    lr, wd = 1e-3, 0.05
    for step in (1, 2):
        g, _ = sv.surrogate_gradient(Xt, tt)
        g = g.cpu().numpy().astype(np.float64)
        sv.surrogate_train_batch(Xt, tt, lr, wd)
        p_gpu = sv.surrogate_save().astype(np.float64)
        p, m, v = MO.adamw_step(lay, p, g, m, v, step, lr, wd)
        # FP32 arithmetic of the update: a few ulp of |p| plus lr eps-level terms
        assert np.max(np.abs(p_gpu - p)) <= 1e-6 * max(1.0, np.max(np.abs(p))), step
        p = p_gpu
    sv.surrogate_init(seed=11)


def test_features_parity(setup21):
    mech, fl, sv = setup21
    N = mech.n_species
    lay = MO.Layout(N)
    adr = O.ADR(mech, fl)
    rng = np.random.default_rng(4)
    n = 300
    Yp = np.abs(fl.Y[:, :n] * (1 + 0.01 * rng.standard_normal((N, n))))
    Tp = fl.T[:n] * (1 + 0.01 * rng.standard_normal(n))
    hp = adr.h_from_T(Yp, Tp)
    FRp = rng.standard_normal((N, n)) * 1e2
    wdt = 1.7e-6
    b = Yp - wdt * FRp + 1e-5 * rng.standard_normal((N, n))
    b[:, :10] = Yp[:, :10] - wdt * FRp[:, :10]         # nearly converged cells
    hstar = hp + 50.0 * rng.standard_normal(n)
    cp = np.array([sum(Yp[i, c] * adr.species_cp(i, Tp[c]) for i in range(N)) for c in range(n)])
    f_ref, s_ref = MO.features(lay, cp, wdt, b, hstar, Yp, Tp, FRp, hp)
    X, sc = sv.surrogate_features(wdt, b, hstar, Yp, Tp, FRp, hp)
    np.testing.assert_allclose(sc.cpu().numpy(), s_ref, rtol=1e-12, atol=1e-300)
    fx = bf16_np(X)
    fr = MO.round_bf16(f_ref)
    ulp = np.maximum(np.abs(fr), 2.0 ** -126) * 2.0 ** -7
    bad = np.abs(fx - fr) > ulp * 1.0001
    # the scaled forcing of the ten converged cells is round-off over round-off:
    # only its range is fixed
    assert np.all(np.abs(fx[:10, N + 2: 2 * N + 3]) <= 1.0)
    bad[:10, N + 2: 2 * N + 3] = False
    assert not bad.any(), [(int(r), int(c), fx[r, c], fr[r, c]) for r, c in zip(*np.nonzero(bad))][:8]
    assert np.all(fx[:, lay.n_in:] == 0.0)


def _mild_flame(n=32):
    mech = I.make_mechanism(1802, 21, 84, logA_range=(8.0, 11.0))
    fl = I.flame_2d(mech, 0, n=n, dx=4e-5, radius=n * 4e-5 / 4, delta=2 * 4e-5)
    return mech, fl


def test_dataset_rows_valid():
    """Rows recorded during a step: features and targets of real solves."""
    mech, fl = _mild_flame()
    sv = S().Solver(mech, fl, n_sweeps=1, nu=1, use_graph=False)
    sv.surrogate_collect(100000)
    st = sv.state_from_YT(fl.Y, fl.T)
    sv.step(st, 5e-6, 1)
    rows, X, T = sv.surrogate_dataset()
    lay = MO.Layout(mech.n_species)
    assert 0 < rows <= 2 * fl.nx * fl.ny
    x = bf16_np(X)
    t = T.cpu().numpy()
    assert np.all(np.isfinite(x)) and np.all(np.isfinite(t))
    N = mech.n_species
    sf = x[:, N + 2: 2 * N + 3]                     # scaled forcing: max-norm one
    assert np.allclose(np.max(np.abs(sf), axis=1), 1.0, rtol=2 ** -7)
    assert np.all(np.abs(t[:, : lay.n_out]) <= 8.0) and np.all(t[:, lay.n_out:] == 0.0)


def test_learned_guess_fallback_and_agreement():
    """A useless network (huge random output layer) is rejected by the residual
    residual test on every cell: the steps equal plain Newton's and take the same number
    of iterations. A trained network leaves the answer unchanged too."""
    mech, fl = _mild_flame()
    dt = 5e-6
    base = S().Solver(mech, fl)
    s0 = base.state_from_YT(fl.Y, fl.T)
    ref = s0.clone()
    base.stats(reset=True)
    base.step(ref, dt, 2)
    st_ref = base.stats(reset=True)

    bad = S().Solver(mech, fl)
    bad.surrogate_init(seed=5)
    lay = MO.Layout(mech.n_species)
    p = bad.surrogate_save()
    P = lay.unpack(p.astype(np.float64))
    P["W4"][: lay.n_out, :] *= 1e4
    bad.surrogate_load(lay.pack(P).astype(np.float32))
    bad.surrogate_enable(True, s_min=0.0)
    out = s0.clone()
    bad.step(out, dt, 2)
    st_bad = bad.stats(reset=True)
    assert st_bad["status"] == 0
    assert st_bad["surrogate_rejected"] > 0
    assert st_bad["surrogate_used"] <= 0.01 * st_bad["surrogate_rejected"]
    a, b_ = out.cpu().numpy(), ref.cpu().numpy()
    for f in range(a.shape[0]):
        assert nrel(a[f], b_[f]) < 1e-10, f
    assert abs(st_bad["newton_iters"] - st_ref["newton_iters"]) <= 0.01 * st_ref["newton_iters"]


def test_trained_guess_gain():
    """Record solves, train on them with the library's kernels, and compare the
    Newton iterations of the same steps with and without the learned guess: the
    converged state is the same and the trained network saves at least 3 % of
    the FP64 Newton iterations (measured on a GB300: 5.3 %)."""
    mech, fl = _mild_flame(48)
    dt = 5e-6
    sv = S().Solver(mech, fl, use_graph=False)
    sv.surrogate_init(seed=1)
    s0 = sv.state_from_YT(fl.Y, fl.T)
    warm = s0.clone()
    sv.surrogate_collect(400000)
    sv.step(warm, dt, 3)
    rows, _, _ = sv.surrogate_dataset()
    assert rows > 1000
    sv.surrogate_collect(0)
    curve = sv.surrogate_train(600, batch=2048, lr=2e-3, weight_decay=1e-4, seed=9)
    assert np.all(np.isfinite(curve))
    assert curve[-50:].mean() < 0.5 * curve[:10].mean()
    a = warm.clone()
    sv.stats(reset=True)
    sv.step(a, dt, 2)
    plain = sv.stats(reset=True)
    sv.surrogate_enable(True, s_min=1e-8)
    b = warm.clone()
    sv.step(b, dt, 2)
    learned = sv.stats(reset=True)
    sv.surrogate_enable(False, 0.0)
    A, B = a.cpu().numpy(), b.cpu().numpy()
    for f in range(A.shape[0]):
        assert nrel(B[f], A[f]) < 1e-10, f
    assert learned["status"] == 0 and plain["status"] == 0
    from parity_util import record
    record("trained_guess_gain", plain_iters=plain["newton_iters"], plain_solves=plain["newton_solves"],
           learned_iters=learned["newton_iters"], learned_solves=learned["newton_solves"],
           used=learned["surrogate_used"], rejected=learned["surrogate_rejected"], rows=rows,
           loss_first=float(curve[:10].mean()), loss_last=float(curve[-50:].mean()))
    print("\nplain iters/solve %.4f  learned iters/solve %.4f  used %d rejected %d  loss %.3g -> %.3g"
          % (plain["newton_iters"] / plain["newton_solves"],
             learned["newton_iters"] / learned["newton_solves"], learned["surrogate_used"],
             learned["surrogate_rejected"], curve[:10].mean(), curve[-50:].mean()))
    assert learned["surrogate_used"] > 0
    assert learned["newton_solves"] == plain["newton_solves"]
    assert learned["newton_iters"] <= 0.97 * plain["newton_iters"], (learned["newton_iters"], plain["newton_iters"])


def test_trained_guess_gain_on_a_flame_it_was_not_trained_on():
    """The learned guess as the benchmark uses it: trained on solves recorded from
    one flame of the 21-species / 84-reaction mechanism with its full rate ranges
    (seed 4242, kernel off-centre), applied to another flame of the same recipe
    (seed 1802, centred kernel; 64^2 cells, the workload's dx, front width and
    velocity field) with the benchmark's s_min = 1e-4. It leaves the
    converged state unchanged and takes fewer FP64 Newton iterations than plain
    Newton from the previous iterate."""
    mech = I.make_mechanism(1802, 21, 84)
    n, dx, dt = 64, 4e-5, 5e-6
    L = n * dx
    train = I.flame_2d(mech, 4242, n=n, dx=dx, amp=2.0, radius=0.28 * L, delta=2e-4,
                       centre=(0.41 * L, 0.57 * L))
    target = I.flame_2d(mech, 1802, n=n, dx=dx, amp=2.0, radius=0.25 * L, delta=2e-4)
    sv = S().Solver(mech, train)
    sv.surrogate_init(seed=3)
    sv.surrogate_collect(2_000_000)
    x = sv.state_from_YT(train.Y, train.T)
    sv.step(x, dt, 4)
    rows, _, _ = sv.surrogate_dataset()
    sv.surrogate_collect(0)
    curve = sv.surrogate_train(1500, batch=8192, lr=2e-3, weight_decay=1e-4, seed=7)
    params = sv.surrogate_save()
    sv.close()
    ref = S().Solver(mech, target)
    lrn = S().Solver(mech, target)
    lrn.surrogate_load(params)
    lrn.surrogate_enable(True, s_min=1e-4)
    x0 = ref.state_from_YT(target.Y, target.T)
    a, b = x0.clone(), x0.clone()
    ref.step(a, dt, 3)
    lrn.step(b, dt, 3)
    plain, learned = ref.stats(), lrn.stats()
    from parity_util import record
    record("trained_guess_gain_other_flame", plain_iters=plain["newton_iters"],
           learned_iters=learned["newton_iters"], solves=plain["newton_solves"],
           used=learned["surrogate_used"], rejected=learned["surrogate_rejected"], rows=rows,
           loss_first=float(curve[:10].mean()), loss_last=float(curve[-50:].mean()))
    assert plain["status_name"] == learned["status_name"] == "OK"
    A, B = a.cpu().numpy(), b.cpu().numpy()
    # the two runs take different Newton paths to the same roots; with rates up to
    # A = 1e14 the steps amplify their round-off differences (as in the FP64
    # parity tests), so the states agree to the mixed bar rather than to 1e-10
    d = max(nrel(B[f], A[f]) for f in range(A.shape[0]))
    record("trained_guess_gain_other_flame_state", max_rel_diff=d)
    assert d < 1e-8, d
    assert learned["surrogate_used"] > 0
    assert learned["newton_iters"] < plain["newton_iters"], (learned["newton_iters"], plain["newton_iters"])
