"""Pins of the FP64 surrogate oracle (oracle/mlp_oracle.py) against facts it
does not compute itself: normal-CDF values, finite differences, the closed
form of the first Adam steps and the IEEE definition of bfloat16 rounding."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as MO


def test_bf16_rounding_definition():
    one = 1.0
    ulp = 2.0 ** -7
    vals = np.array([one, one + ulp / 2, one + 1.5 * ulp, one + ulp / 2 + 2 ** -40, -3.0,
                     2.0 ** -130, 3.0 * 2.0 ** -134, 65504.0, 1e-300])
    got = MO.round_bf16(vals)
    exp = np.array([one,                 # exact
                    one,                 # tie -> even (mantissa 0)
                    one + 2 * ulp,       # tie -> even (mantissa 2)
                    one + ulp,           # above the tie
                    -3.0,
                    2.0 ** -130,         # subnormal, exact multiple of 2^-133
                    4.0 * 2.0 ** -134,   # 1.5 x 2^-133 ties to even (2 x 2^-133)
                    65536.0,             # 65504 needs 11 bits: rounds to 2^16
                    0.0])
    np.testing.assert_array_equal(got, exp)


def test_gelu_values_and_derivative():
    # Phi(1) and Phi(-1) of the standard normal distribution
    assert MO.gelu(np.array(1.0)) == pytest.approx(0.8413447460685429, rel=1e-14)
    assert MO.gelu(np.array(-1.0)) == pytest.approx(-0.15865525393145707, rel=1e-13)
    assert MO.gelu(np.array(0.0)) == 0.0
    assert MO.gelu(np.array(12.0)) == pytest.approx(12.0, rel=1e-15)
    assert abs(MO.gelu(np.array(-12.0))) < 1e-30
    assert MO.gelu_grad(np.array(0.0)) == pytest.approx(0.5, rel=1e-15)
    z = np.linspace(-4, 4, 17)
    h = 1e-6
    fd = (MO.gelu(z + h) - MO.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(MO.gelu_grad(z), fd, rtol=1e-8, atol=1e-10)


def _tiny(seed=0, B=5):
    lay = MO.Layout(n_in=5, n_out=3, H=7)
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(lay.n_params) * 0.5
    P = lay.unpack(p)
    P["W1"][:, lay.n_in:] = 0.0
    P["W4"][lay.n_out:, :] = 0.0
    P["b4"][lay.n_out:] = 0.0
    p = lay.pack(P)
    X = np.zeros((B, lay.ldx))
    X[:, : lay.n_in] = rng.standard_normal((B, lay.n_in))
    t = np.zeros((B, lay.ldo))
    t[:, : lay.n_out] = rng.standard_normal((B, lay.n_out))
    return lay, p, X, t


def test_layout_sizes():
    lay = MO.Layout(21)
    assert (lay.n_in, lay.ldx, lay.n_out, lay.ldo) == (45, 48, 22, 32)
    assert lay.n_params == 256 * 48 + 2 * 256 * 256 + 32 * 256 + 3 * 256 + 32


def test_gradient_matches_finite_differences():
    lay, p, X, t = _tiny()
    g, _ = MO.gradient(lay, p, X, t)
    live = np.ones(lay.n_params, bool)
    P = lay.unpack(np.arange(lay.n_params, dtype=float))
    for idx in np.ravel(P["W1"][:, lay.n_in:]).astype(int):
        live[idx] = False
    for idx in np.ravel(P["W4"][lay.n_out:, :]).astype(int):
        live[idx] = False
    for idx in np.ravel(P["b4"][lay.n_out:]).astype(int):
        live[idx] = False
    h = 1e-6
    fd = np.zeros(lay.n_params)
    for i in np.flatnonzero(live):
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        yp, _ = MO.forward(lay, pp, X)
        ym, _ = MO.forward(lay, pm, X)
        fd[i] = (MO.mse_loss(lay, yp, t) - MO.mse_loss(lay, ym, t)) / (2 * h)
    np.testing.assert_allclose(g[live], fd[live], rtol=1e-6, atol=1e-9)
    assert np.all(g[~live] == 0.0)


def test_gradient_zero_at_perfect_fit():
    lay, p, X, _ = _tiny(1)
    y, _ = MO.forward(lay, p, X)
    g, loss = MO.gradient(lay, p, X, y)
    assert loss == 0.0
    assert np.all(g == 0.0)


def test_adamw_first_steps_closed_form():
    # with a constant gradient, bias-corrected m/sqrt(v) = sign(g) at every step,
    # so each step moves a weight by -lr sign(g) after the decay factor (1 - lr wd)
    lay = MO.Layout(n_in=3, n_out=2, H=4)
    rng = np.random.default_rng(3)
    p0 = rng.standard_normal(lay.n_params)
    g = rng.standard_normal(lay.n_params) * 10.0
    m = np.zeros_like(p0)
    v = np.zeros_like(p0)
    lr, wd = 1e-2, 0.1
    p = p0
    for t in (1, 2, 3):
        p_new, m, v = MO.adamw_step(lay, p, g, m, v, t, lr, wd)
        decay = np.where(np.arange(lay.n_params) < lay.n_weights, 1.0 - lr * wd, 1.0)
        np.testing.assert_allclose(p_new, p * decay - lr * np.sign(g), rtol=0, atol=1e-9)
        p = p_new


def test_features_targets_and_guess_invert():
    lay = MO.Layout(4)
    rng = np.random.default_rng(5)
    n, N = 6, 4
    Yp = rng.uniform(0, 1, (N, n))
    Tp = rng.uniform(300, 2000, n)
    FRp = rng.standard_normal((N, n)) * 1e3
    hp = rng.standard_normal(n) * 1e5
    wdt = 2e-6
    b = Yp - wdt * FRp + rng.standard_normal((N, n)) * 1e-4
    hstar = hp + rng.standard_normal(n) * 10.0
    cp = rng.uniform(1000, 2000, n)
    f, s = MO.features(lay, cp, wdt, b, hstar, Yp, Tp, FRp, hp)
    # the scaled forcing has max-norm one, built from the residual at the guess
    assert np.allclose(np.max(np.abs(f[:, N + 2: 2 * N + 3]), axis=1), 1.0)
    np.testing.assert_allclose(f[:, N + 2: 2 * N + 2] * s[:, None], (b - Yp + wdt * FRp).T, rtol=1e-12)
    assert np.allclose(f[:, N + 1], math.log10(wdt) + 6.0)
    # zero forcing: s = 0 and the scaled features vanish
    f0, s0 = MO.features(lay, cp, wdt, Yp, hp, Yp, Tp, 0.0 * FRp, hp)
    assert np.all(s0 == 0.0) and np.all(f0[:, N + 2:] == 0.0)
    # targets invert the guess map (inside the clip range)
    tY = rng.uniform(-2, 2, (N, n))
    tT = rng.uniform(-0.2, 0.2, n)
    Ys = Yp + s[None, :] * tY
    Ts = Tp * (1 + s * tT)
    t = MO.targets(lay, Yp, Tp, Ys, Ts, s)
    Y0, T0 = MO.guess(Yp, Tp, s, t)
    np.testing.assert_allclose(Y0, Ys, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(T0, Ts, rtol=1e-12)
    tc = MO.targets(lay, Yp, Tp, Yp + 100 * s[None, :], Tp, s)
    assert np.all(tc[:, :N] == 8.0)
