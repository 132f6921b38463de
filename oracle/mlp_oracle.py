"""Plain FP64 numpy oracle of the learned Newton initial guess.

TEST INFRASTRUCTURE ONLY: the independent checker of the CUDA library's
surrogate kernels (only the tests, the smoke check and the benchmark's CPU leg
may import it). It shares no code with the CUDA path.

The paper has no learned component: this is the learned form of the reaction
step S5 (Sec. 3.3), whose Newton iteration otherwise starts from the previous
iterate. Everything here is the plain definition:
  - network y = W4 g(W3 g(W2 g(W1 x + b1) + b2) + b3) + b4 with the Gaussian
    error linear unit g(z) = z Phi(z) (Phi: standard normal CDF);
  - mean-squared loss L = mean over rows and outputs of (y - t)^2 and its
    gradient by the chain rule, layer by layer;
  - AdamW: Adam (Kingma & Ba, 2015) with decoupled weight decay
    (Loshchilov & Hutter, 2019), bias-corrected moments;
  - the cell features and targets of the library's learned guess;
  - round-to-nearest-even to bfloat16 (8-bit exponent, 7 stored mantissa
    bits), used where the kernels store BF16.
Parameter vector layout (matching the library's documented ABI):
W1 [H][ldx], W2 [H][H], W3 [H][H], W4 [ldo][H], b1 [H], b2 [H], b3 [H], b4 [ldo].
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SQRT_HALF = math.sqrt(0.5)


# ---- bfloat16 rounding -----------------------------------------------------
def round_bf16(x):
    """Round float64 values to the nearest bfloat16 (ties to even), as float64."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    tiny = np.abs(x) < 2.0 ** -126          # bf16 subnormal range: spacing 2^-133
    out[tiny] = np.round(x[tiny] / 2.0 ** -133) * 2.0 ** -133
    b = x[~tiny].view(np.uint64)
    keep = (b >> np.uint64(45)) & np.uint64(1)
    r = (b + np.uint64((1 << 44) - 1) + keep) >> np.uint64(45) << np.uint64(45)
    out[~tiny] = r.view(np.float64)
    return out


# ---- activation --------------------------------------------------------------
def gelu(z):
    return z * 0.5 * (1.0 + erf(z * SQRT_HALF))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z * SQRT_HALF)) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


# ---- parameter vector ---------------------------------------------------------
class Layout:
    def __init__(self, n_species=None, *, n_in=None, n_out=None, H=256):
        if n_species is not None:
            n_in, n_out = 2 * n_species + 3, n_species + 1
        self.n_in, self.n_out, self.H = n_in, n_out, H
        self.ldx = (n_in + 7) // 8 * 8
        self.ldo = (n_out + 15) // 16 * 16
        H, ldx, ldo = self.H, self.ldx, self.ldo
        sizes = [H * ldx, H * H, H * H, ldo * H, H, H, H, ldo]
        self.off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.n_params = int(self.off[-1])
        self.n_weights = int(self.off[4])

    def unpack(self, p):
        H, ldx, ldo, o = self.H, self.ldx, self.ldo, self.off
        p = np.asarray(p, dtype=np.float64)
        return dict(W1=p[o[0]:o[1]].reshape(H, ldx), W2=p[o[1]:o[2]].reshape(H, H),
                    W3=p[o[2]:o[3]].reshape(H, H), W4=p[o[3]:o[4]].reshape(ldo, H),
                    b1=p[o[4]:o[5]], b2=p[o[5]:o[6]], b3=p[o[6]:o[7]], b4=p[o[7]:o[8]])

    def pack(self, d):
        return np.concatenate([np.ravel(d[k]) for k in ("W1", "W2", "W3", "W4", "b1", "b2", "b3", "b4")])


# ---- forward / backward ------------------------------------------------------
def forward(lay, p, X, bf16=False):
    """Outputs [B][ldo] and the saved pre-activations. bf16=True rounds the
    weights, the input and the stored hidden activations to bfloat16 where the
    kernels store them (accumulation stays exact here)."""
    P = lay.unpack(p)
    rb = round_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    W = [rb(P["W1"]), rb(P["W2"]), rb(P["W3"]), rb(P["W4"])]
    b = [P["b1"], P["b2"], P["b3"], P["b4"]]
    h = rb(X)
    Z, Hs = [], [h]
    for k in range(3):
        z = h @ W[k].T + b[k]
        Z.append(z)
        h = rb(gelu(z))
        Hs.append(h)
    y = h @ W[3].T + b[3]
    return y, dict(Z=Z, H=Hs, W=W)


def mse_loss(lay, y, t):
    d = (y - t)[:, : lay.n_out]
    return float(np.mean(d * d))


def gradient(lay, p, X, t, bf16=False):
    """Gradient of the mean-squared loss (mean over rows and the n_out outputs)
    with respect to the parameter vector, by the chain rule."""
    y, c = forward(lay, p, X, bf16)
    rb = round_bf16 if bf16 else (lambda a: a)
    B = X.shape[0]
    dy = np.zeros_like(y)
    dy[:, : lay.n_out] = 2.0 * (y - t)[:, : lay.n_out] / (B * lay.n_out)
    Z, Hs, W = c["Z"], c["H"], c["W"]
    g = {}
    dyb = rb(dy)                       # the kernels feed BF16 copies to the GEMMs
    g["W4"] = dyb.T @ Hs[3]
    g["b4"] = dy.sum(axis=0)
    dz = (dyb @ W[3]) * gelu_grad(Z[2])
    for k, (wn, bn) in zip((2, 1, 0), (("W3", "b3"), ("W2", "b2"), ("W1", "b1"))):
        dzb = rb(dz)
        g[wn] = dzb.T @ Hs[k]
        g[bn] = dz.sum(axis=0)
        if k > 0:
            dz = (dzb @ W[k]) * gelu_grad(Z[k - 1])
    g["W4"][lay.n_out:, :] = 0.0
    g["b4"][lay.n_out:] = 0.0
    return lay.pack(g), mse_loss(lay, y, t)


# ---- optimiser ---------------------------------------------------------------
def adamw_step(lay, p, grad, m, v, t, lr, wd, beta1=0.9, beta2=0.999, eps=1e-8):
    """One AdamW step (t = 1, 2, ...); weight decay on the weights only."""
    p, grad, m, v = (np.asarray(a, dtype=np.float64).copy() for a in (p, grad, m, v))
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    decay = np.zeros_like(p)
    decay[: lay.n_weights] = wd
    p = p - lr * decay * p
    p = p - lr * mh / (np.sqrt(vh) + eps)
    return p, m, v


# ---- features and targets of a reaction step --------------------------------
def features(lay, cp_mix, wdt, b, hstar, Yp, Tp, FRp, hp):
    """Per-cell features [n][ldx] (FP64, before BF16 rounding) and scale s [n].
    b, Yp, FRp: [N][n]; hstar, Tp, hp: [n]; cp_mix: mixture cp at (Yp, Tp) [n]."""
    N = Yp.shape[0]
    r = b - Yp + wdt * FRp
    rT = (hstar - hp) / (cp_mix * Tp)
    s = np.maximum(np.max(np.abs(r), axis=0), np.abs(rT))
    inv = np.where(s > 0.0, 1.0 / np.where(s > 0.0, s, 1.0), 0.0)
    n = Tp.shape[0]
    f = np.zeros((n, lay.ldx))
    f[:, :N] = Yp.T
    f[:, N] = (Tp - 1150.0) / 850.0
    f[:, N + 1] = math.log10(wdt) + 6.0
    f[:, N + 2: 2 * N + 2] = (r * inv).T
    f[:, 2 * N + 2] = rT * inv
    return f, s


def targets(lay, Yp, Tp, Ys, Ts, s, clip=8.0):
    """Training targets [n][ldo]: (Y* - Y_p)/s and (T* - T_p)/(T_p s), clipped."""
    N = Yp.shape[0]
    inv = np.where(s > 0.0, 1.0 / np.where(s > 0.0, s, 1.0), 0.0)
    t = np.zeros((Tp.shape[0], lay.ldo))
    t[:, :N] = ((Ys - Yp) * inv).T
    t[:, N] = (Ts - Tp) / Tp * inv
    t[:, : N + 1] = np.clip(t[:, : N + 1], -clip, clip)
    return t


def guess(Yp, Tp, s, pred):
    """Newton start from a prediction [n][ldo]: Y_p + s p_Y, T_p (1 + s p_T) with
    the T factor clamped to [0.5, 1.5]."""
    N = Yp.shape[0]
    Y0 = Yp + s[None, :] * pred[:, :N].T
    T0 = Tp * (1.0 + np.clip(s * pred[:, N], -0.5, 0.5))
    return Y0, T0
