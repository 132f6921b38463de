"""Bounds and records shared by the GPU parity tests (not a test module)."""
import json
import os

import numpy as np

TOL = 1e-10   # FP64 parity bound, relative per field

# Mixed-precision bar: each species i whose largest mass fraction reaches
# Y_FLOOR has max|dY_i| / max|Y_i| <= 1e-8 against the FP64 oracle (T within
# 1e-6, checked by the callers). Both reaction solvers stop on an absolute step
# of 1e-12 in Y, so two correct answers may differ by ~2e-12 in every Y_i, which
# is 1e-8 of Y_i only from Y_i = 2e-4 on; below that the ratio measures the
# stopping tolerance, and those species are held to 2e-12 absolute (plus the
# FP64 sensitivity).
Y_FLOOR = 2e-4


def relerr(a, b):
    """max|a - b| / max|b| (per row for 2D arrays)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.ndim == 1:
        return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)
    return np.max(np.abs(a - b), axis=1) / np.maximum(np.max(np.abs(b), axis=1), 1e-300)


def tol_from(sens):
    """Per-field FP64 bound: max(1e-10, 2 S_f), S_f the oracle's self-sensitivity."""
    return np.maximum(TOL, 2.0 * sens)


def mixed_bar(got, want, sens, N):
    """Assert the mixed-precision bar on the mass fractions; returns the
    per-species relative errors."""
    scale = np.max(np.abs(want[:N]), axis=1)
    absd = np.max(np.abs(got[:N] - want[:N]), axis=1)
    err_i = absd / scale
    big = scale >= Y_FLOOR
    assert np.all(err_i[big] <= np.maximum(1e-8, 2 * sens[:N][big])), (err_i[big], sens[:N][big])
    assert np.all(absd[~big] <= 2e-12 + 2 * sens[:N][~big] * scale[~big]), (absd[~big], scale[~big])
    return err_i


def record(case, **kw):
    """With MISDC_PARITY_LOG set, append one JSON line describing a comparison."""
    path = os.environ.get("MISDC_PARITY_LOG")
    if not path:
        return
    line = {"case": case}
    for k, v in kw.items():
        line[k] = v.tolist() if isinstance(v, np.ndarray) else v
    with open(path, "a") as f:
        f.write(json.dumps(line) + "\n")
