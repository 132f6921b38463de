"""Oracle time steps in parallel worker processes.

TEST INFRASTRUCTURE ONLY (like the rest of this package): the GPU parity tests
use it to run the serial oracle on several flames, and on one-ulp perturbations
of the same input, at the same time. Every worker is a fresh interpreter (the
'spawn' start method), so a pool may be started after CUDA was initialised in
the calling process. Each job is one plain serial oracle run; nothing is split
across workers inside a run.
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np


def _step_job(job):
    import oracle as O
    mech, flame, phi0, dt, scheme, M, sweeps, nu, steps, seed = job
    phi = np.asarray(phi0, dtype=np.float64)
    if seed is not None:   # a one-ulp relative perturbation of every input value
        rng = np.random.default_rng(seed)
        phi = phi * (1 + 1e-16 * rng.standard_normal(phi.shape))
    ad = O.ADR(mech, flame)
    out, st = ad.step(phi, dt, scheme, M, sweeps, nu, n_steps=steps)
    return out, st


class StepPool:
    """Submit oracle time steps of (mechanism, flame, phi0) and collect them later.

    step() returns a future of (state, statistics); with perturb=k it also
    submits k runs whose input is perturbed by one ulp (seeds 100..99+k), and
    sensitivity() then gives the per-field self-sensitivity
    S_f = max over the runs of max|other_f - ref_f| / max|ref_f|.
    """

    def __init__(self, workers: int | None = None):
        n = workers or max(1, min(16, (os.cpu_count() or 2)))
        self.ex = cf.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn"))

    def step(self, mech, flame, phi0, dt, scheme="CISDCQ", M=2, sweeps=4, nu=2, steps=1, perturb=0):
        base = (mech, flame, np.asarray(phi0, dtype=np.float64), dt, scheme, M, sweeps, nu, steps)
        ref = self.ex.submit(_step_job, base + (None,))
        others = [self.ex.submit(_step_job, base + (100 + r,)) for r in range(perturb)]
        return ref, others

    @staticmethod
    def sensitivity(handle):
        ref, others = handle
        want, st = ref.result()
        sens = np.zeros(want.shape[0])
        for f in others:
            other, _ = f.result()
            d = np.max(np.abs(other - want), axis=1) / np.maximum(np.max(np.abs(want), axis=1), 1e-300)
            sens = np.maximum(sens, d)
        return want, st, sens

    def close(self):
        self.ex.shutdown(wait=True)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
