"""ctypes declarations of the C ABI in include/misdc.h (argument marshalling only).

Loading fails loudly when libmisdc.so is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmisdc.so")

OK, E_INVALID, E_CUDA, E_NEWTON, E_MG, E_TIMEOUT, E_NAN, E_OOM, E_TDIAG = range(9)
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "CUDA", 3: "NEWTON", 4: "MG", 5: "TIMEOUT", 6: "NAN",
                7: "OOM", 8: "TDIAG"}
SCHEMES = {"MISDC": 0, "MISDCQ": 1, "CISDCQ": 2}
PRECISIONS = {"fp64": 0, "mixed": 1}

dp = C.POINTER(C.c_double)
ip = C.POINTER(C.c_int)


class MechDesc(C.Structure):
    _fields_ = [("n_species", C.c_int), ("n_reactions", C.c_int), ("W", dp), ("nasa7", dp),
                ("A", dp), ("beta", dp), ("Ea", dp), ("nu_f", ip), ("nu_r", ip), ("D0", dp),
                ("alpha0", C.c_double), ("T_ref", C.c_double), ("theta_exp", C.c_double),
                ("p_ref", C.c_double)]


class GridDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("n_nodes", C.c_int), ("n_sweeps", C.c_int), ("nu", C.c_int), ("scheme", C.c_int),
                ("precision", C.c_int), ("dominant_species", C.c_int), ("rho", C.c_double),
                ("newton_rtol", C.c_double), ("newton_maxit", C.c_int), ("lin_rtol", C.c_double),
                ("mg_levels", C.c_int), ("two_streams", C.c_int), ("use_graph", C.c_int),
                ("profile", C.c_int), ("rates_mma", C.c_int), ("nu_eta", C.c_double),
                ("nu_rho_stall", C.c_double), ("lanes", C.c_int),
                ("lin_rounds", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("newton_solves", C.c_longlong), ("newton_iters", C.c_longlong),
                ("newton_fail", C.c_longlong), ("newton_max", C.c_int), ("status", C.c_int),
                ("lin_sweeps", C.c_longlong), ("lin_resid_max", C.c_double),
                ("kernel_launches", C.c_longlong), ("surrogate_used", C.c_longlong),
                ("surrogate_rejected", C.c_longlong), ("newton_fp64_fallbacks", C.c_longlong),
                ("newton_jacobians", C.c_longlong), ("newton_lu_fp64", C.c_longlong),
                ("newton_certified", C.c_longlong), ("nested_iterations", C.c_longlong),
                ("newton_stored_steps", C.c_longlong), ("newton_floor_stops", C.c_longlong),
                ("newton_chord_cells", C.c_longlong)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


class LowMachDesc(C.Structure):
    _fields_ = [("U_in", C.c_double), ("T_in", C.c_double), ("p0", C.c_double), ("Y_in", dp),
                ("dchi", C.c_int)]


class Tuning(C.Structure):
    _fields_ = [("newton_warps_per_block", C.c_int), ("newton_blocks_per_sm", C.c_int),
                ("newton_dynamic", C.c_int), ("cheb_block", C.c_int),
                ("newton_keep_factors", C.c_int), ("newton_chord_iters", C.c_int),
                ("newton_ms", C.c_double),
                ("cheb_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ["misdc_default_opts", "misdc_create", "misdc_destroy", "misdc_step", "misdc_step_host",
           "misdc_get_stats", "misdc_lobatto", "misdc_enthalpy", "misdc_temperature",
           "misdc_production_rates", "misdc_reaction_solve", "misdc_operators",
           "misdc_diffusion_solve", "misdc_lincomb", "misdc_last_error", "misdc_stage_times",
           "misdc_reaction_solve_noalloc", "misdc_surrogate_dims", "misdc_surrogate_init",
           "misdc_surrogate_load", "misdc_surrogate_save", "misdc_surrogate_enable",
           "misdc_surrogate_collect", "misdc_surrogate_dataset", "misdc_surrogate_train",
           "misdc_surrogate_features", "misdc_surrogate_forward", "misdc_surrogate_gradient",
           "misdc_surrogate_train_batch", "misdc_surrogate_forward_layers", "misdc_surrogate_guess", "misdc_autotune", "misdc_get_tuning", "misdc_set_tuning",
           "misdc_batch_create", "misdc_batch_destroy", "misdc_batch_step", "misdc_batch_stats",
           "misdc_batch_set_grouping", "misdc_batch_grouping",
           "misdc_pde_step", "misdc_pde_smem_bytes", "misdc_exp", "misdc_probe_flops",
           "misdc_lowmach_step", "misdc_surrogate_sweeps"]

_lib = None


class MisdcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("misdc %s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def load(build_if_missing: bool = True):
    """Load libmisdc.so (building it in-tree with nvcc if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH) and build_if_missing:
        from . import build as _build
        _build.build()
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libmisdc.so is not built; run paper_1801_01201_gb300/build.py")
    L = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    L.misdc_default_opts.argtypes = [C.POINTER(Opts)]
    L.misdc_default_opts.restype = None
    L.misdc_create.argtypes = [C.POINTER(MechDesc), C.POINTER(GridDesc), C.POINTER(Opts), vp, C.POINTER(vp)]
    L.misdc_destroy.argtypes = [vp]
    L.misdc_destroy.restype = None
    L.misdc_step.argtypes = [vp, vp, vp, C.c_double, C.c_int, vp]
    L.misdc_step_host.argtypes = [vp, vp, vp, C.c_double, C.c_int, vp]
    L.misdc_get_stats.argtypes = [vp, C.POINTER(Stats), C.c_int]
    L.misdc_lobatto.argtypes = [C.c_int, dp, dp, dp, dp]
    L.misdc_enthalpy.argtypes = [vp, vp, vp, vp, C.c_int, vp]
    L.misdc_temperature.argtypes = [vp, vp, vp, vp, C.c_int, vp]
    L.misdc_production_rates.argtypes = [vp, vp, vp, vp, C.c_int, vp]
    L.misdc_reaction_solve.argtypes = [vp, C.c_double, vp, vp, vp, vp, vp, C.c_int, vp]
    L.misdc_operators.argtypes = [vp, vp, vp, vp, vp, vp]
    L.misdc_diffusion_solve.argtypes = [vp, C.c_double, vp, vp, vp, vp]
    L.misdc_lincomb.argtypes = [C.c_int, C.c_int, C.POINTER(vp), C.POINTER(vp), dp, C.c_size_t, vp]
    L.misdc_stage_times.argtypes = [vp, dp, ip, dp, ip]
    L.misdc_reaction_solve_noalloc.argtypes = [vp, C.c_double, vp, vp, vp, vp, vp, C.c_int, vp]
    fp = C.POINTER(C.c_float)
    L.misdc_surrogate_dims.argtypes = [vp, ip, ip, ip, ip, ip, C.POINTER(C.c_size_t)]
    L.misdc_surrogate_init.argtypes = [vp, C.c_ulonglong]
    L.misdc_surrogate_load.argtypes = [vp, fp, C.c_size_t]
    L.misdc_surrogate_save.argtypes = [vp, fp, C.c_size_t]
    L.misdc_surrogate_enable.argtypes = [vp, C.c_int, C.c_double]
    L.misdc_surrogate_sweeps.argtypes = [vp, C.c_int]
    L.misdc_surrogate_collect.argtypes = [vp, C.c_longlong]
    L.misdc_surrogate_dataset.argtypes = [vp, C.POINTER(C.c_longlong), C.POINTER(vp), C.POINTER(vp)]
    L.misdc_surrogate_train.argtypes = [vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_ulonglong, fp]
    L.misdc_surrogate_features.argtypes = [vp, C.c_double, vp, vp, vp, vp, vp, vp, C.c_int, vp, vp, vp]
    L.misdc_surrogate_forward.argtypes = [vp, vp, C.c_int, vp, vp]
    L.misdc_surrogate_gradient.argtypes = [vp, vp, vp, C.c_int, vp, vp, vp]
    L.misdc_surrogate_forward_layers.argtypes = [vp, vp, C.c_int, vp, vp]
    L.misdc_surrogate_guess.argtypes = [vp, C.c_double, vp, vp, vp, vp, vp, vp, C.c_int, vp, vp, vp]
    L.misdc_surrogate_train_batch.argtypes = [vp, vp, vp, C.c_int, C.c_double, C.c_double, vp, vp]
    L.misdc_autotune.argtypes = [vp, vp, vp, C.c_double, C.POINTER(Tuning)]
    L.misdc_get_tuning.argtypes = [vp, C.POINTER(Tuning)]
    L.misdc_set_tuning.argtypes = [vp, C.POINTER(Tuning)]
    L.misdc_batch_create.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(vp)]
    L.misdc_batch_destroy.argtypes = [vp]
    L.misdc_batch_destroy.restype = None
    L.misdc_batch_step.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), dp, C.c_int, vp]
    L.misdc_batch_stats.argtypes = [vp, C.POINTER(Stats), C.c_int]
    L.misdc_batch_set_grouping.argtypes = [vp, C.c_int]
    L.misdc_batch_grouping.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.misdc_pde_step.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int,
                                 C.c_double, C.c_int, vp, vp, vp, vp, vp, vp]
    L.misdc_exp.argtypes = [vp, vp, C.c_size_t, vp]
    L.misdc_probe_flops.argtypes = [C.c_int, C.c_int, C.c_int, vp, dp, vp]
    L.misdc_lowmach_step.argtypes = [vp, C.POINTER(LowMachDesc), C.c_double, C.c_int, vp, vp, vp, vp, vp]
    L.misdc_pde_smem_bytes.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_size_t)]
    L.misdc_last_error.restype = C.c_char_p
    L.misdc_last_error.argtypes = []
    for name in EXPORTS:
        if name not in ("misdc_default_opts", "misdc_destroy", "misdc_last_error", "misdc_batch_destroy"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def check(rc):
    if rc != OK:
        raise MisdcError(rc, load().misdc_last_error().decode())
    return rc
