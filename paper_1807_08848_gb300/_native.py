"""ctypes declarations of the C ABI in include/msp.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmsp.so")

MSP_OK = 0
MSP_ERR_INVALID_ARG = -1
MSP_ERR_OOM = -2
MSP_ERR_NOT_CONVERGED = -3
MSP_ERR_BREAKDOWN = -4
MSP_ERR_TIMEOUT = -5
MSP_ERR_CUDA = -6
MSP_ERR_STATE = -7
STATUS_NAMES = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "NOT_CONVERGED", -4: "BREAKDOWN",
                -5: "TIMEOUT", -6: "CUDA", -7: "STATE"}

MSP_FP64 = 0
MSP_MIXED = 1


class MediumDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_cells", C.c_int), ("eps", C.c_double),
                ("n_modes", C.c_int), ("modes_host", C.POINTER(C.c_double)),
                ("amp", C.c_double), ("norm", C.c_double),
                ("n_channels", C.c_int), ("channels_host", C.POINTER(C.c_double)),
                ("width", C.c_double), ("contrast", C.c_double),
                ("user_aE_host", C.POINTER(C.c_double)), ("user_aN_host", C.POINTER(C.c_double))]


class PatchDesc(C.Structure):
    _fields_ = [("nx_patches", C.c_int), ("ny_patches", C.c_int),
                ("x_breaks_host", C.POINTER(C.c_int)), ("y_breaks_host", C.POINTER(C.c_int)),
                ("buffers_host", C.POINTER(C.c_int)), ("samples_host", C.POINTER(C.c_int))]


class PatchInfo(C.Structure):
    _fields_ = [("x0", C.c_int), ("x1", C.c_int), ("y0", C.c_int), ("y1", C.c_int),
                ("X0", C.c_int), ("X1", C.c_int), ("Y0", C.c_int), ("Y1", C.c_int),
                ("n_k", C.c_int), ("n_ring", C.c_int), ("samples", C.c_int), ("n_b", C.c_int),
                ("cols", C.c_int), ("snap_offset", C.c_int64)]


class BasisStats(C.Structure):
    _fields_ = [("max_jacobi_sweeps", C.c_int), ("max_cholqr_tries", C.c_int), ("online_shift", C.c_float),
                ("online_blocks", C.c_int), ("online_factor_bits", C.c_int),
                ("mean_jacobi_sweeps", C.c_float), ("online_apply_bits", C.c_int)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("released", C.c_int64),
                ("failed", C.c_int64), ("batches", C.c_int64), ("queued", C.c_int), ("in_flight", C.c_int),
                ("held", C.c_int), ("max_batch_seen", C.c_int), ("mem_in_use", C.c_int64),
                ("mem_peak", C.c_int64)]


class TuneCandidate(C.Structure):
    _fields_ = [("mode", C.c_int), ("rows", C.c_int), ("ms", C.c_float)]


class TuneReport(C.Structure):
    _fields_ = [("probe_items", C.c_int), ("n_candidates", C.c_int), ("candidates", TuneCandidate * 8),
                ("best_mode", C.c_int), ("best_rows", C.c_int), ("best_ms", C.c_float)]


class SolveStats(C.Structure):
    _fields_ = [("n_solves", C.c_int64), ("total_iters", C.c_int64), ("max_iters", C.c_int),
                ("max_refinements", C.c_int), ("n_not_converged", C.c_int), ("unknown_iters", C.c_int64)]


_vp = C.c_void_p
_i = C.c_int
_d = C.c_double
_u64 = C.c_uint64

# name -> (restype, argtypes)
SIGNATURES = {
    "msp_last_error": (C.c_char_p, []),
    "msp_version": (C.c_char_p, []),
    "msp_kernel_launches": (C.c_int64, []),
    "msp_build_medium": (_i, [C.POINTER(MediumDesc), C.POINTER(PatchDesc), _vp, C.POINTER(_vp)]),
    "msp_build_medium_full": (_i, [C.POINTER(MediumDesc), C.POINTER(PatchDesc), _vp, C.POINTER(_vp)]),
    "msp_medium_destroy": (None, [_vp]),
    "msp_medium_counts": (_i, [_vp, C.POINTER(_i), C.POINTER(C.c_int64), C.POINTER(_i)]),
    "msp_medium_patch": (_i, [_vp, _i, C.POINTER(PatchInfo)]),
    "msp_get_coefficients": (_i, [_vp, _vp, _vp, _vp]),
    "msp_sample_patches": (_i, [_vp, _u64, _i, _d, _i, _vp, C.POINTER(SolveStats)]),
    "msp_get_snapshots": (_i, [_vp, _i, _vp, _vp]),
    "msp_sample_patch_list": (_i, [_vp, C.POINTER(_i), _i, _u64, _i, _d, _i, _vp, C.POINTER(SolveStats)]),
    "msp_set_snapshots": (_i, [_vp, _i, _vp, _vp]),
    "msp_get_samples": (_i, [_vp, _i, _u64, _vp, _vp]),
    "msp_sample_patch_static": (_i, [_vp, _vp, _i, C.POINTER(_i), _i, _i, _u64, _i, _d, _i, _vp, _vp, C.POINTER(_i)]),
    "msp_set_wait_limit": (_i, [C.c_int64]),
    "msp_set_gemm_engine": (_i, [_i]),
    "msp_set_svd_mode": (_i, [_i]),
    "msp_extract_basis": (_i, [_vp, _d, _i, _vp, C.POINTER(_vp)]),
    "msp_basis_destroy": (None, [_vp]),
    "msp_basis_info": (_i, [_vp, _i, C.POINTER(_i), C.POINTER(_d)]),
    "msp_get_basis": (_i, [_vp, _i, _vp, _vp]),
    "msp_online_counts": (_i, [_vp, C.POINTER(_i), C.POINTER(_i)]),
    "msp_basis_get_stats": (_i, [_vp, C.POINTER(BasisStats)]),
    "msp_set_extract_timing": (_i, [_i]),
    "msp_basis_extract_timing": (_i, [_vp, C.POINTER(_d), C.POINTER(_d)]),
    "msp_basis_set_preconditioner": (_i, [_vp, _i]),
    "msp_kinetic_build": (_i, [_i, _d, _i, _i, _i, _i, _vp, C.POINTER(_vp)]),
    "msp_kinetic_build_hg": (_i, [_i, _d, _d, _i, _i, _i, _i, _vp, C.POINTER(_vp)]),
    "msp_kinetic_set_solver": (_i, [_vp, _i]),
    "msp_kinetic_destroy": (None, [_vp]),
    "msp_kinetic_velocities": (_i, [_vp, C.POINTER(_d), C.POINTER(_d)]),
    "msp_kinetic_sample": (_i, [_vp, _u64, _i, _d, _i, _vp, C.POINTER(SolveStats)]),
    "msp_kinetic_get_snapshots": (_i, [_vp, _i, _vp, _vp]),
    "msp_kinetic_extract": (_i, [_vp, _d, _vp, C.POINTER(_vp)]),
    "msp_kinetic_basis_destroy": (None, [_vp]),
    "msp_kinetic_basis_info": (_i, [_vp, _i, C.POINTER(_i), C.POINTER(_d)]),
    "msp_kinetic_online_solve": (_i, [_vp, _vp, _i, _vp, _vp, _vp]),
    "msp_online_solve": (_i, [_vp, _vp, _i, _d, _i, _vp, _vp, C.POINTER(_i), _vp]),
    "msp_online_solve_constrained": (_i, [_vp, _vp, _i, _d, _i, _vp, _vp, C.POINTER(_i), _vp]),
    "msp_ras_setup": (_i, [_vp, _vp, _i, _vp]),
    "msp_online_solve_ras": (_i, [_vp, _vp, _i, _d, _i, _vp, _vp, C.POINTER(_i), _vp]),
    "msp_operator_tile_shape": (_i, [_vp, C.POINTER(_i), C.POINTER(_i)]),
    "msp_medium_set_launch": (_i, [_vp, _i, _i, _i]),
    "msp_medium_set_graph": (_i, [_vp, _i]),
    "msp_medium_set_timing": (_i, [_vp, _i]),
    "msp_medium_direct_timing": (_i, [_vp, C.POINTER(_d), C.POINTER(_i)]),
    "msp_medium_autotune": (_i, [_vp, _i, _u64, _d, _i, _i, _vp, C.POINTER(TuneReport)]),
    "msp_apply_operator": (_i, [_vp, _i, _i, _vp, _vp, _i, _i, C.POINTER(_d), _vp]),
    "msp_basis_build_map": (_i, [_vp, _d, _i, _vp]),
    "msp_save_basis": (_i, [_vp, C.c_char_p]),
    "msp_basis_patch": (_i, [_vp, _i, C.POINTER(_i), C.POINTER(_i), C.POINTER(PatchInfo)]),
    "msp_load_basis": (_i, [C.c_char_p, C.POINTER(_vp)]),
    "msp_get_online_system": (_i, [_vp, C.POINTER(_d), C.c_int64, C.POINTER(C.c_int64), C.POINTER(_i),
                                   C.POINTER(_i), C.POINTER(_d), C.POINTER(_d)]),
    "msp_online_solve_map": (_i, [_vp, _vp, _i, _vp, _vp]),
    "msp_basis_set_map_engine": (_i, [_vp, _i]),
    "msp_server_create": (_i, [C.POINTER(_vp), _i, C.c_int64, _i, _i, _i, C.POINTER(_vp)]),
    "msp_server_submit": (_i, [_vp, _i, C.POINTER(_d), C.POINTER(_u64)]),
    "msp_server_poll": (_i, [_vp, _u64, C.POINTER(_i), C.POINTER(_d)]),
    "msp_server_fetch": (_i, [_vp, _u64, C.POINTER(_d)]),
    "msp_server_release": (_i, [_vp, _u64]),
    "msp_server_step": (_i, [_vp, _vp, C.POINTER(_i)]),
    "msp_server_get_stats": (_i, [_vp, C.POINTER(ServerStats)]),
    "msp_server_set_engine": (_i, [_vp, _i, _d, _i]),
    "msp_server_destroy": (None, [_vp]),
}

_lib = None


class MspError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load libmsp.so and declare its entry points.  Raises if the library is
    missing: there is no fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1807_08848_gb300.build.build() "
                           "(there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, allow=()):
    if status != MSP_OK and status not in allow:
        raise MspError(status, load().msp_last_error().decode())
    return status
