"""ctypes declarations of the libsem C ABI (include/sem.h).

Loading fails loudly: there is no CPU fallback for any call.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

SEM_OK = 0
SEM_EINVAL = -1
SEM_ENOMEM = -2
SEM_ECUDA = -3
SEM_ENOTCONV = -4
SEM_EBREAKDOWN = -5
SEM_EMESH = -6
SEM_MAX_N = 11
SEM_MAX_LEVELS = 6
SEM_FP64, SEM_FP32, SEM_BF16G, SEM_FP64P = 0, 1, 2, 3
SEM_AX_LOCAL, SEM_AX_ASSEMBLE, SEM_AX_PAIRS = 0, 1, 2
SEM_GS_ADD, SEM_GS_ADD_MASK = 0, 1
SEM_PC_JACOBI, SEM_PC_PMG = 0, 1
SEM_RHS_NODAL, SEM_RHS_ASSEMBLED, SEM_X0_GIVEN, SEM_OUTER_PAIRS = 0, 1, 2, 4
SEM_BUILD_FP32, SEM_BUILD_BF16G, SEM_BUILD_PAIRS = 1, 2, 4
SEM_GRAD_SUM = 1
SEM_SMOOTH_JACOBI, SEM_SMOOTH_ASM = 0, 1
SEM_ADV_LOCAL, SEM_ADV_ASSEMBLE = 0, 1
SEM_COARSE_AUTO, SEM_COARSE_KERNELS, SEM_COARSE_PIPE = 0, 2, 4


class SemMesh(C.Structure):
    _fields_ = [("E", C.c_int32), ("N", C.c_int32),
                ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("gid", C.c_void_p), ("dirichlet", C.c_void_p)]


class SemOpts(C.Structure):
    _fields_ = [("mg_nlevels", C.c_int32), ("mg_orders", C.c_int32 * SEM_MAX_LEVELS),
                ("cheb_degree", C.c_int32), ("cheb_lmin_factor", C.c_double),
                ("cheb_lmax_factor", C.c_double), ("lanczos_steps", C.c_int32),
                ("lanczos_seed", C.c_uint64), ("coarse_tol", C.c_double),
                ("coarse_maxit", C.c_int32), ("prec_copies", C.c_int32), ("smoother", C.c_int32),
                ("coarse_mode", C.c_int32), ("spin_limit", C.c_int64)]


class SemCoef(C.Structure):
    _fields_ = [("h1", C.c_double), ("h2", C.c_double), ("h1_L", C.c_void_p)]


class SemInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("relres", C.c_double), ("bnorm", C.c_double),
                ("coarse_iters", C.c_int32), ("nlevels", C.c_int32),
                ("lmax", C.c_double * SEM_MAX_LEVELS), ("relres0", C.c_double), ("proj_count", C.c_int32),
                ("graph_steps", C.c_int32)]


class SemLevelDesc(C.Structure):
    _fields_ = [("N", C.c_int32), ("E", C.c_int32), ("nL", C.c_int64), ("nG", C.c_int64),
                ("n_ids", C.c_int64), ("n_idx", C.c_int64), ("n_seg", C.c_int64),
                ("n_seg_idx", C.c_int64)]


_P = C.c_void_p
_I = C.c_int
_D = C.c_double

# name -> (restype, argtypes)
SIGNATURES = {
    "sem_default_opts": (None, [C.POINTER(SemOpts)]),
    "sem_strerror": (C.c_char_p, [_I]),
    "sem_last_error_detail": (C.c_char_p, []),
    "sem_setup": (_I, [C.POINTER(SemMesh), C.POINTER(SemOpts), C.POINTER(_P)]),
    "sem_free": (None, [_P]),
    "sem_num_levels": (_I, [_P]),
    "sem_level_info": (_I, [_P, _I, C.POINTER(SemLevelDesc)]),
    "sem_ax": (_I, [_P, _P, _P, C.POINTER(SemCoef), _I, _P]),
    "sem_gs": (_I, [_P, _P, _I, _P]),
    "sem_level_ax": (_I, [_P, _I, _I, _P, _P, _D, _D, _I, _P]),
    "sem_level_gs": (_I, [_P, _I, _I, _P, _I, _P]),
    "sem_level_dinv": (_I, [_P, _I, _D, _D, _P, _P]),
    "sem_prolong_add": (_I, [_P, _I, _I, _P, _P, _P]),
    "sem_restrict": (_I, [_P, _I, _I, _P, _P, _P]),
    "sem_precond_setup": (_I, [_P, _D, _D, _I, _P]),
    "sem_precond_setup_nodal": (_I, [_P, _P, _D, _I, _P]),
    "sem_cheb_smooth": (_I, [_P, _I, _P, _P, _I, _P]),
    "sem_vcycle": (_I, [_P, _P, _P, _P]),
    "sem_asm_apply": (_I, [_P, _I, _I, _P, _P, _D, _D, _P]),
    "sem_advect": (_I, [_P, _I, _P, _P, _P, _I, _I, _P]),
    "sem_char_advance": (_I, [_P, _I, _P, _P, _P, _I, _D, _D, _I, _P]),
    "sem_get_lmax": (_I, [_P, _P, _I]),
    "sem_solve": (_I, [_P, _P, C.POINTER(SemCoef), _D, _I, _I, _I, _I, _P, C.POINTER(SemInfo), _P]),
    "sem_solve_proj": (_I, [_P, _P, _P, C.POINTER(SemCoef), _D, _I, _I, _I, _I, _P, C.POINTER(SemInfo), _P]),
    "sem_proj_create": (_I, [_P, _I, C.POINTER(_P)]),
    "sem_proj_free": (None, [_P]),
    "sem_proj_reset": (_I, [_P]),
    "sem_proj_count": (_I, [_P]),
    "sem_proj_vectors": (_I, [_P, _I, C.POINTER(_P), C.POINTER(_P)]),
    "sem_proj_project": (_I, [_P, _P, _P, _P, _P]),
    "sem_proj_update": (_I, [_P, C.POINTER(SemCoef), _I, _P, _P, C.POINTER(_I), _P]),
    "sem_grad_h1": (_I, [_P, _P, _P, _P, _I, _P]),
    "sem_rhs": (_I, [_P, _P, _P, _P]),
    "sem_mass_local": (_I, [_P, _P, _P, _P]),
    "sem_dot": (_I, [_P, _P, _P, _P, _P]),
    "sem_dot_static": (_I, [_P, _P, _P, C.c_int64, _P, _P]),
    "sem_measure_peaks": (_I, [_P]),
    "sem_partition_rcb": (_I, [C.c_int32, _P, _P, _P, C.c_int32, _P]),
    "sem_ax_elements": (_I, [_P, C.c_int32, C.c_int32, _P, _P, C.POINTER(SemCoef), _I, _P]),
    "sem_halo_create": (_I, [_P, C.c_int64, _P, _P, C.c_int64, C.POINTER(_P)]),
    "sem_halo_free": (None, [_P]),
    "sem_halo_gather": (_I, [_P, _P, _P, _P]),
    "sem_halo_scatter": (_I, [_P, _P, _P, _I, _P]),
    "sem_get_maps": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P]),
    "sem_get_geom": (_I, [_P, _I, _P]),
    "sem_get_geom_lowp": (_I, [_P, _I, _I, _P]),
    "sem_get_coords": (_I, [_P, _I, _P, _P, _P, _P]),
    "sem_gll": (_I, [_I, _P, _P, _P]),
    "sem_coarse_partition": (_I, [C.c_int32, C.c_int64, _P, _P, _P, _P, _P, _P, C.c_int32, C.c_int64,
                                  C.c_int64, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libsem.so (optionally building it first). Raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"libsem is not built ({path} missing); run __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SemError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        msg = lib.sem_strerror(code).decode()
        detail = lib.sem_last_error_detail().decode()
        super().__init__(f"{where}: {msg} ({code}): {detail}")
        self.code = code


def check(code: int, where: str):
    if code != SEM_OK:
        raise SemError(code, where)
