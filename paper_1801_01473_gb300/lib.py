"""ctypes loader of libstg.so and the C signatures of include/stg.h.

The library is the only compute path: if libstg.so is missing this module
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstg.so")

# enums of stg.h
STG_OK, STG_ERR_ARG, STG_ERR_SHAPE, STG_ERR_CUDA, STG_ERR_NOCONV, STG_ERR_TIMEOUT, STG_ERR_OOM = 0, -1, -2, -3, -4, -5, -6
STG_F64, STG_F32, STG_BF16, STG_F16, STG_DS = 0, 1, 2, 3, 4
STG_RECON18, STG_RECON12 = 18, 12

PREC = {"f64": STG_F64, "f32": STG_F32, "bf16": STG_BF16, "f16": STG_F16, "ds": STG_DS}

# every symbol include/stg.h declares
EXPORTS = [
    "stg_status_string", "stg_last_error", "stg_version",
    "stg_lattice_create", "stg_lattice_destroy", "stg_lattice_sites",
    "stg_gauge_create", "stg_gauge_create_u1", "stg_gauge_update", "stg_gauge_destroy", "stg_gauge_bytes",
    "stg_field_bytes", "stg_field_pack", "stg_field_unpack",
    "stg_dslash", "stg_dslash_eo", "stg_dslash_oe", "stg_dslash_multi", "stg_dslash_host", "stg_normal_op", "stg_normal_op_noalloc",
    "stg_mscg_solve", "stg_mscg_solve_batched", "stg_rational_apply", "stg_pseudofermion_action",
    "stg_fermion_force", "stg_fermion_force_prec",
    "stg_stout_smear", "stg_stout_force", "stg_gauge_action", "stg_gauge_force",
    "stg_md_momenta", "stg_md_update_links", "stg_md_update_momenta", "stg_md_kinetic", "stg_complex_convert",
    "stg_lattice_create_slab", "stg_slab_layout", "stg_slab_dslash_part", "stg_slab_dslash_xpay", "stg_slab_axpy_norm", "stg_slab_shift_update",
    "stg_mscg_state_init", "stg_mscg_state_alpha", "stg_mscg_state_beta",
]


class MscgParams(ctypes.Structure):
    _fields_ = [("nshift", ctypes.c_int32), ("shifts", ctypes.POINTER(ctypes.c_double)),
                ("mass", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("inner_tol", ctypes.c_double), ("reliable_delta", ctypes.c_double),
                ("log_rows", ctypes.c_int32), ("scalar_log", ctypes.POINTER(ctypes.c_double)),
                ("history", ctypes.c_int32)]


class MscgStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("reliable_updates", ctypes.c_int32), ("refine_iters", ctypes.c_int32),
                ("true_resid", ctypes.POINTER(ctypes.c_double)), ("shift_iters", ctypes.POINTER(ctypes.c_int32)),
                ("inner_resid", ctypes.POINTER(ctypes.c_double)), ("fp64_fallback", ctypes.c_int32),
                ("refine_shift_iters", ctypes.POINTER(ctypes.c_int32)),
                ("shift_reliable_updates", ctypes.POINTER(ctypes.c_int32))]


class MscgState(ctypes.Structure):
    """stg_mscg_state: host-side scalar recurrences of the multi-shift CG."""
    _fields_ = [("nshift", ctypes.c_int32), ("i0", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("running", ctypes.c_int32), ("nactive", ctypes.c_int32),
                ("phase", ctypes.c_int32),
                ("s", ctypes.c_double * 32), ("zeta", ctypes.c_double * 32), ("zeta_old", ctypes.c_double * 32),
                ("zeta_new", ctypes.c_double * 32),
                ("alpha", ctypes.c_double), ("alpha_old", ctypes.c_double), ("beta_old", ctypes.c_double),
                ("rr", ctypes.c_double), ("tol2", ctypes.c_double),
                ("cx", ctypes.c_double * 32), ("cr", ctypes.c_double * 32), ("cp", ctypes.c_double * 32),
                ("active", ctypes.c_int32 * 32), ("upd_x", ctypes.c_int32 * 32), ("upd_p", ctypes.c_int32 * 32),
                ("shift_iters", ctypes.c_int32 * 32)]


class Instance(ctypes.Structure):
    _fields_ = [("g_f64", ctypes.c_void_p), ("g_inner", ctypes.c_void_p), ("nrhs", ctypes.c_int32),
                ("b", ctypes.POINTER(ctypes.c_void_p)), ("x", ctypes.POINTER(ctypes.c_void_p)),
                ("stats", ctypes.POINTER(MscgStats))]


class StgError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libstg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libstg.so is not built ({LIB_PATH}); run `python -m paper_1801_01473_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    P, I32, I64, D, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    PP = ctypes.POINTER(ctypes.c_void_p)
    L.stg_status_string.restype = ctypes.c_char_p
    L.stg_status_string.argtypes = [ctypes.c_int]
    L.stg_last_error.restype = ctypes.c_char_p
    L.stg_version.restype = ctypes.c_char_p
    L.stg_lattice_create.argtypes = [ctypes.POINTER(I32), I32, PP]
    L.stg_lattice_destroy.argtypes = [P]
    L.stg_lattice_sites.argtypes = [P, I32]
    L.stg_lattice_sites.restype = I64
    L.stg_gauge_create.argtypes = [P, P, ctypes.c_int, ctypes.c_int, P, PP]
    L.stg_gauge_destroy.argtypes = [P]
    L.stg_gauge_bytes.argtypes = [P]
    L.stg_gauge_bytes.restype = SZ
    L.stg_field_bytes.argtypes = [P, ctypes.c_int]
    L.stg_field_bytes.restype = SZ
    L.stg_field_pack.argtypes = [P, ctypes.c_int, P, P, P]
    L.stg_field_unpack.argtypes = [P, ctypes.c_int, P, P, P]
    L.stg_dslash_eo.argtypes = [P, P, P, P]
    L.stg_dslash_oe.argtypes = [P, P, P, P]
    L.stg_dslash_multi.argtypes = [P, I32, I32, P, P, SZ, P]
    L.stg_dslash_host.argtypes = [P, I32, ctypes.c_int, I32, PP, PP, P]
    L.stg_normal_op.argtypes = [P, D, D, P, P, P, P, P]
    L.stg_normal_op_noalloc.argtypes = [P, D, D, P, P, P, P]
    L.stg_mscg_solve.argtypes = [P, P, ctypes.POINTER(MscgParams), P, PP, ctypes.POINTER(MscgStats), P]
    L.stg_mscg_solve_batched.argtypes = [I32, ctypes.POINTER(Instance), ctypes.POINTER(MscgParams), P]
    L.stg_fermion_force.argtypes = [P, I32, ctypes.POINTER(D), PP, P, I32, P]
    L.stg_rational_apply.argtypes = [P, P, ctypes.POINTER(MscgParams), D, ctypes.POINTER(D), P, P,
                                     ctypes.POINTER(MscgStats), P]
    L.stg_pseudofermion_action.argtypes = [P, I32, D, ctypes.POINTER(D), P, PP, P, P]
    L.stg_stout_smear.argtypes = [P, ctypes.c_int, I32, D, P, P, P]
    L.stg_stout_force.argtypes = [P, ctypes.c_int, I32, D, P, P, P, P, I32, P]
    L.stg_gauge_action.argtypes = [P, D, P, P, P]
    L.stg_gauge_create_u1.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int, P, ctypes.POINTER(P)]
    L.stg_gauge_update.argtypes = [P, P, P, P]
    L.stg_dslash.argtypes = [P, I32, P, P, P]
    L.stg_fermion_force_prec.argtypes = [P, ctypes.c_int, I32, ctypes.POINTER(D), PP, P, I32, P]
    L.stg_gauge_force.argtypes = [P, ctypes.c_int, D, P, P, I32, P]
    L.stg_md_momenta.argtypes = [P, P, P, P]
    L.stg_md_update_links.argtypes = [P, D, P, P, P]
    L.stg_md_update_momenta.argtypes = [P, ctypes.c_int, D, P, P, P]
    L.stg_complex_convert.argtypes = [ctypes.c_int64, ctypes.c_int, P, ctypes.c_int, P, P]
    L.stg_md_kinetic.argtypes = [P, P, P, P]
    L.stg_lattice_create_slab.argtypes = [ctypes.POINTER(I32), I32, I32, I32, PP]
    L.stg_slab_layout.argtypes = [P, ctypes.c_int, ctypes.POINTER(I32), ctypes.POINTER(I64), ctypes.POINTER(I32),
                                  ctypes.POINTER(I64)]
    L.stg_slab_dslash_part.argtypes = [P, I32, I32, P, P, P]
    L.stg_slab_dslash_xpay.argtypes = [P, I32, D, P, P, P, P, P]
    L.stg_slab_axpy_norm.argtypes = [P, ctypes.c_int, D, P, P, P, P]
    L.stg_slab_shift_update.argtypes = [P, ctypes.c_int, I32, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D),
                                        ctypes.POINTER(I32), ctypes.POINTER(I32), PP, PP, P, P]
    L.stg_mscg_state_init.argtypes = [ctypes.POINTER(MscgState), I32, ctypes.POINTER(D), D, D, I32]
    L.stg_mscg_state_alpha.argtypes = [ctypes.POINTER(MscgState), D]
    L.stg_mscg_state_beta.argtypes = [ctypes.POINTER(MscgState), D]
    for name in EXPORTS:
        f = getattr(L, name)
        if f.restype is ctypes.c_int or name in ("stg_lattice_create", "stg_gauge_create", "stg_field_pack",
                                                 "stg_field_unpack", "stg_dslash_eo", "stg_dslash_oe",
                                                 "stg_dslash_multi", "stg_dslash_host", "stg_normal_op", "stg_normal_op_noalloc", "stg_mscg_solve",
                                                 "stg_mscg_solve_batched", "stg_rational_apply", "stg_pseudofermion_action", "stg_fermion_force",
                                                 "stg_stout_smear", "stg_stout_force", "stg_gauge_action",
                                                 "stg_gauge_force", "stg_gauge_create_u1", "stg_gauge_update", "stg_fermion_force_prec", "stg_dslash", "stg_md_momenta", "stg_md_update_links",
                                                 "stg_md_update_momenta", "stg_md_kinetic", "stg_complex_convert",
                                                 "stg_lattice_create_slab", "stg_slab_layout", "stg_slab_dslash_part",
                                                 "stg_slab_dslash_xpay",
                                                 "stg_slab_axpy_norm", "stg_slab_shift_update", "stg_mscg_state_init",
                                                 "stg_mscg_state_alpha", "stg_mscg_state_beta"):
            f.restype = ctypes.c_int
    _lib = L
    return L


def check(status: int, where: str, allow=()) -> int:
    if status != STG_OK and status not in allow:
        L = lib()
        raise StgError(status, where, L.stg_last_error().decode() or L.stg_status_string(status).decode())
    return status
