"""ctypes binding of libqedttn.so: argument marshalling only.

Every name mirrors a declaration of include/qedttn.h.  Loading fails loudly
if the library has not been built (``python -m paper_2011_10658_gb300.build``
or ``__graft_entry__.build()``); there is no fallback implementation.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqedttn.so")

c_int = ctypes.c_int
c_int8_p = ctypes.POINTER(ctypes.c_int8)
c_int16_p = ctypes.POINTER(ctypes.c_int16)
c_int32 = ctypes.c_int32
c_int32_p = ctypes.POINTER(ctypes.c_int32)
c_int64 = ctypes.c_int64
c_int64_p = ctypes.POINTER(ctypes.c_int64)
c_double = ctypes.c_double
c_double_p = ctypes.POINTER(ctypes.c_double)
c_void_p = ctypes.c_void_p


class QedParams(ctypes.Structure):
    _fields_ = [("Lx", c_int32), ("Ly", c_int32), ("Lz", c_int32), ("boundary", c_int32),
                ("t", c_double), ("m", c_double), ("ge2", c_double), ("cB", c_double), ("nu", c_double),
                ("Q", c_int32)]


class SweepStats(ctypes.Structure):
    _fields_ = [("energy", c_double), ("matvecs", c_int32), ("matvecs_mixed", c_int32), ("node_updates", c_int32),
                ("not_converged", c_int32), ("max_rel_residual", c_double), ("seconds", c_double)]


class QedDrive(ctypes.Structure):
    _fields_ = [("nu_start", c_double), ("nu_step", c_double), ("quad_coef", c_double), ("nu_max", c_double),
                ("tol_start", c_double), ("tol_factor", c_double), ("tol_final", c_double), ("conv_rel", c_double),
                ("rise_rel", c_double), ("min_final_sweeps", c_int32), ("max_sweeps", c_int32), ("max_krylov", c_int32)]


class QedDriveState(ctypes.Structure):
    _fields_ = [("stage", c_int32), ("sweep", c_int32), ("since_switch", c_int32), ("final_sweeps", c_int32),
                ("done", c_int32), ("nu", c_double), ("tol", c_double), ("nu_switch", c_double), ("e_prev", c_double)]


class QedDriveRecord(ctypes.Structure):
    _fields_ = [("sweep", c_int32), ("stage", c_int32), ("nu", c_double), ("tol", c_double), ("energy", c_double),
                ("energy_without_penalty", c_double), ("delta_L", c_double), ("matvecs", c_int32),
                ("not_converged", c_int32), ("max_rel_residual", c_double), ("seconds", c_double)]


# (name, restype, argtypes) for every entry point of include/qedttn.h
SIGNATURES = [
    ("qed_last_error", ctypes.c_char_p, []),
    ("qed_basis", c_int, [c_int, c_int8_p, c_int32_p]),
    ("qed_local_op", c_int, [c_int, c_int, c_int, c_int, c_int16_p, c_double_p]),
    ("qed_model_create", c_int, [ctypes.POINTER(QedParams), ctypes.POINTER(c_void_p)]),
    ("qed_model_destroy", None, [c_void_p]),
    ("qed_model_info", c_int, [c_void_p, c_int32_p, c_int32_p, c_int32_p, c_double_p]),
    ("qed_model_terms", c_int, [c_void_p, c_double_p, c_int32_p, c_int32_p, c_int32_p, c_int64, c_int64_p]),
    ("qed_model_tree", c_int, [c_void_p, c_int32_p, c_int64, c_int64_p]),
    ("qed_model_sweep_order", c_int, [c_void_p, c_int32_p, c_int64, c_int64_p]),
    ("qed_model_sectors", c_int, [c_void_p, c_int32, c_int32_p, c_int64, c_int64_p]),
    ("ttn_create", c_int, [c_void_p, c_int32, ctypes.c_uint64, c_int, c_void_p, ctypes.POINTER(c_void_p)]),
    ("ttn_destroy", None, [c_void_p]),
    ("ttn_sweep", c_int, [c_void_p, c_int32, c_double, c_int32, ctypes.POINTER(SweepStats)]),
    ("ttn_batch_sweep", c_int, [ctypes.POINTER(c_void_p), c_int32, c_int32, c_double, c_int32,
                                 ctypes.POINTER(SweepStats)]),
    ("ttn_optimize_node", c_int, [c_void_p, c_int32, c_double, c_int32, c_double_p]),
    ("ttn_set_mixed_tol", c_int, [c_void_p, c_double]),
    ("ttn_set_wait_limit", c_int, [c_void_p, c_int64]),
    ("ttn_set_precision", c_int, [c_void_p, c_int]),
    ("ttn_last_update", c_int, [c_void_p, c_int32_p, c_int32_p, c_double_p, c_double_p, c_double_p]),
    ("ttn_set_profiling", c_int, [c_void_p, c_int]),
    ("ttn_reset_timing", c_int, [c_void_p]),
    ("ttn_kernel_timing", c_int, [c_void_p, c_int, c_double_p, c_int64_p, c_double_p, c_double_p, c_double_p]),
    ("ttn_move_center", c_int, [c_void_p, c_int32]),
    ("ttn_info", c_int, [c_void_p, c_int32_p, c_int32_p, c_int64_p]),
    ("ttn_node_size", c_int, [c_void_p, c_int32, c_int64_p]),
    ("ttn_energy", c_int, [c_void_p, c_double_p, c_double_p, c_double_p]),
    ("ttn_measure", c_int, [c_void_p, c_int, c_double_p, c_int64, c_int64_p]),
    ("ttn_node_export", c_int, [c_void_p, c_int32, c_double_p, c_int64, c_int64_p]),
    ("ttn_node_import", c_int, [c_void_p, c_int32, c_double_p, c_int64]),
    ("ttn_load_tensors", c_int, [c_void_p, ctypes.POINTER(c_double_p), c_int64_p, c_int32]),
    ("qed_launch_count", c_int, [c_int64_p]),
    ("ttn_apply_heff", c_int, [c_void_p, c_double_p, c_double_p, c_int64]),
    ("ttn_apply_heff_device", c_int, [c_void_p, c_void_p, c_void_p, c_int64]),
    ("ttn_save", c_int, [c_void_p, ctypes.c_char_p]),
    ("ttn_load", c_int, [c_void_p, ctypes.c_char_p, c_void_p, ctypes.POINTER(c_void_p)]),
    ("ttn_apply_heff_adjoint_device", c_int, [c_void_p, c_void_p, c_void_p, c_int64]),
    ("ttn_energy_grad", c_int, [c_void_p, c_int32, c_void_p, c_int64, c_double_p, c_void_p, c_double_p]),
    ("ttn_gradient_step", c_int, [c_void_p, c_double, c_double_p, c_double_p]),
    ("ttn_apply_heff_device_noalloc", c_int, [c_void_p, c_void_p, c_void_p, c_int64]),
    ("ttn_set_couplings", c_int, [c_void_p, c_double_p]),
    ("qed_model_set_site_potential", c_int, [c_void_p, c_double_p, c_int32]),
    ("qed_drive_start", c_int, [ctypes.POINTER(QedDrive), ctypes.POINTER(QedDriveState)]),
    ("qed_drive_next", c_int, [ctypes.POINTER(QedDrive), ctypes.POINTER(QedDriveState), c_double]),
    ("ttn_drive", c_int, [c_void_p, ctypes.POINTER(QedDrive), ctypes.POINTER(QedDriveRecord), c_int32, c_int32_p]),
]

STATUS = {0: "QED_OK", -1: "QED_EINVAL", -2: "QED_ENOMEM", -3: "QED_ECUDA", -4: "QED_ENOCONV",
          -5: "QED_ENAN", -6: "QED_ETIMEOUT", -7: "QED_EUNSUPPORTED"}


class QedError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load libqedttn.so once; raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(code, allow=()):
    if code == 0 or code in allow:
        return code
    msg = lib().qed_last_error()
    raise QedError(code, msg.decode() if msg else "")
