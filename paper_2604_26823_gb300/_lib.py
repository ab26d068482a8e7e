"""ctypes declarations of the C ABI in include/mujica_pm.h.

Loading fails loudly when the in-tree library has not been built: there is
no CPU or PyTorch fallback for any entry point.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmujica_pm.so")

PM_OK = 0
PM_ERR_NONFINITE = 4
STATUS = {0: "PM_OK", 1: "PM_ERR_INVALID_ARG", 2: "PM_ERR_UNSUPPORTED", 3: "PM_ERR_CUDA",
          4: "PM_ERR_NONFINITE", 5: "PM_ERR_WORKSPACE", 6: "PM_ERR_LINESEARCH",
          7: "PM_ERR_DEVICE_STATUS"}
PM_PREC_F32, PM_PREC_F64 = 0, 1
PM_LIK_GAUSSIAN, PM_LIK_POISSON = 0, 1
PM_BIAS_AUTO, PM_BIAS_LINEAR, PM_BIAS_POWERLAW_SIGMOID = 0, 1, 2
PM_PROJECT, PM_ROM_FOURIER, PM_ROM_REAL = 1, 2, 4


class PMError(RuntimeError):
    def __init__(self, status, where, message):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {message}")
        self.status = status


class pm_config(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("n_steps", ctypes.c_int32), ("lpt_order", ctypes.c_int32),
        ("rsd_axis", ctypes.c_int32), ("likelihood", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("checkpoint_every", ctypes.c_int32), ("lightcone", ctypes.c_int32), ("bias", ctypes.c_int32),
        ("box", ctypes.c_double), ("omega_m", ctypes.c_double), ("a_init", ctypes.c_double),
        ("bias_b", ctypes.c_double), ("sigma", ctypes.c_double), ("alpha", ctypes.c_double),
        ("delta_th", ctypes.c_double), ("K", ctypes.c_double), ("nbar_cell", ctypes.c_double),
        ("rho_floor", ctypes.c_double), ("prior_weight", ctypes.c_double), ("observer", ctypes.c_double * 3),
    ]


# name -> (restype, argtypes)
_P = ctypes.c_void_p
_D = ctypes.c_double
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_U32 = ctypes.c_uint32
_U64 = ctypes.c_uint64
_DP = ctypes.POINTER(ctypes.c_double)
_I64P = ctypes.POINTER(ctypes.c_int64)
_I32P = ctypes.POINTER(ctypes.c_int32)
_SZP = ctypes.POINTER(ctypes.c_size_t)
_CFGP = ctypes.POINTER(pm_config)

SIGNATURES = {
    "pm_last_error": (ctypes.c_char_p, []),
    "pm_version": (ctypes.c_char_p, []),
    "pm_launch_count": (ctypes.c_int64, []),
    "pm_fma_rate": (_I32, [_I32, _I64, _P, _DP, _P]),
    "pm_linear_power_table": (_I32, [_D, _D, _D, _D, _D, _D, _D, _I32, _DP, _DP]),
    "pm_growth": (_I32, [_D, _I32, _DP, _DP, _DP, _DP, _DP]),
    "pm_distance_table": (_I32, [_D, _D, _I32, _DP, _DP]),
    "pm_workspace_bytes": (_I32, [_CFGP, _SZP]),
    "pm_plan_create": (_I32, [_CFGP, _DP, _DP, _I32, _P, ctypes.c_size_t, ctypes.POINTER(_P)]),
    "pm_plan_destroy": (_I32, [_P]),
    "pm_forward": (_I32, [_P, _P, _P, _P, _DP, _P, _P]),
    "pm_adjoint": (_I32, [_P, _P, _P, _P, _D, _P, _DP, _P, _P]),
    "pm_last_terms": (_I32, [_P, _DP, _DP]),
    "pm_linear_field": (_I32, [_P, _P, _P, _P]),
    "pm_lpt": (_I32, [_P, _P, _P, _P, _P]),
    "pm_force": (_I32, [_P, _P, _P, _P, _P]),
    "pm_evolve": (_I32, [_P, _P, _P, _P, _P]),
    "pm_expected_counts": (_I32, [_P, _P, _P, _P, _P]),
    "pm_refine_noise": (_I32, [_P, _P, _I32, _P, _P, _P]),
    "pm_coarsen": (_I32, [_I32, _I32, _I32, _I32, _P, _P, _P]),
    "pm_power_spectra": (_I32, [_P, _P, _P, _I32, _D, _D, _DP, _DP, _DP, _DP, _DP, _P]),
    "pm_smooth": (_I32, [_P, _P, _D, _P, _P]),
    "pm_tweb": (_I32, [_P, _P, _D, _D, _P, _P, _P, _P]),
    "pm_eigvec_cosines": (_I32, [ctypes.c_int64, _I32, _P, _P, _P, _P]),
    "pm_confusion": (_I32, [ctypes.c_int64, _I32, _P, _P, _P, _P, _P]),
    "pm_profile": (_I32, [_P, _I32, _I32]),
    "pm_profile_read": (_I32, [_P, _I32, _DP, _I64P, _DP, _DP, _DP]),
    "pm_rom_fourier_counts": (_I32, [_P, _I64P]),
    "pm_count_positive": (_I32, [_P, _P, _I64P, _P]),
    "project_rank_match": (_I32, [_P, _P, _U32, _P, _P, _P, _U64, _U64, _I64P, _P, _P]),
    "pm_project_noalloc": (_I32, [_I64, _I32, _P, _U64, _U64, _I64P, _P]),
    "lbfgs_workspace_bytes": (_I32, [_I64, _I32, _I32, _SZP]),
    "lbfgs_create": (_I32, [_I64, _I32, _I32, _P, ctypes.c_size_t, ctypes.POINTER(_P)]),
    "lbfgs_destroy": (_I32, [_P]),
    "lbfgs_reset": (_I32, [_P]),
    "lbfgs_step": (_I32, [_P, _P, _P, _P, _DP, _DP, _I32P, _P]),
    "pm_axpy": (_I32, [_I64, _I32, _D, _P, _P, _P, _P]),
}

_lib = None


def load():
    """Load the CUDA library (built by ``paper_2604_26823_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"the CUDA library {LIB_PATH} is not built; run "
            "`python -c 'import __graft_entry__ as g; g.build()'` (there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status, where):
    if status != PM_OK:
        msg = load().pm_last_error().decode(errors="replace")
        raise PMError(status, where, msg)
