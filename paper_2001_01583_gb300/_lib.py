"""ctypes declarations of the gbnfft C ABI (include/gbnfft.h).

Argument marshalling only: every step of a transform runs in the CUDA
library.  Loading fails loudly if libgbnfft.so has not been built; there is
no fallback implementation.
"""
import ctypes
import os
import re

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libgbnfft.so")
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gbnfft.h")

# nfft_status
OK = 0
ERR_INVALID_ARG = -1
ERR_DOMAIN = -2
ERR_OOM = -3
ERR_CUDA = -4
ERR_CUFFT = -5
ERR_NOT_READY = -6
ERR_TIMEOUT = -7
ERR_UNSUPPORTED = -8

GAUSSIAN = 0
KAISER_BESSEL = 1
B_SPLINE = 2
SINC_POWER = 3
WINDOWS = {"gaussian": GAUSSIAN, "kaiser_bessel": KAISER_BESSEL, "kb": KAISER_BESSEL, "b_spline": B_SPLINE,
           "bspline": B_SPLINE, "sinc_power": SINC_POWER}

FP64 = 0
FP32_MIXED = 1
PRECISIONS = {"fp64": FP64, "fp32": FP32_MIXED, "fp32_mixed": FP32_MIXED}

METHOD_AUTO, METHOD_TILED, METHOD_GLOBAL, METHOD_WARP, METHOD_GRID_WARP = 0, 1, 2, 3, 4
(OPT_METHOD, OPT_BIN_0, OPT_BIN_1, OPT_BIN_2, OPT_MAX_SUBPROBLEM, OPT_RHS_CAPACITY, OPT_PROFILE, OPT_THREADS,
 OPT_SPREAD_THREADS, OPT_INTERP_THREADS, OPT_SPARSE_POINTS, OPT_SPARSE_POINTS_INTERP, OPT_OWNER_SPREAD,
 OPT_TENSOR_SPREAD, OPT_TENSOR_INTERP, OPT_PRUNED_FFT) = range(16)
STAGES = ("sort", "spread", "fft", "deconv", "pad", "ifft", "interp")


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int),
        ("N", ctypes.c_int64 * 3),
        ("n", ctypes.c_int64 * 3),
        ("M", ctypes.c_int64),
        ("m", ctypes.c_int),
        ("taps", ctypes.c_int),
        ("window", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("method", ctypes.c_int),
        ("bin", ctypes.c_int * 3),
        ("n_bins", ctypes.c_int64),
        ("rhs_capacity", ctypes.c_int),
        ("threads", ctypes.c_int),
        ("device_bytes", ctypes.c_int64),
        ("sigma", ctypes.c_double * 3),
        ("max_subproblem", ctypes.c_int),
        ("spread_threads", ctypes.c_int),
        ("interp_threads", ctypes.c_int),
        ("sparse_points", ctypes.c_int),
        ("sparse_points_interp", ctypes.c_int),
        ("owner_spread", ctypes.c_int),
        ("kernel_launches", ctypes.c_int64),
        ("spread_block_threads", ctypes.c_int),
        ("interp_block_threads", ctypes.c_int),
        ("tensor_spread", ctypes.c_int),
        ("tensor_interp", ctypes.c_int),
        ("pruned_fft", ctypes.c_int),
    ]


class BatchItem(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int),
        ("N", ctypes.c_int64 * 3),
        ("M", ctypes.c_int64),
        ("sigma", ctypes.c_double),
        ("m", ctypes.c_int),
        ("window", ctypes.c_int),
        ("nrhs", ctypes.c_int),
    ]


class NFFTError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, status_string(status), status))


_lib = None


def _declare(lib):
    vp = ctypes.c_void_p
    i64p = ctypes.POINTER(ctypes.c_int64)
    sig = {
        "nfft_plan_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, i64p, ctypes.c_int64, ctypes.c_double,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]),
        "nfft_plan_destroy": (ctypes.c_int, [vp]),
        "nfft_set_points": (ctypes.c_int, [vp, vp]),
        "nfft_adjoint": (ctypes.c_int, [vp, vp, vp, ctypes.c_int]),
        "nfft_forward": (ctypes.c_int, [vp, vp, vp, ctypes.c_int]),
        "nfft_sync": (ctypes.c_int, [vp]),
        "nfft_set_stream": (ctypes.c_int, [vp, vp]),
        "nfft_set_option": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int64]),
        "nfft_get_info": (ctypes.c_int, [vp, ctypes.POINTER(PlanInfo)]),
        "nfft_stage_times": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_double), i64p, ctypes.c_int]),
        "nfft_plan_params": (ctypes.c_int, [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_int, ctypes.c_int, i64p,
                                            ctypes.POINTER(ctypes.c_int)]),
        "nfft_ewald_reciprocal": (ctypes.c_int, [vp, vp, ctypes.c_double, ctypes.c_double,
                                                  ctypes.POINTER(ctypes.c_double)]),
        "nfft_ewald_reciprocal_sum": (ctypes.c_int, [vp, vp, ctypes.c_double, ctypes.c_double, vp]),
        "nfft_ewald_reciprocal_forces": (ctypes.c_int, [vp, vp, ctypes.c_double, ctypes.c_double, vp]),
        "nfft_ewald_reciprocal_sum_noalloc": (ctypes.c_int, [ctypes.c_int, i64p, ctypes.c_int, vp, ctypes.c_double,
                                                              ctypes.c_double, vp, vp]),
        "nfft_ewald_real_space": (ctypes.c_int, [ctypes.c_int64, vp, vp, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_double, ctypes.POINTER(ctypes.c_double), vp]),
        "nfft_ewald_real_space_forces": (ctypes.c_int, [ctypes.c_int64, vp, vp, ctypes.c_double, ctypes.c_double,
                                                         ctypes.c_double, vp, ctypes.POINTER(ctypes.c_double), vp]),
        "nfft_batch_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(BatchItem), ctypes.c_int,
                                              vp]),
        "nfft_batch_destroy": (ctypes.c_int, [vp]),
        "nfft_batch_set_points": (ctypes.c_int, [vp, ctypes.POINTER(vp)]),
        "nfft_batch_adjoint": (ctypes.c_int, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp)]),
        "nfft_batch_forward": (ctypes.c_int, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp)]),
        "nfft_batch_sync": (ctypes.c_int, [vp]),
        "nfft_autotune": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
        "nfft_batch_autotune": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
        "nfft_batch_set_option": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int64]),
        "nfft_batch_stage_times": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_double), i64p, ctypes.c_int]),
        "nfft_mlp_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_uint64, vp]),
        "nfft_mlp_destroy": (ctypes.c_int, [vp]),
        "nfft_mlp_num_params": (ctypes.c_int, [vp, i64p]),
        "nfft_mlp_set_params": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_float)]),
        "nfft_mlp_get_params": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int]),
        "nfft_mlp_forward": (ctypes.c_int, [vp, vp, vp, ctypes.c_int]),
        "nfft_mlp_gradients": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_float)]),
        "nfft_mlp_train_step": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_int, ctypes.c_float, vp]),
        "nfft_picker_features": (ctypes.c_int, [ctypes.c_int, i64p, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                                ctypes.POINTER(ctypes.c_double)]),
        "nfft_picker_configure": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                                 ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                                 ctypes.c_double, ctypes.c_double]),
        "nfft_rule_of_thumb": (ctypes.c_int, [ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "nfft_pick_params": (ctypes.c_int, [vp, ctypes.c_int, i64p, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "nfft_deconv_amplification": (ctypes.c_int, [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "nfft_batch_kernel_launches": (ctypes.c_int, [vp, i64p]),
        "nfft_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "nfft_version": (ctypes.c_int, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load(path: str = LIB_PATH):
    """Load libgbnfft.so (built by __graft_entry__.build() or build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError("libgbnfft.so is not built (%s); run paper_2001_01583_gb300/build.py" % path)
        _lib = _declare(ctypes.CDLL(path))
    return _lib


def header_functions(path: str = HEADER):
    """Names of the functions include/gbnfft.h declares."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nfft_[a-z_0-9]+)\s*\(", text)))


def status_string(status: int) -> str:
    try:
        return load().nfft_status_string(int(status)).decode()
    except ImportError:
        return "status %d" % status


def check(status: int, what: str = "gbnfft"):
    if status != OK:
        raise NFFTError(status, what)
