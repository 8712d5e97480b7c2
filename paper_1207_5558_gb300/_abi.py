"""ctypes binding of libslsht (include/slsht.h): the same names, argument
marshalling only.  Every step of the transform runs in the library's CUDA
kernels; if the library is missing this module raises instead of falling back.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libslsht.so")
HEADER = os.path.join(HERE, "..", "include", "slsht.h")

SLSHT_OK = 0
SLSHT_PENDING = 1
SLSHT_E_ARG = -1
SLSHT_E_H00 = -2
SLSHT_E_NOMEM = -3
SLSHT_E_BUSY = -4
SLSHT_E_TIMEOUT = -5
SLSHT_E_CUDA = -6
SLSHT_E_STATE = -7

SLSHT_FP64 = 0
SLSHT_FP32_BULK = 1

SLSHT_OPT_BETA_ROUTE = 1
SLSHT_OPT_ALPHA_ENGINE = 2
SLSHT_OPT_CHUNK_PAIRS = 3
SLSHT_OPT_GAUNT_TABLE = 4
SLSHT_OPT_WAIT_TEST = 5
SLSHT_OPT_REAL_FIELDS = 6
SLSHT_OPT_COUPLING = 7
SLSHT_OPT_FP64_ARITH = 8
SLSHT_OPT_WINDOW_ORDERS = 9
SLSHT_OPT_ROTWIN_ENGINE = 10

SLSHT_BATCH_NO_GRAPH = 1
SLSHT_BATCH_NO_TUNE = 2
SLSHT_BATCH_NO_TC = 4
SLSHT_BATCH_NO_DD = 8
SLSHT_BATCH_FP64_DD = 16

SLSHT_BQ_TILE_COLS = 1
SLSHT_BQ_ALPHA_FORM = 2
SLSHT_BQ_TUNED = 3
SLSHT_BQ_TILES = 4
SLSHT_BQ_KERNELS = 5
SLSHT_BQ_GRAPH = 6
SLSHT_BQ_BYTES = 7
SLSHT_BQ_SAMPLES = 8
SLSHT_BQ_ENGINE = 9

SLSHT_NSTAGES = 8
SLSHT_NOALLOC_SCRATCH_BYTES = 32 << 20
STAGE_NAMES = ["tables", "couple", "ctensor", "beta_gamma", "alpha", "inverse", "copy", "other"]


class slsht_desc(ctypes.Structure):
    _fields_ = [("L_f", ctypes.c_int32), ("L_h", ctypes.c_int32), ("n_alpha", ctypes.c_int32),
                ("n_beta", ctypes.c_int32), ("n_gamma", ctypes.c_int32), ("prec", ctypes.c_int32)]


class slsht_batch_item(ctypes.Structure):
    _fields_ = [("desc", slsht_desc), ("f_lm", ctypes.c_void_p), ("h_lm", ctypes.c_void_p),
                ("lm", ctypes.c_void_p), ("n_pairs", ctypes.c_int32), ("g_out", ctypes.c_void_p)]


class slsht_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64 * SLSHT_NSTAGES), ("ms", ctypes.c_double * SLSHT_NSTAGES),
                ("samples_written", ctypes.c_uint64)]


_lib = None


def load(path=LIB_PATH):
    """Load libslsht.so once; raises RuntimeError when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libslsht.so not found at %s: run __graft_entry__.build() "
                           "(there is no CPU fallback)" % path)
    lib = ctypes.CDLL(path)
    vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    sig = {
        "slsht_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_size_t]),
        "slsht_destroy": (None, [vp]),
        "slsht_forward": (ctypes.c_int, [vp, ctypes.POINTER(slsht_desc), vp, vp, vp, i32, vp, vp]),
        "slsht_inverse": (ctypes.c_int, [vp, ctypes.POINTER(slsht_desc), vp, vp, vp, i32, vp, vp]),
        "slsht_inverse_alt": (ctypes.c_int, [vp, ctypes.POINTER(slsht_desc), vp, vp, vp, i32, i32, vp, i32, vp,
                                             vp]),
        "slsht_steer_gamma": (ctypes.c_int, [vp, ctypes.POINTER(slsht_desc), vp, i32, vp, i32, i32, vp, vp]),
        "slsht_forward_noalloc": (ctypes.c_int, [ctypes.POINTER(slsht_desc), vp, vp, vp, i32, vp, vp]),
        "slsht_forward_windows": (ctypes.c_int, [vp, ctypes.POINTER(slsht_desc), vp, i32, vp, vp, i32, vp, vp]),
        "slsht_window_ellipse": (ctypes.c_int, [vp, i32, ctypes.c_double, ctypes.c_double, i32, i32, vp,
                                                ctypes.POINTER(ctypes.c_double), vp]),
        "slsht_batch_create": (ctypes.c_int, [vp, i32, ctypes.POINTER(slsht_batch_item), i32, vp,
                                              ctypes.POINTER(vp)]),
        "slsht_batch_launch": (ctypes.c_int, [vp, vp]),
        "slsht_tune": (ctypes.c_int, [vp, ctypes.POINTER(slsht_desc)]),
        "slsht_batch_query": (ctypes.c_int, [vp, i32, i32, ctypes.POINTER(i64)]),
        "slsht_batch_destroy": (None, [vp]),
        "slsht_submit": (ctypes.c_int, [vp, ctypes.POINTER(slsht_desc), vp, vp, vp, i32, vp,
                                        ctypes.POINTER(u64)]),
        "slsht_poll": (ctypes.c_int, [vp, u64]),
        "slsht_poll_times": (ctypes.c_int, [vp, u64, vp]),
        "slsht_drain": (ctypes.c_int, [vp, i64]),
        "slsht_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "slsht_last_error": (ctypes.c_char_p, []),
        "slsht_check_args": (ctypes.c_int, [ctypes.POINTER(slsht_desc), vp, i32]),
        "slsht_profile": (ctypes.c_int, [vp, ctypes.c_int]),
        "slsht_get_stats": (ctypes.c_int, [vp, ctypes.POINTER(slsht_stats), ctypes.c_int]),
        "slsht_set_option": (ctypes.c_int, [vp, ctypes.c_int, i64]),
        "slsht_mem_used": (ctypes.c_size_t, [vp]),
        "slsht_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def header_functions(path=HEADER):
    """Names of every function the C header declares."""
    import re
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(slsht_[a-z_0-9]+)\s*\(", txt)))


def ptr(x):
    """Device or host address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    if hasattr(x, "ctypes"):
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError("cannot take the address of %r" % type(x))


class SlshtError(RuntimeError):
    def __init__(self, code, where):
        lib = load()
        msg = "%s: %s (%d)" % (where, lib.slsht_strerror(code).decode(), code)
        if code in (SLSHT_E_CUDA, SLSHT_E_TIMEOUT, SLSHT_E_NOMEM):
            msg += ": " + lib.slsht_last_error().decode()
        super().__init__(msg)
        self.code = code


def check(code, where):
    if code < 0:
        raise SlshtError(code, where)
    return code
