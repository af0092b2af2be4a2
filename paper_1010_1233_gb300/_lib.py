"""ctypes binding of libflb.so (include/flb.h): argument marshalling only.

The library is built in-tree by ``paper_1010_1233_gb300.build``.  There is no
fallback: if the shared library cannot be loaded every call raises.
"""
import ctypes
import os
from ctypes import POINTER, c_double, c_float, c_int, c_int32, c_size_t, c_uint16, c_uint32, c_uint64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libflb.so")
# the bounds-checked debug build (build.py --checked); chosen with FLB_CHECKED=1
CHECKED_LIB_PATH = os.path.join(HERE, "libflb_checked.so")
if os.environ.get("FLB_CHECKED") == "1":
    LIB_PATH = CHECKED_LIB_PATH

FLB_OK, FLB_EINVAL, FLB_ENOMEM, FLB_ECUDA, FLB_EUNSTABLE, FLB_ETIMEOUT, FLB_ESTATE = 0, -1, -2, -3, -4, -5, -6
FLB_D1Q3, FLB_D2Q9, FLB_D3Q15, FLB_D3Q19 = 1, 2, 3, 4
FLB_FP64, FLB_FP32_DEV = 0, 1
FIELD_UX, FIELD_UY = 9, 10
FLB_NET_WARP, FLB_NET_TCGEN05 = 0, 1


class FlbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"flb error {code}: {msg}")
        self.code = code


class flb_replica(ctypes.Structure):
    _fields_ = [("lattice", c_int32), ("nx", c_int32), ("ny", c_int32), ("tau", c_double * 20),
                ("rho0", c_double), ("kT", c_double), ("u0", c_double * 3), ("seed", c_uint64),
                ("stream", c_uint32), ("noise_mask", c_uint32), ("init_mode", c_uint32),
                ("field_mask", c_uint32), ("noise_mode", c_uint32), ("nz", c_int32)]


_SIGS = {
    "flb_workspace_bytes": (c_int, [c_int, POINTER(flb_replica), c_int, POINTER(c_size_t)]),
    "flb_create": (c_int, [c_int, POINTER(flb_replica), c_int, c_void_p, c_size_t, c_void_p, POINTER(c_void_p)]),
    "flb_run": (c_int, [c_void_p, c_uint64, c_uint32]),
    "flb_sync": (c_int, [c_void_p]),
    "flb_reset_stats": (c_int, [c_void_p]),
    "flb_get_correlator": (c_int, [c_void_p, c_int, c_int, c_int, POINTER(c_double), POINTER(c_uint64)]),
    "flb_get_populations": (c_int, [c_void_p, c_int, POINTER(c_double)]),
    "flb_set_populations": (c_int, [c_void_p, c_int, POINTER(c_double)]),
    "flb_get_populations_window": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, POINTER(c_double)]),
    "flb_get_conserved": (c_int, [c_void_p, c_int, POINTER(c_double)]),
    "flb_get_fields": (c_int, [c_void_p, c_int, POINTER(c_double)]),
    "flb_mlp_param_count": (c_int, []),
    "flb_mlp_gram": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p, c_void_p]),
    "flb_mlp_scratch_bytes": (c_int, [c_int, c_int, POINTER(c_size_t)]),
    "flb_mlp_train_step": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_float, c_float, c_float, c_float,
                                   c_void_p, c_int, c_int, c_void_p, c_int, c_int, c_void_p, c_void_p,
                                   c_void_p, c_void_p, c_size_t, c_void_p]),
    "flb_get_step": (c_int, [c_void_p, POINTER(c_uint64)]),
    "flb_time_correlator_bytes": (c_int, [c_void_p, c_int, c_int, POINTER(c_size_t)]),
    "flb_set_time_correlator": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_size_t]),
    "flb_set_time_correlator3": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                                         c_size_t]),
    "flb_get_time_correlator": (c_int, [c_void_p, c_int, c_int, c_int, POINTER(c_double), POINTER(c_uint64)]),
    "flb_set_mlp": (c_int, [c_void_p, POINTER(c_uint16), POINTER(c_float), c_int]),
    "flb_save": (c_int, [c_void_p, c_void_p, POINTER(c_size_t)]),
    "flb_load": (c_int, [c_void_p, c_void_p, c_size_t]),
    "flb_set_step_config": (c_int, [c_void_p, c_int, c_int, c_int]),
    "flb_get_step_config": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
    "flb_set_network_engine": (c_int, [c_void_p, c_int]),
    "flb_get_network_engine": (c_int, [c_void_p, POINTER(c_int)]),
    "flb_autotune": (c_int, [c_void_p, c_int, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_double)]),
    "flb_set_graphs": (c_int, [c_void_p, c_int]),
    "flb_kernel_launches": (c_int, [c_void_p, POINTER(c_uint64)]),
    "flb_probe_wait_timeout": (c_int, [c_void_p, c_uint64]),
    "flb_debug_bounds": (c_int, [POINTER(c_uint64), POINTER(c_uint32), c_int]),
    "flb_destroy": (None, [c_void_p]),
    "flb_last_error": (ctypes.c_char_p, []),
    "flb_spectra_scratch_bytes": (c_int, [c_int, c_int, c_int, c_int, POINTER(c_size_t), POINTER(c_size_t)]),
    "flb_spectra_accumulate": (c_int, [c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                                       c_size_t, c_void_p]),
    "flb_spectra_accumulate_static": (c_int, [c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                              c_void_p]),
    "flb_stability": (c_int, [POINTER(flb_replica), c_int, POINTER(c_double), POINTER(c_int32)]),
    "flb_philox": (c_int, [c_void_p, c_int, c_uint32, c_uint32, c_uint32, c_uint32, c_uint64, c_int,
                           c_void_p, c_void_p, c_void_p]),
}

_lib = None


def lib():
    """Load libflb.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with python -m paper_1010_1233_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(rc):
    if rc != FLB_OK:
        raise FlbError(rc, lib().flb_last_error().decode())
    return rc


def exported_symbols():
    return list(_SIGS)
