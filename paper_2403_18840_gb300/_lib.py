"""ctypes binding of libfdcore (include/fdcore.h): argument marshalling only.

The library is built in-tree by ``paper_2403_18840_gb300.build``; importing
this module without it raises -- there is no fallback path.
"""
import ctypes
import os

from . import build as _build

FD_OK, FD_EINVAL, FD_EFORMAT, FD_ENOMEM, FD_ECUDA, FD_ETIMEOUT, FD_ENOTSUP = range(7)
FD_TILE_SAMPLES = 16384


class FdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("fdcore status %d: %s" % (status, msg))
        self.status = status


class fd_jit_options(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in ("threads", "min_blocks", "max_modules", "root_units", "sync_every",
                                              "leaf_calls", "spt", "unit_cap", "pair", "sv_smem", "cross_roots",
                                              "leaf_cache", "lc_global")]


class fd_params(ctypes.Structure):
    _fields_ = [("k_ext", ctypes.c_double), ("k_F", ctypes.c_double), ("mu", ctypes.c_double),
                ("beta", ctypes.c_double), ("Lambda", ctypes.c_double), ("k_cut", ctypes.c_double),
                ("order", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_c = ctypes
_vp = _c.c_void_p
_i32 = _c.c_int32
_i64 = _c.c_int64
_u64 = _c.c_uint64
_f32 = _c.c_float
_f64 = _c.c_double
_pd = _c.POINTER(_c.c_double)
_pf = _c.POINTER(_c.c_float)
_pi = _c.POINTER(_c.c_int32)

# name: (restype, argtypes)
SIGNATURES = {
    "fd_last_error": (_c.c_char_p, []),
    "fd_device_status": (_i32, [_vp]),
    "fd_debug_set_wait_polls": (_i32, [_i64]),
    "fd_graph_load": (_i32, [_vp, _c.c_size_t, _c.POINTER(_vp)]),
    "fd_graph_info": (_i32, [_vp, _pi, _pi, _c.POINTER(_i64), _pi]),
    "fd_graph_roots": (_i32, [_vp, _pi]),
    "fd_graph_free": (None, [_vp]),
    "fd_graph_set_launch": (_i32, [_vp, _i32, _i32]),
    "fd_graph_jit": (_i32, [_vp, _c.POINTER(fd_jit_options), _c.c_char_p]),
    "fd_graph_jit_enable": (_i32, [_vp, _i32]),
    "fd_graph_jit_info": (_i32, [_vp, _pi, _c.POINTER(_c.c_double)]),
    "fd_jit_emit": (_i32, [_vp, _c.c_size_t, _c.POINTER(fd_jit_options), _i32, _c.c_char_p, _i64,
                           _c.POINTER(_i64), _pi]),
    "fd_vegas_create": (_i32, [_i32, _i32, _c.POINTER(_vp)]),
    "fd_vegas_free": (None, [_vp]),
    "fd_vegas_set_edges": (_i32, [_vp, _pd]),
    "fd_vegas_get_edges": (_i32, [_vp, _pd]),
    "fd_vegas_get_hist": (_i32, [_vp, _pd]),
    "fd_vegas_set_hist": (_i32, [_vp, _pd]),
    "fd_vegas_clear_hist": (_i32, [_vp, _vp]),
    "fd_vegas_update": (_i32, [_vp, _f64, _vp]),
    "fd_vegas_update_batch": (_i32, [_c.POINTER(_vp), _i32, _f64, _vp]),
    "fd_integrand_eval_iter_dev": (_i32, [_c.POINTER(_vp), _i32, _c.POINTER(fd_params), _pi, _i32,
                                          _c.POINTER(_vp), _u64, _u64, _vp, _i64, _vp, _vp]),
    "fd_counter_add": (_i32, [_vp, _c.c_uint32, _vp]),
    "fd_map_samples": (_i32, [_vp, _u64, _u64, _i32, _i64, _i32, _vp, _vp, _vp]),
    "fd_integrand_eval": (_i32, [_c.POINTER(_vp), _i32, _c.POINTER(fd_params), _pi, _i32,
                                 _c.POINTER(_vp), _vp, _vp, _u64, _u64, _i64, _vp, _vp, _vp]),
    "fd_integrand_eval_target": (_i32, [_c.POINTER(_vp), _i32, _c.POINTER(fd_params), _pi, _i32,
                                        _c.POINTER(_vp), _vp, _vp, _u64, _u64, _i64, _vp, _vp, _vp]),
    "fd_partials_count": (_i64, [_i32, _i32, _i64]),
    "fd_tile_samples": (_i64, [_i64]),
    "fd_integrand_eval_stats_noalloc": (_i32, [_c.POINTER(_vp), _i32, _c.POINTER(fd_params), _pi, _i32,
                                               _c.POINTER(_vp), _vp, _vp, _u64, _u64, _i64, _vp, _vp, _vp]),
    "fd_accumulate": (_i32, [_vp, _i32, _i32, _i64, _vp, _vp]),
    "fd_flow_create": (_i32, [_i32, _i32, _i32, _u64, _c.POINTER(_vp)]),
    "fd_flow_free": (None, [_vp]),
    "fd_flow_param_count": (_i64, [_vp]),
    "fd_flow_set_params": (_i32, [_vp, _pf, _i64]),
    "fd_flow_get_params": (_i32, [_vp, _pf, _i64]),
    "fd_flow_sample": (_i32, [_vp, _u64, _u64, _i32, _i64, _vp, _vp, _vp]),
    "fd_flow_sample_defensive": (_i32, [_vp, _u64, _u64, _i32, _i64, _f64, _vp, _vp, _c.POINTER(_c.c_double), _vp]),
    "fd_flow_set_tensor_path": (_i32, [_vp, _i32]),
    "fd_flow_log_density": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "fd_flow_grad": (_i32, [_vp, _vp, _vp, _i64, _vp, _vp, _vp]),
    "fd_flow_train": (_i32, [_vp, _vp, _vp, _i64, _i32, _f32, _pf, _vp]),
    "fd_measure_peak": (_i32, [_i32, _pd]),
    "fd_mcmc_chains": (_i32, [_vp, _i32, _i64, _i32, _i64, _i32, _f64, _u64, _u64, _i32, _vp, _vp, _vp]),
    "fd_nsf_create": (_i32, [_i32, _i32, _c.POINTER(_vp)]),
    "fd_nsf_free": (None, [_vp]),
    "fd_nsf_param_count": (_i64, [_vp]),
    "fd_nsf_set_params": (_i32, [_vp, _pf, _i64]),
    "fd_nsf_forward": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp]),
    "fd_nsf_set_tensor_path": (_i32, [_vp, _i32]),
    "fd_nsf_sample": (_i32, [_vp, _u64, _u64, _i32, _i64, _vp, _vp, _vp]),
    "fd_nsf_sample_w": (_i32, [_vp, _u64, _u64, _i32, _i64, _vp, _vp, _vp]),
    "fd_nsf_log_density": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp]),
    "fd_nsf_kl_grad": (_i32, [_vp, _vp, _vp, _i64, _vp, _vp, _vp]),
    "fd_nsf_train": (_i32, [_vp, _vp, _vp, _i64, _i32, _f32, _vp, _vp]),
    "fd_nsf_get_params": (_i32, [_vp, _pf, _i64]),
    "fd_mcmc_estimate": (_i32, [_vp, _i32, _i64, _i32, _vp, _vp]),
    "fd_postprocess": (_i32, [_i32, _pd, _pd, _pd, _f64, _f64, _f64, _pd, _pd, _pd, _pd]),
}

_lib = None


def lib(build_if_missing=True):
    """The loaded library (built first when sources changed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise FdError(FD_ENOTSUP, "libfdcore.so is missing (run paper_2403_18840_gb300.build.build())")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        if not hasattr(L, name):
            continue
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(status):
    if status != FD_OK:
        raise FdError(status, lib().fd_last_error().decode())
    return status
