"""ctypes loader for libginimds.so (the sm_103a CUDA library).

Only argument marshalling lives here.  If the library is missing the import of
any entry point raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# GINI_DEBUG=1 loads the debug build (device-side index checks, see
# gini_debug_checks in include/gini_mds.h), built by build.build(debug=True).
DEBUG = os.environ.get("GINI_DEBUG") == "1"
LIB_PATH = os.path.join(_HERE, "_build_debug" if DEBUG else "_build", "libginimds.so")

(GINI_OK, GINI_EINVAL, GINI_ENONFINITE, GINI_EDEGENERATE, GINI_ENOMEM, GINI_ECUDA, GINI_ETIMEOUT,
 GINI_EINDEX) = range(8)
DTYPES = {"f32": 0, "bf16": 1, "bf16x2": 2, "fp8": 3}
METRICS = {"gini": 0, "euclid": 1}
LOSSES = {"kruskal": 0, "sammon": 1}
LAYOUTS = {"full": 0, "tiled": 1}
OPS = {"rank": 0, "dist": 1, "stress": 2, "fit": 3, "stress_det": 4, "fit_det": 5, "dist_fp8": 6}

_c = ctypes
_vp = _c.c_void_p
_i64 = _c.c_int64


class Problem(_c.Structure):
    """Mirror of gini_problem in include/gini_mds.h."""
    _fields_ = [("X_dev", _vp), ("n", _i64), ("p", _i64), ("ldx", _i64)]


class BatchOpts(_c.Structure):
    """Mirror of gini_batch_opts in include/gini_mds.h."""
    _fields_ = [("deterministic", _c.c_int), ("delta_dtype", _c.c_int), ("tile_rows", _c.c_int),
                ("ctas_per_sm", _c.c_int)]


class FitArgs(_c.Structure):
    """Mirror of gini_fit_args in include/gini_mds.h."""
    _fields_ = [
        ("n", _i64), ("k", _c.c_int), ("nu", _c.c_double),
        ("delta_dev", _vp), ("layout", _c.c_int), ("dtype", _c.c_int), ("ldd", _i64),
        ("col_scale_dev", _vp), ("sum_delta2", _c.c_double), ("eta", _c.c_double),
        ("iters", _c.c_int), ("polish_iters", _c.c_int), ("Y_dev", _vp),
        ("history_dev", _vp), ("final_stress_dev", _vp), ("metric", _c.c_int),
        ("loss", _c.c_int), ("deterministic", _c.c_int),
    ]


# name -> (restype, argtypes); every symbol include/gini_mds.h declares.
SIGNATURES = {
    "gini_status_str": (_c.c_char_p, [_c.c_int]),
    "gini_last_cuda_error": (_c.c_char_p, []),
    "gini_version": (_c.c_int, []),
    "gini_launch_count": (_c.c_uint64, []),
    "gini_tile_size": (_c.c_int, []),
    "gini_tiled_elems": (_i64, [_i64]),
    "gini_workspace_size": (_c.c_size_t, [_c.c_int, _i64, _i64, _c.c_int, _c.c_int]),
    "gini_check": (_c.c_int, [_vp, _vp]),
    "gini_rank": (_c.c_int, [_vp, _i64, _i64, _i64, _vp, _vp, _c.c_size_t, _vp]),
    "gini_dist": (_c.c_int, [_vp, _i64, _i64, _i64, _c.POINTER(_c.c_double), _c.c_int,
                             _c.c_int, _c.c_int, _vp, _i64, _i64, _vp, _vp, _vp, _c.c_size_t,
                             _vp]),
    "gini_pack": (_c.c_int, [_vp, _i64, _i64, _c.c_int, _vp, _vp, _vp]),
    "gini_stress_grad": (_c.c_int, [_vp, _i64, _c.c_int, _c.c_double, _vp, _c.c_int, _c.c_int,
                                    _i64, _vp, _c.c_double, _vp, _vp, _vp, _c.c_size_t, _vp]),
    "gini_mds_fit": (_c.c_int, [_c.POINTER(FitArgs), _vp, _c.c_size_t, _vp]),
    "gini_stress_grad_ex": (_c.c_int, [_vp, _i64, _c.c_int, _c.c_double, _vp, _c.c_int,
                                       _c.c_int, _i64, _vp, _c.c_int, _c.c_int, _c.c_double,
                                       _vp, _vp, _vp, _c.c_size_t, _vp]),
    "gini_delta_sums": (_c.c_int, [_vp, _i64, _c.c_int, _c.c_int, _i64, _vp, _vp, _vp]),
    "gini_nu_search_workspace_size": (_c.c_size_t, [_i64, _i64, _vp, _c.c_int, _c.c_int,
                                                    _c.c_int, _c.c_int]),
    "gini_nu_search": (_c.c_int, [_vp, _i64, _i64, _i64, _vp, _c.c_int, _vp, _c.c_int, _c.c_int,
                                  _c.c_int, _c.c_double, _vp, _vp, _vp, _vp, _vp, _vp,
                                  _c.c_size_t, _vp]),
    "gini_alternating_nu_workspace_size": (_c.c_size_t, [_i64, _i64, _c.c_int, _c.c_int,
                                                         _c.c_int]),
    "gini_alternating_nu": (_c.c_int, [_vp, _i64, _i64, _i64, _c.c_int, _vp, _c.c_int,
                                       _c.c_double, _c.c_int, _c.c_int, _c.c_double, _c.c_int,
                                       _c.c_int, _vp, _vp, _vp, _vp, _c.c_size_t, _vp]),
    "gini_eval_workspace_size": (_c.c_size_t, [_i64, _c.c_int, _c.c_int]),
    "gini_neighbour_scores": (_c.c_int, [_vp, _i64, _i64, _i64, _vp, _c.c_int, _vp, _c.c_int,
                                         _c.c_int, _vp, _vp, _c.c_size_t, _vp]),
    "gini_silhouette": (_c.c_int, [_vp, _i64, _c.c_int, _vp, _c.c_int, _vp, _vp, _c.c_size_t,
                                   _vp]),
    "gini_distance_correlations": (_c.c_int, [_vp, _i64, _i64, _i64, _vp, _c.c_int, _c.c_int,
                                              _vp, _vp, _c.c_size_t, _vp]),
    "gini_selftest_wait_timeout": (_c.c_int, [_c.c_uint64, _vp, _c.c_size_t, _vp]),
    "gini_debug_checks": (_c.c_int, []),
    "gini_debug_index_record": (_c.c_int, [_vp, _c.POINTER(_c.c_uint32), _c.POINTER(_i64),
                                           _c.POINTER(_i64), _c.POINTER(_c.c_uint32)]),
    "gini_selftest_index_check": (_c.c_int, [_vp, _c.c_size_t, _vp]),
    "gini_cmds_workspace_size": (_c.c_size_t, [_i64, _c.c_int]),
    "gini_classical_mds": (_c.c_int, [_vp, _i64, _c.c_int, _c.c_int, _i64, _vp, _c.c_int,
                                      _c.c_int, _c.c_uint64, _vp, _vp, _vp, _c.c_size_t, _vp]),
    "gini_stress_grad_noalloc": (_c.c_int, [_vp, _i64, _c.c_int, _c.c_double, _vp, _c.c_int,
                                            _c.c_int, _i64, _vp, _c.c_double, _vp, _vp, _vp]),
    "gini_default_step": (_c.c_double, [_i64, _c.c_int, _c.c_double, _c.c_double, _c.c_double]),
    "gini_batch_workspace_size": (_c.c_size_t, [_c.POINTER(Problem), _c.c_int, _c.c_int,
                                                _c.c_int, _c.c_int, _c.POINTER(BatchOpts)]),
    "gini_fit_batched": (_c.c_int, [_c.POINTER(Problem), _c.c_int, _c.POINTER(_c.c_double),
                                    _c.c_int, _c.c_int, _c.c_int, _c.c_double, _vp, _vp, _vp,
                                    _vp, _c.POINTER(_c.c_int), _c.POINTER(BatchOpts), _vp,
                                    _c.c_size_t, _vp]),
    "gini_set_deterministic": (None, [_c.c_int]),
    "gini_get_deterministic": (_c.c_int, []),
}

_lib = None


class GiniError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().gini_status_str(status).decode()
        if status == GINI_ECUDA:
            msg += ": " + lib().gini_last_cuda_error().decode()
        super().__init__(f"{where}: {msg}")
        self.status = status


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            how = ("`python -c 'from paper_2605_25124_gb300 import build; build.build(debug=True)'`"
                   if DEBUG else "`python -c 'import __graft_entry__ as g; g.build()'`")
            raise RuntimeError(
                f"libginimds.so not found at {LIB_PATH}; build it with {how} (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int, where: str) -> None:
    if status != GINI_OK:
        raise GiniError(status, where)
