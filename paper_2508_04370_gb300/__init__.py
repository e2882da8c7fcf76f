"""GB300 (sm_103a) multifrontal LDL^T factorise/solve for the regularised
interior point method of Zanetti & Gondzio (arXiv 2508.04370, Sec. 3-4).

Thin ctypes binding of the C ABI in include/ipm_mf.h: every function below
has the C name and only marshals arguments (torch tensors or integer device
pointers for device buffers, numpy arrays for host buffers, a torch stream
or raw cudaStream_t handle for streams).  All numeric work runs in the CUDA
library; importing this package fails if the library has not been built.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libipm_mf.so")
INCLUDE = os.path.join(os.path.dirname(_HERE), "include", "ipm_mf.h")

IPM_OK = 0
IPM_ERR_INVALID_ARG = -1
IPM_ERR_NOT_ANALYSED = -2
IPM_ERR_OOM = -3
IPM_ERR_CUDA = -4
IPM_ERR_NONFINITE = -5
IPM_ERR_DEVICE_TIMEOUT = -6
IPM_ERR_NOT_FACTORISED = -7
IPM_ERR_NO_DEVICE = -8
IPM_ERR_SCRATCH_TOO_SMALL = -9
IPM_WARN_DYNREG_APPLIED = 1
IPM_WARN_LARGE_REG = 2
IPM_WARN_REFINE_NOT_CONVERGED = 3

IPM_FORM_AUTO = 0
IPM_FORM_AUGMENTED = 1
IPM_FORM_NORMAL = 2
IPM_ORD_AMD = 0
IPM_ORD_ND = 1
IPM_ORD_USER = 2
IPM_ORD_NATURAL = 3
IPM_PREC_FP64 = 0
IPM_PREC_MIXED = 1
IPM_PREC_SLICED = 2
IPM_SCHED_AUTO = 0
IPM_SCHED_LEVELS = 1
IPM_SCHED_DEPENDENCY = 2


class ipm_options(ct.Structure):
    _fields_ = [
        ("nb", ct.c_int32),
        ("amalg_width", ct.c_int32),
        ("amalg_zero_frac", ct.c_double),
        ("eps_piv", ct.c_double),
        ("large_reg", ct.c_double),
        ("precision", ct.c_int32),
        ("mixed_min_front", ct.c_int32),
        ("omega_target", ct.c_double),
        ("refine_max", ct.c_int32),
        ("gmres_restarts", ct.c_int32),
        ("nd_leaf", ct.c_int32),
        ("dense_row_factor", ct.c_double),
        ("device", ct.c_int32),
        ("spin_limit_log2", ct.c_int32),
        ("verbose", ct.c_int32),
        ("level_kernel", ct.c_int32),
        ("pivoting", ct.c_int32),
        ("schedule", ct.c_int32),
    ]


class ipm_info(ct.Structure):
    _fields_ = [
        ("m", ct.c_int32), ("n", ct.c_int32), ("N", ct.c_int32), ("form", ct.c_int32), ("ordering", ct.c_int32),
        ("nsuper", ct.c_int32), ("nlevels", ct.c_int32), ("nfronts_small", ct.c_int32),
        ("nfronts_large", ct.c_int32), ("max_front", ct.c_int32), ("max_k", ct.c_int32),
        ("nnz_A", ct.c_int64), ("nnz_K_lower", ct.c_int64), ("nnz_L", ct.c_int64),
        ("flops_factor", ct.c_double), ("flops_tensor", ct.c_double), ("device_bytes", ct.c_int64),
        ("npos", ct.c_int32), ("nneg", ct.c_int32), ("ndynreg", ct.c_int32),
        ("max_dynreg", ct.c_double), ("norm_K1", ct.c_double), ("refine_steps", ct.c_int32),
        ("gmres_iters", ct.c_int32), ("omega", ct.c_double), ("omega_hist", ct.c_double * 16), ("status", ct.c_int32),
        ("ms_analyse", ct.c_double), ("est_cost_ne", ct.c_double), ("est_cost_as", ct.c_double),
        ("nnz_ne_seen", ct.c_int64), ("precision_fallbacks", ct.c_int32), ("mixed_active", ct.c_int32),
        ("tune_small_threads", ct.c_int32 * 3), ("tune_level_ratio", ct.c_double), ("tune_ms", ct.c_double),
        ("amalg_zero_frac", ct.c_double), ("tune_level_ctas_per_sm", ct.c_int32), ("graph_kernels", ct.c_int32),
        ("schedule", ct.c_int32), ("steps_levels", ct.c_int32), ("steps_dependency", ct.c_int32),
        ("nfronts_thin", ct.c_int32),
    ]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["omega_hist"] = list(self.omega_hist)[: min(16, max(self.refine_steps - self.gmres_iters + 1, 1))]
        d["tune_small_threads"] = list(self.tune_small_threads)
        return d


class ipm_kernel_stat(ct.Structure):
    _fields_ = [("launches", ct.c_int64), ("ms", ct.c_double), ("flops", ct.c_double), ("bytes", ct.c_double)]


KERNEL_CLASSES = ["small_fronts", "large_assemble", "large_panel", "large_update", "large_update_tc", "forward",
                  "backward", "residual", "other", "slice", "pivot_block"]

_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
    lib = ct.CDLL(LIB_PATH)
    P = ct.c_void_p
    I = ct.c_int
    lib.ipm_default_options.argtypes = [ct.POINTER(ipm_options)]
    lib.ipm_default_options.restype = None
    lib.ipm_create.argtypes = [ct.POINTER(P), ct.POINTER(ipm_options)]
    lib.ipm_destroy.argtypes = [P]
    lib.ipm_analyse.argtypes = [P, ct.c_int32, ct.c_int32, P, P, ct.c_int32, ct.c_int32, P]
    lib.ipm_analyse_batch.argtypes = [P, ct.c_int32, P, P, P, P, ct.c_int32]
    lib.ipm_set_values.argtypes = [P, P, P]
    lib.ipm_save_analysis.argtypes = [P, ct.c_char_p]
    lib.ipm_load_analysis.argtypes = [P, ct.c_char_p]
    lib.ipm_factorise.argtypes = [P, P, ct.c_double, ct.c_double, P]
    lib.ipm_autotune.argtypes = [P, P, ct.c_double, ct.c_double, ct.c_int32, P]
    lib.ipm_set_launch_shapes.argtypes = [P, P, ct.c_double]
    lib.ipm_set_level_ctas.argtypes = [P, ct.c_int32]
    lib.ipm_solve.argtypes = [P, P, P, P, P, P]
    lib.ipm_iterate_host.argtypes = [P, P, ct.c_double, ct.c_double, ct.c_int32, P, P, P, P, P]
    lib.ipm_sync_status.argtypes = [P, P]
    lib.ipm_get_info.argtypes = [P, ct.POINTER(ipm_info)]
    lib.ipm_get_symbolic.argtypes = [P, P, P, P, P, P, P, P]
    lib.ipm_get_sizes.argtypes = [P, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int64),
                                  ct.POINTER(ct.c_int64)]
    lib.ipm_get_factor.argtypes = [P, P, P, P]
    lib.ipm_graph_capture.argtypes = [P, P, ct.c_double, ct.c_double, P, P, P, P, ct.c_int32, P]
    lib.ipm_graph_launch.argtypes = [P, P]
    lib.ipm_launch_counts.argtypes = [P, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32)]
    lib.ipm_solve_noalloc.argtypes = [P, P, P, P, P, P]
    lib.ipm_test_recip_pivot.argtypes = [P, P, P, ct.c_int64, P]
    lib.ipm_get_pivots.argtypes = [P, P, P, P]
    lib.ipm_measure_fp64_peak.argtypes = [ct.c_int32, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]
    lib.ipm_set_profiling.argtypes = [P, ct.c_int32]
    lib.ipm_kernel_stats.argtypes = [P, P, ct.c_int32]
    lib.ipm_kernel_trace.argtypes = [P, P, P, P, P, ct.c_int32, P]
    for name in ("ipm_create", "ipm_destroy", "ipm_analyse", "ipm_analyse_batch", "ipm_set_values", "ipm_factorise",
                 "ipm_solve", "ipm_iterate_host", "ipm_sync_status", "ipm_get_info", "ipm_get_symbolic",
                 "ipm_get_sizes", "ipm_get_factor", "ipm_graph_capture", "ipm_graph_launch", "ipm_launch_counts",
                 "ipm_set_profiling", "ipm_kernel_stats", "ipm_solve_noalloc", "ipm_test_recip_pivot",
                 "ipm_measure_fp64_peak", "ipm_get_pivots", "ipm_kernel_trace"):
        getattr(lib, name).restype = I
    _lib = lib
    return lib


def library():
    """The loaded ctypes library (raises ImportError if not built)."""
    return _load()


# ------------------------------------------------------------ marshalling

def _dptr(x):
    """Device pointer of a torch CUDA tensor (or an int address)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if getattr(x, "is_cuda", False):
        if not x.is_contiguous():
            raise ValueError("device buffers must be contiguous")
        return x.data_ptr()
    raise TypeError("expected a CUDA tensor or an integer device address")


def _hptr(a, dtype):
    """Host pointer of a numpy array with the exact dtype (kept alive by caller)."""
    if a is None:
        return None
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"expected a C-contiguous numpy array of {dtype}")
    return a.ctypes.data


def _stream(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# -------------------------------------------------------------- C names

def ipm_default_options() -> ipm_options:
    o = ipm_options()
    _load().ipm_default_options(ct.byref(o))
    return o


def ipm_create(opt: ipm_options | None = None):
    h = ct.c_void_p()
    rc = _load().ipm_create(ct.byref(h), ct.byref(opt) if opt is not None else None)
    if rc:
        raise RuntimeError(f"ipm_create failed ({rc})")
    return h


def ipm_destroy(ctx) -> int:
    return _load().ipm_destroy(ctx)


def ipm_analyse(ctx, m, n, colptr, rowidx, form=IPM_FORM_AUGMENTED, ordering=IPM_ORD_AMD, user_perm=None) -> int:
    cp = np.ascontiguousarray(colptr, dtype=np.int64)
    ri = np.ascontiguousarray(rowidx, dtype=np.int32)
    up = None if user_perm is None else np.ascontiguousarray(user_perm, dtype=np.int32)
    return _load().ipm_analyse(ctx, int(m), int(n), _hptr(cp, np.int64), _hptr(ri, np.int32), int(form),
                               int(ordering), _hptr(up, np.int32) if up is not None else None)


def ipm_analyse_batch(ctx, ms, ns, colptrs, rowidxs, ordering=IPM_ORD_AMD) -> int:
    ms = np.ascontiguousarray(ms, dtype=np.int32)
    ns = np.ascontiguousarray(ns, dtype=np.int32)
    cps = np.ascontiguousarray(colptrs, dtype=np.int64)
    ris = np.ascontiguousarray(rowidxs, dtype=np.int32)
    return _load().ipm_analyse_batch(ctx, int(ms.size), _hptr(ms, np.int32), _hptr(ns, np.int32),
                                     _hptr(cps, np.int64), _hptr(ris, np.int32), int(ordering))


def ipm_save_analysis(ctx, path) -> int:
    return _load().ipm_save_analysis(ctx, os.fsencode(path))


def ipm_load_analysis(ctx, path) -> int:
    return _load().ipm_load_analysis(ctx, os.fsencode(path))


def ipm_set_values(ctx, Ax_dev, stream=None) -> int:
    return _load().ipm_set_values(ctx, _dptr(Ax_dev), _stream(stream))


def ipm_factorise(ctx, theta_dev, rho, delta, stream=None) -> int:
    return _load().ipm_factorise(ctx, _dptr(theta_dev), float(rho), float(delta), _stream(stream))


def ipm_autotune(ctx, theta_dev, rho, delta, reps=3, stream=None) -> int:
    return _load().ipm_autotune(ctx, _dptr(theta_dev), float(rho), float(delta), int(reps), _stream(stream))


def ipm_set_level_ctas(ctx, per_sm=0) -> int:
    return _load().ipm_set_level_ctas(ctx, int(per_sm))


def ipm_set_launch_shapes(ctx, small_threads=None, level_ratio=-1.0) -> int:
    arr = None if small_threads is None else np.ascontiguousarray(small_threads, dtype=np.int32)
    ptr = None if arr is None else _hptr(arr, np.int32)
    return _load().ipm_set_launch_shapes(ctx, ptr, float(level_ratio))


def ipm_solve(ctx, r7_dev, r1_dev, dx_dev, dy_dev, stream=None) -> int:
    return _load().ipm_solve(ctx, _dptr(r7_dev), _dptr(r1_dev), _dptr(dx_dev), _dptr(dy_dev), _stream(stream))


def ipm_solve_noalloc(ctx, r7_dev, r1_dev, dx_dev, dy_dev, stream=None) -> int:
    """ipm_solve without any device allocation (fixed file-scope work space)."""
    return _load().ipm_solve_noalloc(ctx, _dptr(r7_dev), _dptr(r1_dev), _dptr(dx_dev), _dptr(dy_dev),
                                     _stream(stream))


def ipm_iterate_host(ctx, theta, rho, delta, r7, r1, dx, dy, nrhs=1, stream=None) -> int:
    return _load().ipm_iterate_host(ctx, _hptr(theta, np.float64), float(rho), float(delta), int(nrhs),
                                    _hptr(r7, np.float64), _hptr(r1, np.float64), _hptr(dx, np.float64),
                                    _hptr(dy, np.float64), _stream(stream))


def ipm_sync_status(ctx, stream=None) -> int:
    return _load().ipm_sync_status(ctx, _stream(stream))


def ipm_get_info(ctx):
    info = ipm_info()
    rc = _load().ipm_get_info(ctx, ct.byref(info))
    return rc, info


def ipm_get_sizes(ctx):
    N, ns = ct.c_int32(), ct.c_int32()
    nr, nl = ct.c_int64(), ct.c_int64()
    rc = _load().ipm_get_sizes(ctx, ct.byref(N), ct.byref(ns), ct.byref(nr), ct.byref(nl))
    if rc:
        raise RuntimeError(f"ipm_get_sizes failed ({rc})")
    return N.value, ns.value, nr.value, nl.value


def ipm_get_symbolic(ctx):
    N, ns, nr, _ = ipm_get_sizes(ctx)
    out = dict(perm=np.empty(N, np.int32), etree=np.empty(N, np.int32), colcount=np.empty(N, np.int64),
               snode_ptr=np.empty(ns + 1, np.int32), sn_parent=np.empty(ns, np.int32),
               sn_rptr=np.empty(ns + 1, np.int64), sn_rows=np.empty(max(nr, 1), np.int32))
    rc = _load().ipm_get_symbolic(ctx, _hptr(out["perm"], np.int32), _hptr(out["etree"], np.int32),
                                  _hptr(out["colcount"], np.int64), _hptr(out["snode_ptr"], np.int32),
                                  _hptr(out["sn_parent"], np.int32), _hptr(out["sn_rptr"], np.int64),
                                  _hptr(out["sn_rows"], np.int32))
    if rc:
        raise RuntimeError(f"ipm_get_symbolic failed ({rc})")
    out["sn_rows"] = out["sn_rows"][:nr]
    out["amalg_zero_frac"] = ipm_get_info(ctx)[1].amalg_zero_frac
    return out


def ipm_get_factor(ctx):
    N, ns, nr, nl = ipm_get_sizes(ctx)
    L = np.empty(max(nl, 1), np.float64)
    D = np.empty(max(N, 1), np.float64)
    dyn = np.empty(max(N, 1), np.float64)
    rc = _load().ipm_get_factor(ctx, _hptr(L, np.float64), _hptr(D, np.float64), _hptr(dyn, np.float64))
    if rc:
        raise RuntimeError(f"ipm_get_factor failed ({rc})")
    return L[:nl], D[:N], dyn[:N]


def ipm_graph_capture(ctx, theta_dev, rho, delta, r7_dev, r1_dev, dx_dev, dy_dev, nsolves=1, stream=None) -> int:
    return _load().ipm_graph_capture(ctx, _dptr(theta_dev), float(rho), float(delta), _dptr(r7_dev), _dptr(r1_dev),
                                     _dptr(dx_dev), _dptr(dy_dev), int(nsolves), _stream(stream))


def ipm_graph_launch(ctx, stream=None) -> int:
    return _load().ipm_graph_launch(ctx, _stream(stream))


def ipm_launch_counts(ctx):
    a, b = ct.c_int32(), ct.c_int32()
    _load().ipm_launch_counts(ctx, ct.byref(a), ct.byref(b))
    return a.value, b.value


def ipm_test_recip_pivot(x_dev, rcp_dev, quo_dev, stream=None) -> int:
    return _load().ipm_test_recip_pivot(_dptr(x_dev), _dptr(rcp_dev), _dptr(quo_dev), int(x_dev.numel()),
                                        _stream(stream))


def ipm_get_pivots(ctx):
    """(lperm, Doff, bsize) of a factorisation in the pivoting mode."""
    N = ipm_get_sizes(ctx)[0]
    lp, do, bs = np.empty(N, np.int32), np.empty(N, np.float64), np.empty(N, np.int32)
    rc = _load().ipm_get_pivots(ctx, lp.ctypes.data, do.ctypes.data, bs.ctypes.data)
    if rc:
        raise RuntimeError(f"ipm_get_pivots failed ({rc})")
    return dict(lperm=lp, Doff=do, bsize=bs)


def ipm_measure_fp64_peak(device=0):
    """(dfma_tflops, dmma_tflops) measured on `device`."""
    a, b = ct.c_double(), ct.c_double()
    rc = _load().ipm_measure_fp64_peak(int(device), ct.byref(a), ct.byref(b))
    if rc:
        raise RuntimeError(f"ipm_measure_fp64_peak failed ({rc})")
    return a.value, b.value


def ipm_set_profiling(ctx, enable=True) -> int:
    return _load().ipm_set_profiling(ctx, 1 if enable else 0)


def ipm_kernel_stats(ctx, reset=False):
    """Per kernel class: dict(launches, ms, flops, bytes)."""
    arr = (ipm_kernel_stat * len(KERNEL_CLASSES))()
    rc = _load().ipm_kernel_stats(ctx, ct.cast(arr, ct.c_void_p), 1 if reset else 0)
    if rc:
        raise RuntimeError(f"ipm_kernel_stats failed ({rc})")
    return {name: dict(launches=a.launches, ms=a.ms, flops=a.flops, bytes=a.bytes)
            for name, a in zip(KERNEL_CLASSES, arr)}


def ipm_kernel_trace(ctx, cap=1 << 20):
    """Profiled launches since the last trace, in issue order: dict of numpy
    arrays cls, stream, start_ms, end_ms (times from the batch's first launch)."""
    cls = np.zeros(cap, np.int32)
    stream = np.zeros(cap, np.int32)
    t0 = np.zeros(cap, np.float64)
    t1 = np.zeros(cap, np.float64)
    n = ct.c_int32(0)
    rc = _load().ipm_kernel_trace(ctx, _hptr(cls, np.int32), _hptr(stream, np.int32), _hptr(t0, np.float64),
                                  _hptr(t1, np.float64), cap, ct.addressof(n))
    if rc:
        raise RuntimeError(f"ipm_kernel_trace failed ({rc})")
    k = min(cap, n.value)
    return dict(cls=cls[:k], stream=stream[:k], start_ms=t0[:k], end_ms=t1[:k], count=n.value)


def declared_symbols():
    """Function names declared in include/ipm_mf.h."""
    import re

    with open(INCLUDE) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:int|void)\s+\*?\s*(ipm_\w+)\s*\(", text, flags=re.M)))


from .solver import Solver  # noqa: E402,F401
from .batch import BatchSolver, lpt_partition, shard  # noqa: E402,F401
