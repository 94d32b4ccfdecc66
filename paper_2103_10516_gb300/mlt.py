"""Python binding of the C ABI in include/mlt.h (ctypes; argument marshalling only).

Every computation runs in libmlt.so.  Importing this module does not need a GPU,
but calling anything that touches the device does; there is no CPU fallback.
If the library has not been built, ``lib()`` raises instead of degrading.

Device memory and streams may come from PyTorch: any function taking an array
accepts a numpy array (host) or a torch tensor (host or CUDA); ``stream`` is a
cudaStream_t as an int (``torch.cuda.current_stream().cuda_stream``) or None.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmlt.so")

MLT_OK, MLT_EINVAL, MLT_ENOMEM, MLT_ECUDA, MLT_ERANGE, MLT_ETIMEOUT = 0, -1, -2, -3, -4, -5
MLT_F64, MLT_F32, MLT_PATTERN = 0, 1, 2
MLT_GRAM, MLT_DEVICE_PTRS, MLT_REORDER = 1, 2, 4
MLT_FN = {"log": 0, "sqrt": 1, "exp": 2, "inv": 3, "pow": 4, "cube": 5}
MLT_PREC = {"fp64": 0, "fp32": 1, "df64": 3}
MLT_DIRECT = 1
MLT_LOW_CV = 4
MLT_BOUNDS_GERSHGORIN, MLT_BOUNDS_LANCZOS = 0, 1
MLT_MAX_LEVELS = 1024
MLT_MAX_DEGREE = 4096
MLT_MODE = {"budget": 0, "variance": 1}
MLT_COST = {"symmetric": 0, "linear": 1}

EXPORTS = ["mlt_create_csr", "mlt_destroy", "mlt_matrix_info", "mlt_spectrum_bounds",
           "mlt_cheb_coeffs", "mlt_moments", "mlt_mlmc_default_params", "mlt_mlmc_estimate",
           "mlt_triangle_trace", "mlt_profile_start", "mlt_profile_stop", "mlt_last_error",
           "mlt_surrogate_create", "mlt_surrogate_destroy", "mlt_surrogate_set_params",
           "mlt_surrogate_get_params", "mlt_surrogate_loss_grad", "mlt_surrogate_train",
           "mlt_surrogate_predict", "mlt_learned_train", "mlt_learned_estimate",
           "mlt_moments_batched", "mlt_autotune", "mlt_moments_noalloc", "mlt_low_traces",
           "mlt_release_cached", "mlt_poly_apply", "mlt_hutchpp_estimate", "mlt_pilot_variances",
           "mlt_select_levels", "mlt_band_samples", "mlt_mlmc_combine", "mlt_triangle_estimate",
           "mlt_fp64_rate", "mlt_surrogate_get_norm", "mlt_batch_create", "mlt_batch_run",
           "mlt_batch_destroy"]
MLT_TRI_CV = {"none": 0, "fit": 1, "cheb": 2}


class MLTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (code %d)" % (msg, code))
        self.code = code


class mlt_mlmc_params(ctypes.Structure):
    _fields_ = [("fn", ctypes.c_int), ("fn_p", ctypes.c_double), ("a", ctypes.c_double),
                ("b", ctypes.c_double), ("n", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("nlevels", ctypes.c_int), ("levels", ctypes.c_int32 * MLT_MAX_LEVELS),
                ("m", ctypes.c_int64 * MLT_MAX_LEVELS), ("m_pilot", ctypes.c_int),
                ("mode", ctypes.c_int), ("target", ctypes.c_double), ("cost_model", ctypes.c_int),
                ("max_levels", ctypes.c_int), ("reuse_pilot", ctypes.c_int),
                ("precision", ctypes.c_int), ("flags", ctypes.c_uint), ("stream", ctypes.c_void_p)]


class mlt_hutchpp_result(ctypes.Structure):
    _fields_ = [("estimate", ctypes.c_double), ("std_error", ctypes.c_double),
                ("t_sketch", ctypes.c_double), ("t_rest", ctypes.c_double),
                ("rank", ctypes.c_int), ("matvecs", ctypes.c_int64)]


class mlt_mlmc_result(ctypes.Structure):
    _fields_ = [("estimate", ctypes.c_double), ("std_error", ctypes.c_double),
                ("nlevels", ctypes.c_int), ("levels", ctypes.c_int32 * MLT_MAX_LEVELS),
                ("m", ctypes.c_int64 * MLT_MAX_LEVELS),
                ("level_mean", ctypes.c_double * MLT_MAX_LEVELS),
                ("level_var", ctypes.c_double * MLT_MAX_LEVELS),
                ("probes", ctypes.c_int64), ("matvecs", ctypes.c_int64)]


class mlt_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


_lib = None


def lib():
    """The loaded libmlt.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libmlt.so is not built (%s); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, u64, dbl, ci, cu = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                      ctypes.c_uint64, ctypes.c_double, ctypes.c_int, ctypes.c_uint)
    L.mlt_create_csr.argtypes = [i64, i64, i64, vp, vp, vp, ci, dbl, cu, vp, ctypes.POINTER(vp)]
    L.mlt_destroy.argtypes = [vp]
    L.mlt_release_cached.argtypes = []
    L.mlt_matrix_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.mlt_spectrum_bounds.argtypes = [vp, ci, ci, u64, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
    L.mlt_cheb_coeffs.argtypes = [ci, dbl, dbl, dbl, ci, vp]
    L.mlt_moments.argtypes = [vp, dbl, dbl, u64, i64, i64, vp, ci, cu, vp, i64, vp]
    L.mlt_mlmc_default_params.argtypes = [ctypes.POINTER(mlt_mlmc_params)]
    L.mlt_mlmc_default_params.restype = None
    L.mlt_mlmc_estimate.argtypes = [vp, ctypes.POINTER(mlt_mlmc_params), ctypes.POINTER(mlt_mlmc_result)]
    L.mlt_triangle_trace.argtypes = [vp, u64, i64, i64, ci, ci, vp, ctypes.POINTER(dbl),
                                     ctypes.POINTER(dbl), vp]
    L.mlt_low_traces.argtypes = [vp, dbl, dbl, vp, ctypes.POINTER(ci), vp]
    L.mlt_poly_apply.argtypes = [vp, dbl, dbl, vp, ci, vp, i64, vp, i64, ci, cu, vp]
    L.mlt_hutchpp_estimate.argtypes = [vp, dbl, dbl, vp, ci, u64, i64, ci, ci, ci, vp,
                                       ctypes.POINTER(mlt_hutchpp_result), vp]
    L.mlt_pilot_variances.argtypes = [vp, ci, vp, i64, i64, vp]
    L.mlt_select_levels.argtypes = [vp, ci, ci, ci, ci, dbl, ci, vp, vp, ctypes.POINTER(ci)]
    L.mlt_band_samples.argtypes = [vp, ci, ci, vp, i64, i64, vp]
    L.mlt_mlmc_combine.argtypes = [ci, vp, vp, vp, ctypes.POINTER(mlt_mlmc_result)]
    L.mlt_triangle_estimate.argtypes = [vp, i64, i64, ci, dbl, dbl, ctypes.POINTER(dbl), ctypes.POINTER(dbl),
                                        ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
    L.mlt_fp64_rate.argtypes = [i64, ctypes.POINTER(dbl), vp]
    L.mlt_profile_start.argtypes = []
    L.mlt_profile_stop.argtypes = [ctypes.POINTER(mlt_kernel_stat), ci, ctypes.POINTER(ci)]
    L.mlt_last_error.argtypes = []
    L.mlt_last_error.restype = ctypes.c_char_p
    _bind_learned(L)
    _bind_batch(L)
    _bind_noalloc(L)
    for name in EXPORTS:
        if name not in ("mlt_mlmc_default_params", "mlt_last_error"):
            getattr(L, name).restype = ci
    _lib = L
    return L


def _check(rc):
    if rc != MLT_OK:
        raise MLTError(rc, lib().mlt_last_error().decode(errors="replace"))


def _ptr(a):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError("expected a numpy array or torch tensor")


def _is_cuda(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def _stream(stream):
    return None if stream is None else int(stream)


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def mlt_create_csr(nrows, ncols, nnz, rowptr, col, vals=None, val_type=None, scale=1.0,
                   flags=0, stream=None):
    """Returns an opaque handle (int).  rowptr int64, col int32, vals float64/float32."""
    if val_type is None:
        if vals is None:
            val_type = MLT_PATTERN
        else:
            dt = str(vals.dtype)
            val_type = MLT_F32 if dt.endswith("float32") else MLT_F64
    if _is_cuda(rowptr):
        flags |= MLT_DEVICE_PTRS
    h = ctypes.c_void_p()
    _check(lib().mlt_create_csr(nrows, ncols, nnz, _ptr(rowptr), _ptr(col), _ptr(vals), val_type,
                                float(scale), flags, _stream(stream), ctypes.byref(h)))
    return h.value


def mlt_destroy(handle):
    if handle:
        _check(lib().mlt_destroy(handle))


def mlt_release_cached():
    """Return the device memory cached by destroyed handles to the driver."""
    _check(lib().mlt_release_cached())


def mlt_matrix_info(handle):
    d, nnz = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().mlt_matrix_info(handle, ctypes.byref(d), ctypes.byref(nnz)))
    return d.value, nnz.value


def mlt_spectrum_bounds(handle, method=MLT_BOUNDS_GERSHGORIN, steps=0, seed=0):
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().mlt_spectrum_bounds(handle, method, steps, seed, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def mlt_poly_apply(handle, a, b, c, X, Y=None, stream=None):
    """Y = p(At) X for the columns of X (d x ncols; numpy on the host, or a CUDA
    tensor), p = sum_k c[k] T_k.  Returns Y (a new array unless given)."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    dev = _is_cuda(X)
    if Y is None:
        Y = X.new_empty(X.shape) if dev else np.empty(X.shape, dtype=np.float64)
    ncols = X.shape[1]
    _check(lib().mlt_poly_apply(handle, float(a), float(b), _ptr(c), len(c) - 1, _ptr(X), ncols, _ptr(Y), ncols,
                                ncols, MLT_DEVICE_PTRS if dev else 0, _stream(stream)))
    return Y


def mlt_hutchpp_estimate(handle, a, b, c, seed, probe_offset, s, g, precision="fp64", samples=None, stream=None):
    """Hutch++ on tr p(At) (precision "fp32": the sketch in FP32); returns the
    mlt_hutchpp_result (and fills `samples`, a float64 array of g entries)."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    r = mlt_hutchpp_result()
    prec = MLT_PREC[precision] if isinstance(precision, str) else precision
    _check(lib().mlt_hutchpp_estimate(handle, float(a), float(b), _ptr(c), len(c) - 1, seed, probe_offset, s, g,
                                      prec, _ptr(samples), ctypes.byref(r), _stream(stream)))
    return r


def mlt_low_traces(handle, a, b, stream=None):
    """[tr T_0, tr T_1, tr T_2] of the mapped operator (two values for X^T X)."""
    t = np.zeros(3)
    k = ctypes.c_int()
    _check(lib().mlt_low_traces(handle, float(a), float(b), _ptr(t), ctypes.byref(k), _stream(stream)))
    return t[: k.value]


def mlt_cheb_coeffs(fn, a, b, n, p=0.0):
    c = np.zeros(n + 1)
    _check(lib().mlt_cheb_coeffs(MLT_FN[fn] if isinstance(fn, str) else fn, float(p), float(a),
                                 float(b), int(n), _ptr(c)))
    return c


def mlt_moments(handle, a, b, seed, probe_offset, degrees, precision="fp64", flags=0, out=None,
                stream=None):
    """mu[p, j] for j <= degrees[p]; `out` (nprobes x ld, float64, host or CUDA) is
    filled in place, else a new numpy array is returned."""
    deg = np.ascontiguousarray(degrees, dtype=np.int32)
    if out is None:
        ld = int(deg.max()) + 1 if deg.size else 1
        out = np.zeros((deg.size, ld))
    ld = out.shape[1]
    prec = MLT_PREC[precision] if isinstance(precision, str) else precision
    _check(lib().mlt_moments(handle, float(a), float(b), int(seed), int(probe_offset), deg.size,
                             _ptr(deg), prec, int(flags), _ptr(out), ld, _stream(stream)))
    return out


def mlt_mlmc_default_params():
    p = mlt_mlmc_params()
    lib().mlt_mlmc_default_params(ctypes.byref(p))
    return p


def mlt_mlmc_estimate(handle, params):
    r = mlt_mlmc_result()
    _check(lib().mlt_mlmc_estimate(handle, ctypes.byref(params), ctypes.byref(r)))
    return _result_dict(r)


def _result_dict(r):
    L = r.nlevels
    return {"estimate": r.estimate, "stderr": r.std_error, "levels": list(r.levels[:L]),
            "m": list(r.m[:L]), "level_mean": list(r.level_mean[:L]),
            "level_var": list(r.level_var[:L]), "probes": r.probes, "matvecs": r.matvecs}


def mlt_pilot_variances(c, mu):
    """(n+1) x (n+1) table V[lo, hi] of the pilot rows mu (m x ld, host), n = len(c) - 1."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    mu = np.ascontiguousarray(np.atleast_2d(mu), dtype=np.float64)
    n = c.size - 1
    V = np.zeros((n + 1, n + 1))
    _check(lib().mlt_pilot_variances(_ptr(c), n, _ptr(mu), mu.shape[1], mu.shape[0], _ptr(V)))
    return V


def mlt_select_levels(V, cost_model="symmetric", m_pilot=0, mode="budget", target=1.0, max_levels=0):
    """(levels, m) from the variance table V ((n+1) x (n+1), host)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    n = V.shape[0] - 1
    lv = np.zeros(n + 1, dtype=np.int32)
    m = np.zeros(n + 1, dtype=np.int64)
    L = ctypes.c_int()
    _check(lib().mlt_select_levels(_ptr(V), n, MLT_COST[cost_model] if isinstance(cost_model, str) else cost_model,
                                   int(m_pilot), MLT_MODE[mode] if isinstance(mode, str) else mode, float(target),
                                   int(max_levels), _ptr(lv), _ptr(m), ctypes.byref(L)))
    return [int(v) for v in lv[:L.value]], [int(v) for v in m[:L.value]]


def mlt_band_samples(c, lo, hi, mu):
    """Q_{lo,hi} of every row of mu (host)."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    mu = np.ascontiguousarray(np.atleast_2d(mu), dtype=np.float64)
    q = np.zeros(mu.shape[0])
    _check(lib().mlt_band_samples(_ptr(c), int(lo), int(hi), _ptr(mu), mu.shape[1], mu.shape[0], _ptr(q)))
    return q


def mlt_mlmc_combine(levels, m, samples):
    """Eq. multiEstimator from per-level samples concatenated level by level."""
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    mm = np.ascontiguousarray(m, dtype=np.int64)
    smp = np.ascontiguousarray(samples, dtype=np.float64)
    if smp.size != int(mm.sum()):
        raise ValueError("mlt_mlmc_combine: %d samples for %d expected" % (smp.size, int(mm.sum())))
    r = mlt_mlmc_result()
    _check(lib().mlt_mlmc_combine(lv.size, _ptr(lv), _ptr(mm), _ptr(smp), ctypes.byref(r)))
    return _result_dict(r)


def mlt_triangle_estimate(x, nnz, cv="fit", a=0.0, b=0.0):
    """(estimate, stderr, a1, a2) from per-probe triangle moments x (nprobes x 3, host int64)."""
    x = np.ascontiguousarray(x, dtype=np.int64)
    est, se, a1, a2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().mlt_triangle_estimate(_ptr(x), x.shape[0], int(nnz), MLT_TRI_CV[cv] if isinstance(cv, str) else cv,
                                       float(a), float(b), ctypes.byref(est), ctypes.byref(se), ctypes.byref(a1),
                                       ctypes.byref(a2)))
    return est.value, se.value, a1.value, a2.value


def mlt_triangle_trace(handle, seed, probe_offset, nprobes, block=256, use_cv=True, x=None,
                       stream=None):
    """Returns (estimate, stderr); per-probe (x1, x2, x3) go to `x` if given."""
    est, se = ctypes.c_double(), ctypes.c_double()
    _check(lib().mlt_triangle_trace(handle, int(seed), int(probe_offset), int(nprobes), int(block),
                                    int(bool(use_cv)), _ptr(x), ctypes.byref(est), ctypes.byref(se),
                                    _stream(stream)))
    return est.value, se.value


def mlt_fp64_rate(iters=1 << 16, stream=None):
    """Measured FP64 FMA rate of the current device (TFLOP/s)."""
    t = ctypes.c_double()
    _check(lib().mlt_fp64_rate(int(iters), ctypes.byref(t), _stream(stream)))
    return t.value


def mlt_profile_start():
    _check(lib().mlt_profile_start())


def mlt_profile_stop(max_stats=64):
    """{kernel name: (launches, total ms)} of the launches since mlt_profile_start()."""
    arr = (mlt_kernel_stat * max_stats)()
    n = ctypes.c_int()
    _check(lib().mlt_profile_stop(arr, max_stats, ctypes.byref(n)))
    return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(n.value)}


def mlt_last_error():
    return lib().mlt_last_error().decode(errors="replace")


# ---------------------------------------------------------------------------
# convenience: a handle bound to a CSR (arrays from paper_2103_10516_gb300.synth)
# ---------------------------------------------------------------------------

class Matrix:
    """Owns one mlt_matrix handle built from host CSR arrays (or CUDA tensors)."""

    def __init__(self, csr, gram=False, scale=1.0, vals_dtype=None, stream=None, reorder=False):
        vals = csr.val
        if vals is not None and vals_dtype is not None:
            vals = np.ascontiguousarray(vals, dtype=vals_dtype)
        self._keep = (csr.rowptr, csr.col, vals)
        flags = (MLT_GRAM if gram else 0) | (MLT_REORDER if reorder else 0)
        self.handle = mlt_create_csr(csr.nrows, csr.ncols, csr.nnz, csr.rowptr, csr.col, vals,
                                     scale=scale, flags=flags, stream=stream)
        self.dim, self.nnz = mlt_matrix_info(self.handle)

    def close(self):
        if self.handle:
            mlt_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def moments(self, a, b, seed, probe_offset, degrees, **kw):
        return mlt_moments(self.handle, a, b, seed, probe_offset, degrees, **kw)

    def bounds(self):
        return mlt_spectrum_bounds(self.handle)

    def triangles(self, seed, probe_offset, nprobes, use_cv=True, x=None, stream=None):
        return mlt_triangle_trace(self.handle, seed, probe_offset, nprobes, 256, use_cv, x, stream)

    def mlmc(self, fn, a, b, n, seed=0, levels=None, m=None, m_pilot=10, mode="budget",
             target=1000.0, cost_model="symmetric", max_levels=0, reuse_pilot=True,
             precision="fp64", direct=False, p=0.0, low_cv=False, stream=None):
        P = mlt_mlmc_default_params()
        P.fn = MLT_FN[fn] if isinstance(fn, str) else fn
        P.fn_p = p
        P.a, P.b, P.n, P.seed = float(a), float(b), int(n), int(seed)
        if levels is not None:
            P.nlevels = len(levels)
            for k, (l, mk) in enumerate(zip(levels, m)):
                P.levels[k] = int(l)
                P.m[k] = int(mk)
        else:
            P.nlevels = 0
        P.m_pilot = int(m_pilot)
        P.mode = MLT_MODE[mode]
        P.target = float(target)
        P.cost_model = MLT_COST[cost_model]
        P.max_levels = int(max_levels)
        P.reuse_pilot = int(bool(reuse_pilot))
        P.precision = MLT_PREC[precision]
        P.flags = (MLT_DIRECT if direct else 0) | (MLT_LOW_CV if low_cv else 0)
        P.stream = _stream(stream)
        return mlt_mlmc_estimate(self.handle, P)


# ---------------------------------------------------------------------------
# learned coarse level
# ---------------------------------------------------------------------------

MLT_NET_IN, MLT_NET_HID, MLT_NET_NPARAMS = 16, 128, 18817
NET_OFF = {"W1": (0, (128, 16)), "b1": (2048, (128,)), "W2": (2176, (128, 128)),
           "b2": (18560, (128,)), "w3": (18688, (128,)), "b3": (18816, ())}


class mlt_learned_params(ctypes.Structure):
    _fields_ = [("fn", ctypes.c_int), ("fn_p", ctypes.c_double), ("a", ctypes.c_double),
                ("b", ctypes.c_double), ("n", ctypes.c_int), ("l1", ctypes.c_int),
                ("m_net", ctypes.c_int64), ("m_1", ctypes.c_int64), ("m_2", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("probe_offset", ctypes.c_int64),
                ("precision", ctypes.c_int), ("stream", ctypes.c_void_p)]


def _bind_learned(L):
    vp, i64, u64, dbl, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
    L.mlt_surrogate_create.argtypes = [u64, ctypes.POINTER(vp)]
    L.mlt_surrogate_destroy.argtypes = [vp]
    L.mlt_surrogate_set_params.argtypes = [vp, vp]
    L.mlt_surrogate_get_params.argtypes = [vp, vp]
    L.mlt_surrogate_loss_grad.argtypes = [vp, vp, vp, i64, ctypes.POINTER(dbl), vp, vp]
    L.mlt_surrogate_train.argtypes = [vp, vp, vp, i64, ci, i64, dbl, ctypes.POINTER(dbl), vp]
    L.mlt_surrogate_predict.argtypes = [vp, vp, i64, vp, vp]
    L.mlt_surrogate_get_norm.argtypes = [vp, vp, ctypes.POINTER(ci)]
    L.mlt_learned_train.argtypes = [vp, vp, ctypes.POINTER(mlt_learned_params), i64, i64, ci, i64, dbl,
                                    ctypes.POINTER(dbl)]
    L.mlt_learned_estimate.argtypes = [vp, vp, ctypes.POINTER(mlt_learned_params),
                                       ctypes.POINTER(mlt_mlmc_result)]


def pack_params(P):
    """Dict of arrays (W1, b1, W2, b2, w3, b3) -> FP32 vector of MLT_NET_NPARAMS."""
    v = np.zeros(MLT_NET_NPARAMS, dtype=np.float32)
    for k, (off, shape) in NET_OFF.items():
        a = np.asarray(P[k], dtype=np.float32).ravel()
        v[off: off + a.size] = a
    return v


def unpack_params(v):
    out = {}
    for k, (off, shape) in NET_OFF.items():
        size = int(np.prod(shape)) if shape else 1
        a = np.asarray(v[off: off + size], dtype=np.float64)
        out[k] = a.reshape(shape) if shape else float(a[0])
    return out


class Surrogate:
    """Owns one mlt_surrogate handle."""

    def __init__(self, seed=0):
        h = ctypes.c_void_p()
        _check(lib().mlt_surrogate_create(int(seed), ctypes.byref(h)))
        self.handle = h.value

    def close(self):
        if self.handle:
            _check(lib().mlt_surrogate_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, P):
        v = pack_params(P) if isinstance(P, dict) else np.ascontiguousarray(P, dtype=np.float32)
        _check(lib().mlt_surrogate_set_params(self.handle, _ptr(v)))

    def get_params(self):
        v = np.zeros(MLT_NET_NPARAMS, dtype=np.float32)
        _check(lib().mlt_surrogate_get_params(self.handle, _ptr(v)))
        return v

    def loss_grad(self, X, T, stream=None):
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        g = np.zeros(MLT_NET_NPARAMS, dtype=np.float32)
        loss = ctypes.c_double()
        _check(lib().mlt_surrogate_loss_grad(self.handle, _ptr(X), _ptr(T), X.shape[0],
                                             ctypes.byref(loss), _ptr(g), _stream(stream)))
        return loss.value, g

    def train(self, X, T, epochs, batch, lr, stream=None):
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        loss = ctypes.c_double()
        _check(lib().mlt_surrogate_train(self.handle, _ptr(X), _ptr(T), X.shape[0], int(epochs),
                                         int(batch), float(lr), ctypes.byref(loss), _stream(stream)))
        return loss.value

    def get_norm(self):
        """(feature means (16), feature stds (16), target mean, target std), or
        None before training set them."""
        v = np.zeros(2 * MLT_NET_IN + 2)
        h = ctypes.c_int()
        _check(lib().mlt_surrogate_get_norm(self.handle, _ptr(v), ctypes.byref(h)))
        if not h.value:
            return None
        return v[:MLT_NET_IN], v[MLT_NET_IN:2 * MLT_NET_IN], float(v[2 * MLT_NET_IN]), float(v[2 * MLT_NET_IN + 1])

    def predict(self, X, stream=None):
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.zeros(X.shape[0], dtype=np.float32)
        _check(lib().mlt_surrogate_predict(self.handle, _ptr(X), X.shape[0], _ptr(y), _stream(stream)))
        return y


def learned_params(fn, a, b, n, l1, m_net, m_1, m_2, seed=0, probe_offset=0, precision="fp64",
                   p=0.0, stream=None):
    P = mlt_learned_params()
    P.fn = MLT_FN[fn] if isinstance(fn, str) else fn
    P.fn_p, P.a, P.b, P.n, P.l1 = float(p), float(a), float(b), int(n), int(l1)
    P.m_net, P.m_1, P.m_2 = int(m_net), int(m_1), int(m_2)
    P.seed, P.probe_offset = int(seed), int(probe_offset)
    P.precision = MLT_PREC[precision] if isinstance(precision, str) else precision
    P.stream = _stream(stream)
    return P


def mlt_learned_train(matrix, surrogate, P, n_train, train_offset, epochs, batch, lr):
    loss = ctypes.c_double()
    _check(lib().mlt_learned_train(matrix, surrogate, ctypes.byref(P), int(n_train), int(train_offset),
                                   int(epochs), int(batch), float(lr), ctypes.byref(loss)))
    return loss.value


def mlt_learned_estimate(matrix, surrogate, P):
    r = mlt_mlmc_result()
    _check(lib().mlt_learned_estimate(matrix, surrogate, ctypes.byref(P), ctypes.byref(r)))
    L = r.nlevels
    return {"estimate": r.estimate, "stderr": r.std_error, "levels": list(r.levels[:L]),
            "m": list(r.m[:L]), "level_mean": list(r.level_mean[:L]),
            "level_var": list(r.level_var[:L]), "probes": r.probes, "matvecs": r.matvecs}


def mixed_at(k):
    """Precision code: the first k recurrence steps in FP32, the rest in FP64."""
    return 2 | (int(k) << 8)


# ---------------------------------------------------------------------------
# batched moments and the autotuner
# ---------------------------------------------------------------------------

class mlt_moments_job(ctypes.Structure):
    _fields_ = [("matrix", ctypes.c_void_p), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("probe_offset", ctypes.c_int64),
                ("nprobes", ctypes.c_int64), ("degree", ctypes.c_void_p), ("mu", ctypes.c_void_p),
                ("ld_mu", ctypes.c_int64), ("group_width", ctypes.c_int)]


def _bind_batch(L):
    L.mlt_moments_batched.argtypes = [ctypes.POINTER(mlt_moments_job), ctypes.c_int, ctypes.c_int,
                                      ctypes.c_uint, ctypes.c_void_p]
    L.mlt_autotune.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                               ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]
    L.mlt_batch_create.argtypes = [ctypes.POINTER(mlt_moments_job), ctypes.c_int, ctypes.c_int, ctypes.c_uint,
                                   ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    L.mlt_batch_run.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    L.mlt_batch_destroy.argtypes = [ctypes.c_void_p]


def _job_array(jobs):
    arr = (mlt_moments_job * len(jobs))()
    keep = []
    for i, j in enumerate(jobs):
        deg = np.ascontiguousarray(j["degrees"], dtype=np.int32)
        keep.append(deg)
        out = j["out"]
        arr[i].matrix = j["matrix"]
        arr[i].a, arr[i].b = float(j["a"]), float(j["b"])
        arr[i].seed, arr[i].probe_offset = int(j.get("seed", 0)), int(j.get("probe_offset", 0))
        arr[i].nprobes = deg.size
        arr[i].degree = _ptr(deg)
        arr[i].mu = _ptr(out)
        arr[i].ld_mu = out.shape[1]
        arr[i].group_width = int(j.get("group_width", 0))
    return arr, keep


class Batch:
    """A persistent batch (mlt_batch_create): the jobs' CUDA graph is built
    once; run(shift) replays it with probe ids shifted by `shift`.  The jobs'
    output arrays must outlive the batch."""

    def __init__(self, jobs, precision="fp64", flags=0, stream=None):
        arr, keep = _job_array(jobs)
        self._keep = (keep, [j["out"] for j in jobs])
        h = ctypes.c_void_p()
        prec = MLT_PREC[precision] if isinstance(precision, str) else precision
        _check(lib().mlt_batch_create(arr, len(jobs), prec, int(flags), _stream(stream), ctypes.byref(h)))
        self.handle = h.value

    def run(self, shift=0, stream=None):
        _check(lib().mlt_batch_run(self.handle, int(shift), _stream(stream)))

    def close(self):
        if self.handle:
            lib().mlt_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mlt_moments_batched(jobs, precision="fp64", flags=0, stream=None):
    """jobs: list of dicts with matrix (handle), a, b, seed, probe_offset, degrees,
    out (numpy or CUDA tensor nprobes x ld) and optionally group_width."""
    arr = (mlt_moments_job * len(jobs))()
    keep = []
    for i, j in enumerate(jobs):
        deg = np.ascontiguousarray(j["degrees"], dtype=np.int32)
        keep.append(deg)
        out = j["out"]
        arr[i].matrix = j["matrix"]
        arr[i].a, arr[i].b = float(j["a"]), float(j["b"])
        arr[i].seed, arr[i].probe_offset = int(j.get("seed", 0)), int(j.get("probe_offset", 0))
        arr[i].nprobes = deg.size
        arr[i].degree = _ptr(deg)
        arr[i].mu = _ptr(out)
        arr[i].ld_mu = out.shape[1]
        arr[i].group_width = int(j.get("group_width", 0))
    prec = MLT_PREC[precision] if isinstance(precision, str) else precision
    _check(lib().mlt_moments_batched(arr, len(jobs), prec, int(flags), _stream(stream)))


def mlt_autotune(handle, precision="fp64", trial_steps=8, stream=None):
    best = ctypes.c_int()
    prec = MLT_PREC[precision] if isinstance(precision, str) else precision
    _check(lib().mlt_autotune(handle, prec, int(trial_steps), ctypes.byref(best), _stream(stream)))
    return best.value


# ---------------------------------------------------------------------------
# moments without device allocation (fixed 32 MiB array inside the library)
# ---------------------------------------------------------------------------

def _bind_noalloc(L):
    vp, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    L.mlt_moments_noalloc.argtypes = [i64, i64, vp, vp, vp, dbl, dbl, dbl, ctypes.c_uint64, i64,
                                      ctypes.c_int, vp, vp, i64, vp]


def _noalloc_arg(name, t, dtype, min_len=None, exact_len=None):
    """Check one tensor argument of mlt_moments_noalloc: the C side receives raw
    device pointers and cannot see a wrong dtype, a short array or host memory."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError("mlt_moments_noalloc: %s must be a torch tensor" % name)
    if t.dtype != dtype:
        raise ValueError("mlt_moments_noalloc: %s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("mlt_moments_noalloc: %s must be contiguous" % name)
    if exact_len is not None and t.numel() != exact_len:
        raise ValueError("mlt_moments_noalloc: %s needs %d entries, has %d" % (name, exact_len, t.numel()))
    if min_len is not None and t.numel() < min_len:
        raise ValueError("mlt_moments_noalloc: %s needs at least %d entries, has %d" % (name, min_len, t.numel()))


def mlt_moments_noalloc(d, nnz, rowptr, col, vals, scale, a, b, seed, probe_offset, degrees, mu,
                        stream=None):
    """All array arguments but `degrees` are CUDA tensors the caller owns; mu is
    nprobes x ld and is written in place.  Raises ValueError, before anything
    reaches the library, when a tensor has the wrong dtype, is too short, is not
    contiguous or is not in CUDA memory."""
    import torch
    deg = np.ascontiguousarray(degrees, dtype=np.int32)
    d, nnz = int(d), int(nnz)
    if d < 1 or nnz < 0:
        raise ValueError("mlt_moments_noalloc: need d >= 1 and nnz >= 0")
    _noalloc_arg("rowptr", rowptr, torch.int64, exact_len=d + 1)
    _noalloc_arg("col", col, torch.int32, min_len=nnz)
    if vals is not None:
        _noalloc_arg("vals", vals, torch.float64, min_len=nnz)
    _noalloc_arg("mu", mu, torch.float64)
    if mu.dim() != 2 or mu.shape[0] < deg.size:
        raise ValueError("mlt_moments_noalloc: mu must be 2-D with at least %d rows" % deg.size)
    if deg.size and mu.shape[1] < int(deg.max()) + 1:
        raise ValueError("mlt_moments_noalloc: mu needs at least max degree + 1 = %d columns" % (int(deg.max()) + 1))
    for name, t in (("rowptr", rowptr), ("col", col), ("vals", vals), ("mu", mu)):
        if t is not None and not t.is_cuda:
            raise ValueError("mlt_moments_noalloc: %s must be in CUDA memory" % name)
    _check(lib().mlt_moments_noalloc(d, nnz, _ptr(rowptr), _ptr(col), _ptr(vals), float(scale),
                                     float(a), float(b), int(seed), int(probe_offset), deg.size, _ptr(deg),
                                     _ptr(mu), mu.shape[1], _stream(stream)))
    return mu
