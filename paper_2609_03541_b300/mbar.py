"""ctypes binding of ``libbumbar.so`` (argument marshalling only).

Every computation happens inside the library's CUDA kernels. The names
follow the C ABI in ``include/bumbar.h``: ``Context`` wraps an ``mbar_ctx``
and its methods call ``mbar_create / mbar_set_coordinate / mbar_bin /
mbar_bin_count / mbar_get_bins / mbar_sci_step / mbar_hessian /
mbar_newton_step / mbar_solve / mbar_free_energies / mbar_destroy``;
``lse_pass`` calls the stateless ``mbar_lse_pass``.

Loading fails loudly (``LibraryMissing``) when the library has not been
built; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbumbar.so")

MBAR_FP64 = 0
MBAR_MIXED = 1

STATUS = {
    0: "MBAR_OK", 1: "MBAR_EINVAL", 2: "MBAR_ENOMEM", 3: "MBAR_ECUDA", 4: "MBAR_ENOTCONV",
    5: "MBAR_ESTATE", 6: "MBAR_ETIMEOUT", 7: "MBAR_EUNSUPPORTED",
}


class LibraryMissing(RuntimeError):
    pass


class MbarError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class Opts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("n0", ctypes.c_int32),
        ("eps", ctypes.c_double),
        ("inc", ctypes.c_int32),
        ("n_intermediate", ctypes.c_int32),
        ("h0", ctypes.c_double),
        ("use_binning", ctypes.c_int32),
        ("f_tol", ctypes.c_double),
        ("warm_tol", ctypes.c_double),
        ("max_newton", ctypes.c_int32),
        ("max_sci", ctypes.c_int32),
        ("noise_floor", ctypes.c_double),
    ]


class Report(ctypes.Structure):
    _fields_ = [
        ("iters_first_loop", ctypes.c_int64),
        ("iters_second_loop", ctypes.c_int64),
        ("iters_newton", ctypes.c_int64),
        ("newton_fallbacks", ctypes.c_int64),
        ("n_rebins", ctypes.c_int64),
        ("final_bins", ctypes.c_int64),
        ("max_abs_grad", ctypes.c_double),
        ("last_step", ctypes.c_double),
        ("seconds_width", ctypes.c_double),
        ("seconds_levels", ctypes.c_double),
        ("seconds_sci", ctypes.c_double),
        ("seconds_newton", ctypes.c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class TuneResult(ctypes.Structure):
    _fields_ = [
        ("family", ctypes.c_int32),
        ("lanes_per_sample", ctypes.c_int32),
        ("chunks_per_lane", ctypes.c_int32),
        ("threads", ctypes.c_int32),
        ("stage_bytes", ctypes.c_int32),
        ("candidates", ctypes.c_int32),
        ("ms", ctypes.c_double),
        ("heuristic_ms", ctypes.c_double),
        ("cached", ctypes.c_int32),
        ("pad", ctypes.c_int32),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "pad"}


TUNE_SAMPLES, TUNE_FACTORISED = 0, 1


BATCH_PERSISTENT = 1


class ServerConfig(ctypes.Structure):
    _fields_ = [
        ("workers", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("hbm_budget_bytes", ctypes.c_uint64),
        ("opts", Opts),
    ]


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p

_SIGNATURES = {
    "mbar_opts_default": ([ctypes.POINTER(Opts), ctypes.c_int32], ctypes.c_int),
    "mbar_create": ([ctypes.POINTER(_vp), ctypes.c_int64, ctypes.c_int64, _i64p, _vp, ctypes.c_int32,
                     ctypes.POINTER(Opts), _vp], ctypes.c_int),
    "mbar_set_coordinate": ([_vp, _vp, ctypes.c_int32], ctypes.c_int),
    "mbar_bin": ([_vp, ctypes.c_double, _i64p], ctypes.c_int),
    "mbar_bin_count": ([_vp, ctypes.c_int64, _dp, _i64p], ctypes.c_int),
    "mbar_get_bins": ([_vp, _i64p, _i64p, _dp], ctypes.c_int),
    "mbar_sci_step": ([_vp, _dp, _dp, _dp, _dp, _dp], ctypes.c_int),
    "mbar_hessian": ([_vp, _dp, _dp], ctypes.c_int),
    "mbar_covariance": ([_vp, _dp], ctypes.c_int),
    "mbar_newton_step": ([_vp, _dp, _dp, _dp], ctypes.c_int),
    "mbar_solve": ([_vp, _dp, ctypes.POINTER(Report)], ctypes.c_int),
    "mbar_free_energies": ([_vp, _dp], ctypes.c_int),
    "mbar_destroy": ([_vp], ctypes.c_int),
    "mbar_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "mbar_last_error": ([], ctypes.c_char_p),
    "mbar_device_bytes": ([_vp, _i64p], ctypes.c_int),
    "mbar_set_timing": ([_vp, ctypes.c_int32], ctypes.c_int),
    "mbar_set_exclusive": ([_vp, ctypes.c_int32], ctypes.c_int),
    "mbar_get_timing": ([_vp, ctypes.c_int32, _i64p, _dp, _dp], ctypes.c_int),
    "mbar_kernel_launches": ([_i64p], ctypes.c_int),
    "mbar_get_trace": ([_vp, _i64p, _dp, ctypes.c_int64], ctypes.c_int),
    "mbar_set_hessian_path": ([ctypes.c_int32], ctypes.c_int),
    "mbar_reweight": ([_vp, _vp, ctypes.c_int32, _dp, _dp], ctypes.c_int),
    "mbar_weighted_histogram2d": ([_vp, _vp, _vp, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_int64, _dp], ctypes.c_int),
    "mbar_selftest_wait_timeout": ([ctypes.c_int64, _dp], ctypes.c_int),
    "mbar_footprint_bytes": ([ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32], ctypes.c_uint64),
    "mbar_footprint_factorised_bytes": ([ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32],
                                        ctypes.c_uint64),
    "mbar_server_submit_factorised": ([_vp, ctypes.c_int64, ctypes.c_int64, _i64p, _vp, _vp, _vp, ctypes.c_int32,
                                       _i64p], ctypes.c_int),
    "mbar_autotune_lse": ([ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(TuneResult)], ctypes.c_int),
    "mbar_autotune_enable": ([ctypes.c_int32], ctypes.c_int),
    "mbar_autotune_cache": ([ctypes.c_char_p], ctypes.c_int),
    "mbar_autotune_clear": ([], ctypes.c_int),
    "mbar_server_create": ([ctypes.POINTER(_vp), ctypes.POINTER(ServerConfig)], ctypes.c_int),
    "mbar_server_submit": ([_vp, ctypes.c_int64, ctypes.c_int64, _i64p, _vp, ctypes.c_int32, _vp, ctypes.c_int32,
                            _i64p], ctypes.c_int),
    "mbar_server_poll": ([_vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "mbar_server_wait": ([_vp, ctypes.c_int64, _dp, ctypes.POINTER(Report), _dp, _dp], ctypes.c_int),
    "mbar_server_stats": ([_vp, _i64p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint64)],
                          ctypes.c_int),
    "mbar_server_destroy": ([_vp], ctypes.c_int),
    "mbar_batch_solve": ([ctypes.c_int32, _i64p, _i64p, ctypes.POINTER(_i64p), ctypes.POINTER(_vp), ctypes.c_int32,
                          ctypes.POINTER(_vp), ctypes.c_int32, ctypes.POINTER(ServerConfig), ctypes.POINTER(_dp),
                          ctypes.POINTER(Report), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "mbar_lse_static_scratch_bytes": ([], ctypes.c_size_t),
    "mbar_lse_pass_static": ([_vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _vp, _vp, _vp,
                              _vp, _vp, _vp], ctypes.c_int),
    "mbar_lse_scratch_bytes": ([ctypes.c_int64, ctypes.c_int64, ctypes.c_int32], ctypes.c_size_t),
    "mbar_lse_pass": ([_vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _vp, _vp, _vp, _vp,
                       _vp, _vp, ctypes.c_size_t, _vp], ctypes.c_int),
    "mbar_lse_samples_scratch_bytes": ([ctypes.c_int64, ctypes.c_int64], ctypes.c_size_t),
    "mbar_lse_factorised_scratch_bytes": ([ctypes.c_int64, ctypes.c_int64], ctypes.c_size_t),
    "mbar_create_factorised": ([ctypes.POINTER(_vp), ctypes.c_int64, ctypes.c_int64, _i64p, _vp, _vp, _vp,
                                ctypes.c_int32, ctypes.POINTER(Opts), _vp], ctypes.c_int),
    "mbar_lse_pass_factorised": ([_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp, _vp,
                                  ctypes.c_size_t, _vp], ctypes.c_int),
    "mbar_lse_pass_samples": ([_vp, ctypes.c_int64, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t,
                               _vp], ctypes.c_int),
}


def lib():
    """The loaded library (loads it on first use)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise LibraryMissing(
                f"{LIB_PATH} is not built; run `python -m paper_2609_03541_b300.build` (nvcc, sm_103a)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        msg = lib().mbar_last_error().decode(errors="replace")
        raise MbarError(status, msg)


def default_opts(precision: int = MBAR_MIXED, **overrides) -> Opts:
    o = Opts()
    _check(lib().mbar_opts_default(ctypes.byref(o), int(precision)))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _device_ptr(x):
    """(pointer, on_device) for a numpy array or a CUDA torch tensor."""
    if hasattr(x, "data_ptr") and getattr(x, "is_cuda", False):
        return ctypes.c_void_p(x.data_ptr()), 1
    return None, 0


def _factorised_args(a, b, phi, K: int):
    """(arrays kept alive, [a, b, phi] pointers, N, on_device) of a
    factorised input: float64 ``a``, ``b`` (K) and ``phi`` (N), all numpy
    arrays or all contiguous float64 CUDA tensors."""
    ptrs = [_device_ptr(x) for x in (a, b, phi)]
    on_dev = ptrs[0][1]
    if any(p[1] != on_dev for p in ptrs):
        raise ValueError("a, b and phi must all be host arrays or all CUDA tensors")
    if on_dev:
        for x in (a, b, phi):
            if x.dtype.__repr__() != "torch.float64" or not x.is_contiguous():
                raise ValueError("device a, b, phi must be contiguous float64 CUDA tensors")
        keep = (a, b, phi)
        vp = [p[0] for p in ptrs]
        N = int(phi.numel())
    else:
        keep = tuple(_f64(x) for x in (a, b, phi))
        vp = [ctypes.c_void_p(x.ctypes.data) for x in keep]
        N = int(keep[2].shape[0])
    if len(keep[0]) != K or len(keep[1]) != K:
        raise ValueError("a and b need one entry per state")
    return keep, vp, N, on_dev


class Context:
    """One MBAR problem resident on the device (``mbar_ctx``)."""

    def __init__(self, u_kn, N_k, precision: int = MBAR_MIXED, opts: Opts | None = None, stream=None):
        self._h = ctypes.c_void_p()
        Nk = np.ascontiguousarray(np.asarray(N_k, dtype=np.int64))
        K = int(Nk.shape[0])
        dptr, on_dev = _device_ptr(u_kn)
        if on_dev:
            if u_kn.dtype.__repr__() != "torch.float64" or not u_kn.is_contiguous():
                raise ValueError("device u_kn must be a contiguous float64 CUDA tensor")
            N = int(u_kn.shape[1])
            uptr = dptr
            self._keep = u_kn
        else:
            u = _f64(u_kn)
            N = int(u.shape[1])
            uptr = ctypes.c_void_p(u.ctypes.data)
            self._keep = u
        if opts is None:
            opts = default_opts(precision)
        else:
            opts.precision = precision
        st = ctypes.c_void_p(stream if isinstance(stream, int) else (stream.cuda_stream if stream is not None else 0))
        _check(lib().mbar_create(ctypes.byref(self._h), K, N, Nk.ctypes.data_as(_i64p), uptr, on_dev,
                                 ctypes.byref(opts), st))
        self._keep = None
        self.K, self.N, self.precision = K, N, precision

    @classmethod
    def factorised(cls, a, b, phi, N_k, precision: int = MBAR_MIXED, opts: Opts | None = None, stream=None):
        """``mbar_create_factorised``: u_kn = a_k + b_k phi_n generated on the
        device from float64 ``a``, ``b`` (K) and ``phi`` (N), all numpy
        arrays or all CUDA tensors; ``phi`` also becomes the bin coordinate."""
        self = cls.__new__(cls)
        self._h = ctypes.c_void_p()
        Nk = np.ascontiguousarray(np.asarray(N_k, dtype=np.int64))
        K = int(Nk.shape[0])
        keep, vp, N, on_dev = _factorised_args(a, b, phi, K)
        if opts is None:
            opts = default_opts(precision)
        else:
            opts.precision = precision
        st = ctypes.c_void_p(stream if isinstance(stream, int) else (stream.cuda_stream if stream is not None else 0))
        _check(lib().mbar_create_factorised(ctypes.byref(self._h), K, N, Nk.ctypes.data_as(_i64p), vp[0], vp[1],
                                            vp[2], on_dev, ctypes.byref(opts), st))
        self._keep = None
        self.K, self.N, self.precision = K, N, precision
        return self

    # -- binning ---------------------------------------------------------
    def set_coordinate(self, phi):
        dptr, on_dev = _device_ptr(phi)
        if on_dev:
            _check(lib().mbar_set_coordinate(self._h, dptr, 1))
        else:
            p = _f64(phi)
            _check(lib().mbar_set_coordinate(self._h, ctypes.c_void_p(p.ctypes.data), 0))

    def bin(self, h: float) -> int:
        nb = ctypes.c_int64()
        _check(lib().mbar_bin(self._h, float(h), ctypes.byref(nb)))
        return nb.value

    def bin_count(self, n: int):
        w = ctypes.c_double()
        nb = ctypes.c_int64()
        _check(lib().mbar_bin_count(self._h, int(n), ctypes.byref(w), ctypes.byref(nb)))
        return w.value, nb.value

    def get_bins(self, n_bins: int):
        keys = np.empty(n_bins, dtype=np.int64)
        H = np.empty(n_bins, dtype=np.int64)
        u = np.empty((self.K, n_bins), dtype=np.float64)
        _check(lib().mbar_get_bins(self._h, keys.ctypes.data_as(_i64p), H.ctypes.data_as(_i64p), _ptr(u)))
        return keys, H, u

    # -- evaluation ----------------------------------------------------------
    def sci_step(self, f, n_cols: int | None = None, want_logden: bool = False):
        f = _f64(f)
        fo = np.empty(self.K)
        g = np.empty(self.K)
        s = np.empty(1)
        ld = np.empty(n_cols if n_cols is not None else self.N) if want_logden else None
        _check(lib().mbar_sci_step(self._h, _ptr(f), _ptr(fo), _ptr(g), _ptr(s),
                                   _ptr(ld) if ld is not None else None))
        return (fo, g, float(s[0]), ld) if want_logden else (fo, g, float(s[0]))

    def hessian(self, f):
        f = _f64(f)
        H = np.empty((self.K, self.K))
        _check(lib().mbar_hessian(self._h, _ptr(f), _ptr(H)))
        return H

    def covariance(self):
        """``mbar_covariance``: K x K asymptotic covariance of f at the current
        solution, gauge f_0 = 0 (row and column 0 zero)."""
        C = np.empty((self.K, self.K))
        _check(lib().mbar_covariance(self._h, _ptr(C)))
        return C

    def newton_step(self, f):
        f = _f64(f)
        fo = np.empty(self.K)
        st = ctypes.c_double()
        _check(lib().mbar_newton_step(self._h, _ptr(f), _ptr(fo), ctypes.byref(st)))
        return fo, st.value

    def solve(self, f_init=None) -> Report:
        rep = Report()
        fi = _f64(f_init) if f_init is not None else None
        _check(lib().mbar_solve(self._h, _ptr(fi) if fi is not None else None, ctypes.byref(rep)))
        return rep

    def free_energies(self) -> np.ndarray:
        f = np.empty(self.K)
        _check(lib().mbar_free_energies(self._h, _ptr(f)))
        return f

    def device_bytes(self) -> int:
        b = ctypes.c_int64()
        _check(lib().mbar_device_bytes(self._h, ctypes.byref(b)))
        return b.value

    def set_exclusive(self, exclusive: bool):
        """``mbar_set_exclusive``: True (default) lets the solve use every SM
        (graphs, the whole-GPU loop on small levels); False for contexts
        that share the GPU with concurrent solves."""
        _check(lib().mbar_set_exclusive(self._h, int(bool(exclusive))))

    def set_timing(self, enable: bool):
        _check(lib().mbar_set_timing(self._h, int(bool(enable))))

    def timing(self, kind: int):
        """(launches, total device ms, streamed bytes) of one launch kind:
        0 unbinned LSE pass, 1 Hessian, 2 Newton solve, 3 unbinned pass that
        only confirms a Newton step below f_tol, 4 second-loop round of
        Algorithm 1 (binned passes), 5 one-launch first loop."""
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        by = ctypes.c_double()
        _check(lib().mbar_get_timing(self._h, int(kind), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)))
        return n.value, ms.value, by.value

    def trace(self) -> np.ndarray:
        """Rows (phase, n, a, b) of the last solve (see mbar_get_trace)."""
        n = ctypes.c_int64()
        _check(lib().mbar_get_trace(self._h, ctypes.byref(n), None, 0))
        out = np.empty((n.value, 4))
        _check(lib().mbar_get_trace(self._h, ctypes.byref(n), _ptr(out), n.value))
        return out

    # -- reweighting (Eqs. 5-6) and the weighted 2-D histogram -----------------
    def reweight(self, u0):
        """(p, log C): weights of every sample (original order) at the target
        state with reduced potential u0 (``mbar_reweight``)."""
        p = np.empty(self.N)
        logc = ctypes.c_double()
        dptr, on_dev = _device_ptr(u0)
        if on_dev:
            _check(lib().mbar_reweight(self._h, dptr, 1, _ptr(p), ctypes.byref(logc)))
        else:
            a = _f64(u0)
            _check(lib().mbar_reweight(self._h, ctypes.c_void_p(a.ctypes.data), 0, _ptr(p), ctypes.byref(logc)))
        return p, logc.value

    def weighted_histogram2d(self, x, y, x0: float, dx: float, nx: int, y0: float, dy: float, ny: int):
        """``mbar_weighted_histogram2d`` of the last reweight weights."""
        out = np.empty((int(nx), int(ny)))
        xa, ya = _f64(x), _f64(y)
        _check(lib().mbar_weighted_histogram2d(self._h, ctypes.c_void_p(xa.ctypes.data), ctypes.c_void_p(ya.ctypes.data),
                                               0, float(x0), float(dx), int(nx), float(y0), float(dy), int(ny),
                                               _ptr(out)))
        return out

    def close(self):
        if self._h:
            _check(lib().mbar_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_hessian_path(path: int):
    """0 = by size (tensor cores for K >= 64), 1 = CUDA cores, 2 = tensor cores."""
    _check(lib().mbar_set_hessian_path(int(path)))


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    n = ctypes.c_int64()
    _check(lib().mbar_kernel_launches(ctypes.byref(n)))
    return n.value


def lse_scratch_bytes(K: int, n: int, dtype_bytes: int) -> int:
    return int(lib().mbar_lse_scratch_bytes(int(K), int(n), int(dtype_bytes)))


def lse_pass(v, f, log_N, Q, H=None, logden=None, scratch=None, stream=None):
    """Stateless fused LSE pass over a resident K x n CUDA tensor ``v``
    (float32 or float64, row pitch = v.stride(0)). All arguments are CUDA
    tensors; ``scratch`` is a uint8 tensor of ``lse_scratch_bytes`` bytes,
    zero before its first use."""
    K, n = int(v.shape[0]), int(v.shape[1])
    eb = int(v.element_size())
    st = stream.cuda_stream if stream is not None else 0
    _check(lib().mbar_lse_pass(
        ctypes.c_void_p(v.data_ptr()), eb, K, n, int(v.stride(0)),
        ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(log_N.data_ptr()),
        ctypes.c_void_p(H.data_ptr()) if H is not None else None,
        ctypes.c_void_p(Q.data_ptr()),
        ctypes.c_void_p(logden.data_ptr()) if logden is not None else None,
        ctypes.c_void_p(scratch.data_ptr()), int(scratch.numel()), ctypes.c_void_p(st)))


def lse_samples_scratch_bytes(K: int, n: int) -> int:
    return int(lib().mbar_lse_samples_scratch_bytes(int(K), int(n)))


def lse_pass_samples(v_nk, K, f, log_N, Q, H=None, logden=None, scratch=None, stream=None):
    """``mbar_lse_pass_samples``: the fused LSE pass over a sample-major
    float32 CUDA tensor ``v_nk`` of shape (n, Kp), Kp = K rounded up to 4
    (padding entries finite). ``scratch``: uint8 tensor of
    ``lse_samples_scratch_bytes`` bytes, zero before its first use."""
    n = int(v_nk.shape[0])
    st = stream.cuda_stream if stream is not None else 0
    _check(lib().mbar_lse_pass_samples(
        ctypes.c_void_p(v_nk.data_ptr()), int(K), n,
        ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(log_N.data_ptr()),
        ctypes.c_void_p(H.data_ptr()) if H is not None else None,
        ctypes.c_void_p(Q.data_ptr()),
        ctypes.c_void_p(logden.data_ptr()) if logden is not None else None,
        ctypes.c_void_p(scratch.data_ptr()), int(scratch.numel()), ctypes.c_void_p(st)))


def lse_factorised_scratch_bytes(K: int, n: int) -> int:
    return int(lib().mbar_lse_factorised_scratch_bytes(int(K), int(n)))


def lse_pass_factorised(a, b, phi, f, log_N, Q, H=None, logden=None, scratch=None, stream=None):
    """``mbar_lse_pass_factorised``: the fused LSE pass over u_kp = a_k + b_k
    phi_p from float64 CUDA tensors ``a``, ``b`` (K) and ``phi`` (n);
    ``logden`` float64 (n) or None. ``scratch``: uint8 tensor of
    ``lse_factorised_scratch_bytes`` bytes, zero before its first use."""
    K, n = int(a.numel()), int(phi.numel())
    st = stream.cuda_stream if stream is not None else 0
    _check(lib().mbar_lse_pass_factorised(
        ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(phi.data_ptr()), K, n,
        ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(log_N.data_ptr()),
        ctypes.c_void_p(H.data_ptr()) if H is not None else None,
        ctypes.c_void_p(Q.data_ptr()),
        ctypes.c_void_p(logden.data_ptr()) if logden is not None else None,
        ctypes.c_void_p(scratch.data_ptr()), int(scratch.numel()), ctypes.c_void_p(st)))


def lse_pass_static(v, f, log_N, Q, H=None, logden=None, stream=None):
    """``mbar_lse_pass_static``: the fused LSE pass with the library's built-in
    scratch array (no device allocation by the call). Arguments as in
    ``lse_pass`` minus ``scratch``."""
    K, n = int(v.shape[0]), int(v.shape[1])
    st = stream.cuda_stream if stream is not None else 0
    _check(lib().mbar_lse_pass_static(
        ctypes.c_void_p(v.data_ptr()), int(v.element_size()), K, n, int(v.stride(0)),
        ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(log_N.data_ptr()),
        ctypes.c_void_p(H.data_ptr()) if H is not None else None,
        ctypes.c_void_p(Q.data_ptr()),
        ctypes.c_void_p(logden.data_ptr()) if logden is not None else None,
        ctypes.c_void_p(st)))


# ---------------------------------------------------------------------------
# serving and batching (mbar_server_* / mbar_batch_solve)
# ---------------------------------------------------------------------------

def footprint_bytes(K: int, N: int, precision: int = MBAR_MIXED, use_binning: int = 1) -> int:
    """``mbar_footprint_bytes``: estimated peak device memory of one solve."""
    return int(lib().mbar_footprint_bytes(int(K), int(N), int(precision), int(use_binning)))


def autotune_lse(family: int, K: int, n: int) -> dict:
    """``mbar_autotune_lse``: the tuned launch shape of one LSE pass family
    (TUNE_SAMPLES or TUNE_FACTORISED) for (K, n); searched unless cached."""
    r = TuneResult()
    _check(lib().mbar_autotune_lse(int(family), int(K), int(n), ctypes.byref(r)))
    return r.as_dict()


def autotune_enable(on: bool = True) -> None:
    """``mbar_autotune_enable``: plans take the tuned shapes (process-wide)."""
    _check(lib().mbar_autotune_enable(1 if on else 0))


def autotune_cache(path) -> None:
    """``mbar_autotune_cache``: append tuned shapes to, and load them from, ``path``."""
    _check(lib().mbar_autotune_cache(None if path is None else str(path).encode()))


def autotune_clear() -> None:
    """``mbar_autotune_clear``: empty the in-memory table."""
    _check(lib().mbar_autotune_clear())


def footprint_factorised_bytes(K: int, N: int, precision: int = MBAR_MIXED, use_binning: int = 1) -> int:
    """``mbar_footprint_factorised_bytes``: the same for a factorised solve."""
    return int(lib().mbar_footprint_factorised_bytes(int(K), int(N), int(precision), int(use_binning)))


def server_config(workers: int = 8, hbm_budget_bytes: int = 160 << 30, precision: int = MBAR_MIXED,
                  opts: Opts | None = None, persistent: bool = False) -> ServerConfig:
    """``mbar_server_config``; persistent: MBAR_BATCH_PERSISTENT for
    ``batch_solve`` (the first loops of a group in one persistent launch)."""
    cfg = ServerConfig()
    cfg.workers = int(workers)
    cfg.flags = BATCH_PERSISTENT if persistent else 0
    cfg.hbm_budget_bytes = int(hbm_budget_bytes)
    cfg.opts = opts if opts is not None else default_opts(precision)
    cfg.opts.precision = int(precision)
    return cfg


def _u_arg(u_kn):
    """(pointer, on_device, keep-alive object, N) for a host array or a CUDA tensor."""
    dptr, on_dev = _device_ptr(u_kn)
    if on_dev:
        if u_kn.dtype.__repr__() != "torch.float64" or not u_kn.is_contiguous():
            raise ValueError("device u_kn must be a contiguous float64 CUDA tensor")
        return dptr, 1, u_kn, int(u_kn.shape[1])
    u = _f64(u_kn)
    return ctypes.c_void_p(u.ctypes.data), 0, u, int(u.shape[1])


def _phi_arg(phi):
    if phi is None:
        return None, 0, None
    dptr, on_dev = _device_ptr(phi)
    if on_dev:
        return dptr, 1, phi
    p = _f64(phi)
    return ctypes.c_void_p(p.ctypes.data), 0, p


class Server:
    """``mbar_server``: worker threads, each with its own CUDA stream, solve
    admitted requests concurrently; admission keeps the sum of the requests'
    footprints within the memory budget."""

    def __init__(self, cfg: ServerConfig):
        self._h = ctypes.c_void_p()
        _check(lib().mbar_server_create(ctypes.byref(self._h), ctypes.byref(cfg)))
        self._keep = {}
        self._K = {}

    def submit(self, u_kn, N_k, phi=None) -> int:
        Nk = np.ascontiguousarray(np.asarray(N_k, dtype=np.int64))
        uptr, u_dev, ukeep, N = _u_arg(u_kn)
        pptr, p_dev, pkeep = _phi_arg(phi)
        rid = ctypes.c_int64()
        _check(lib().mbar_server_submit(self._h, int(Nk.shape[0]), N, Nk.ctypes.data_as(_i64p), uptr, u_dev, pptr,
                                        p_dev, ctypes.byref(rid)))
        self._keep[rid.value] = (ukeep, pkeep)   # read at admission: alive until wait
        self._K[rid.value] = int(Nk.shape[0])
        return rid.value

    def submit_factorised(self, a, b, phi, N_k) -> int:
        """``mbar_server_submit_factorised``: one solve of u_kn = a_k +
        b_k phi_n (arguments as ``Context.factorised``)."""
        Nk = np.ascontiguousarray(np.asarray(N_k, dtype=np.int64))
        K = int(Nk.shape[0])
        keep, vp, N, on_dev = _factorised_args(a, b, phi, K)
        rid = ctypes.c_int64()
        _check(lib().mbar_server_submit_factorised(self._h, K, N, Nk.ctypes.data_as(_i64p), vp[0], vp[1], vp[2],
                                                   on_dev, ctypes.byref(rid)))
        self._keep[rid.value] = keep   # read at admission: alive until wait
        self._K[rid.value] = K
        return rid.value

    def poll(self, rid: int) -> int:
        st = ctypes.c_int32()
        _check(lib().mbar_server_poll(self._h, int(rid), ctypes.byref(st)))
        return st.value

    def wait(self, rid: int):
        """(f, report, latency_s, run_s) of request ``rid``; raises on a failed solve."""
        f = np.zeros(self._K[rid])
        rep = Report()
        lat = ctypes.c_double()
        run = ctypes.c_double()
        status = lib().mbar_server_wait(self._h, int(rid), _ptr(f), ctypes.byref(rep), ctypes.byref(lat),
                                        ctypes.byref(run))
        self._keep.pop(rid, None)
        self._K.pop(rid, None)
        _check(status)
        return f, rep, lat.value, run.value

    def stats(self):
        c = ctypes.c_int64()
        pr = ctypes.c_int32()
        pb = ctypes.c_uint64()
        _check(lib().mbar_server_stats(self._h, ctypes.byref(c), ctypes.byref(pr), ctypes.byref(pb)))
        return {"completed": c.value, "peak_running": pr.value, "peak_bytes": pb.value}

    def close(self):
        if self._h:
            _check(lib().mbar_server_destroy(self._h))
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def batch_solve(problems, cfg: ServerConfig):
    """``mbar_batch_solve`` over ``problems`` = [(u_kn, N_k, phi or None), ...]
    (all host arrays or all CUDA tensors). Returns ([f_p], [report_p], [status_p])."""
    P = len(problems)
    Ks, Ns, nk_arrs, uptrs, pptrs, keep = [], [], [], [], [], []
    on_dev = None
    p_dev = 0
    for u, Nk, phi in problems:
        uptr, ud, ukeep, N = _u_arg(u)
        on_dev = ud if on_dev is None else on_dev
        if ud != on_dev:
            raise ValueError("batch_solve: all u_kn on the host or all on the device")
        pptr, pd, pkeep = _phi_arg(phi)
        if phi is not None:
            p_dev = pd
        nk = np.ascontiguousarray(np.asarray(Nk, dtype=np.int64))
        Ks.append(int(nk.shape[0]))
        Ns.append(N)
        nk_arrs.append(nk)
        uptrs.append(uptr)
        pptrs.append(pptr)
        keep.append((ukeep, pkeep))
    K_a = np.asarray(Ks, dtype=np.int64)
    N_a = np.asarray(Ns, dtype=np.int64)
    nk_ptrs = (_i64p * P)(*[a.ctypes.data_as(_i64p) for a in nk_arrs])
    u_ptrs = (_vp * P)(*[p.value for p in uptrs])
    phi_ptrs = (_vp * P)(*[(p.value if p is not None else None) for p in pptrs])
    fs = [np.zeros(k) for k in Ks]
    f_ptrs = (_dp * P)(*[_ptr(f) for f in fs])
    reps = (Report * P)()
    sts = (ctypes.c_int * P)()
    lib().mbar_batch_solve(P, K_a.ctypes.data_as(_i64p), N_a.ctypes.data_as(_i64p), nk_ptrs, u_ptrs, int(on_dev or 0),
                           phi_ptrs, int(p_dev), ctypes.byref(cfg), f_ptrs, reps, sts)
    return fs, [reps[i] for i in range(P)], [int(sts[i]) for i in range(P)]


def selftest_wait_timeout(limit_us: int = 50_000):
    """``mbar_selftest_wait_timeout``: (status name, seconds waited)."""
    w = ctypes.c_double()
    st = lib().mbar_selftest_wait_timeout(int(limit_us), ctypes.byref(w))
    return STATUS.get(st, str(st)), w.value
