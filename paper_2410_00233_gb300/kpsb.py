"""Thin ctypes binding of the kpsb C ABI (include/kpsb.h); argument marshalling only.

Every computation runs in libkpsb.so (CUDA, sm_103a).  Images and factors are column-major
(numpy Fortran order); host arrays are copied into Fortran-contiguous float64/float32
buffers before the call.  Device pointers are plain integers (e.g. ``tensor.data_ptr()``)
and streams are ``cudaStream_t`` handles as integers (``torch.cuda.Stream.cuda_stream``).
The library must have been built (``python -m paper_2410_00233_gb300.build`` or
``__graft_entry__.build()``); loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkpsb.so")

KPSB_OK = 0
STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "EBREAKDOWN",
          -6: "ENOTCONV", -7: "EBUSY", -8: "ENOTFOUND"}
BC_ZERO, BC_REFLEXIVE = 0, 1
EGKB, RSVD = 0, 1
ANISO, ISO = 0, 1
P_FP64, P_FP32, P_TF32X3, P_TF32X2, P_BF16X3, P_BF16X2 = 0, 1, 2, 3, 4, 5
THR_EXACT, THR_PAPER = 0, 1


class KpsbError(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__(f"{fn} failed: {STATUS.get(code, code)} ({msg})")
        self.code = code


class BuildOpts(C.Structure):
    _fields_ = [("p", C.c_int), ("k_min", C.c_int), ("one_sided", C.c_int), ("power_iters", C.c_int),
                ("seed", C.c_ulonglong), ("start_host", C.POINTER(C.c_float)), ("stream", C.c_void_p),
                ("fp64", C.c_int)]


class SBOpts(C.Structure):
    _fields_ = [("beta", C.c_double), ("tau_sb", C.c_double), ("tau_cgls", C.c_double),
                ("i_max", C.c_int), ("fixed_inner", C.c_int), ("prec", C.c_int),
                ("threshold_rule", C.c_int), ("stream", C.c_void_p), ("sub_batches", C.c_int)]


class SBStats(C.Structure):
    _fields_ = [("l_end", C.c_int), ("iota_total", C.c_int), ("rc_sb", C.c_double), ("status", C.c_int)]


class Problem(C.Structure):
    _fields_ = [("psf", C.POINTER(C.c_double)), ("s0", C.c_int), ("s1", C.c_int), ("n", C.c_int),
                ("bc", C.c_int), ("rank_or_tol", C.c_double), ("method", C.c_int), ("opts", BuildOpts)]


class SBJob(C.Structure):
    _fields_ = [("kp", C.c_void_p), ("b", C.c_void_p), ("x", C.c_void_p), ("mu", C.c_double),
                ("lambda_", C.c_double), ("beta", C.c_double), ("tv", C.c_int), ("iters", C.c_int),
                ("stats", C.POINTER(SBStats))]


class Request(C.Structure):
    _fields_ = [("psf", C.POINTER(C.c_double)), ("s0", C.c_int), ("s1", C.c_int), ("n", C.c_int),
                ("bc", C.c_int), ("rank_or_tol", C.c_double), ("method", C.c_int),
                ("b", C.POINTER(C.c_double)), ("mu", C.c_double), ("lambda_", C.c_double),
                ("beta", C.c_double), ("tv", C.c_int), ("iters", C.c_int), ("prec", C.c_int),
                ("psf_key", C.c_ulonglong)]


class SrvStats(C.Structure):
    _fields_ = [("submitted", C.c_ulonglong), ("completed", C.c_ulonglong), ("failed", C.c_ulonglong),
                ("cache_hits", C.c_ulonglong), ("cache_misses", C.c_ulonglong), ("rounds", C.c_ulonglong),
                ("bytes_in_use", C.c_size_t), ("peak_bytes", C.c_size_t), ("active", C.c_int),
                ("queued", C.c_int), ("cached", C.c_int)]


_lib = None

_SIGS = {
    "kp_build": (C.c_int, [C.POINTER(C.c_double), C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                           C.c_int, C.POINTER(BuildOpts), C.POINTER(C.c_void_p)]),
    "kp_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                          C.POINTER(C.c_double)]),
    "kp_get_factors": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                 C.POINTER(C.c_double)]),
    "kp_from_factors": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                  C.POINTER(C.c_double), C.POINTER(C.c_void_p)]),
    "kp_apply": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int, C.c_int]),
    "kp_dense_blur": (C.c_int, [C.POINTER(C.c_double), C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "kp_build_dense": (C.c_int, [C.POINTER(C.c_double), C.c_int, C.c_double, C.c_int, C.POINTER(BuildOpts),
                                 C.POINTER(C.c_void_p)]),
    "kp_apply_dev": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "kp_free": (None, [C.c_void_p]),
    "sb_solve": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_double, C.c_double, C.c_int, C.c_int,
                           C.POINTER(SBOpts), C.POINTER(C.c_double), C.POINTER(SBStats)]),
    "sb_solve_dev": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_int,
                               C.POINTER(SBOpts), C.c_void_p, C.POINTER(SBStats)]),
    "kp_build_batched": (C.c_int, [C.c_int, C.POINTER(Problem), C.POINTER(C.c_void_p)]),
    "sb_solve_batched": (C.c_int, [C.c_int, C.POINTER(SBJob), C.c_int, C.POINTER(SBOpts)]),
    "kp_blur_dev": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                              C.c_int, C.c_void_p]),
    "kp_ra_apply_dev": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int,
                                  C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "kp_ra_apply_noalloc_dev": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                          C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "kp_ra_materialize_dev": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                        C.c_void_p]),
    "kpsb_small_svd": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "kpsb_last_error": (C.c_char_p, []),
    "srv_create": (C.c_int, [C.c_size_t, C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "srv_submit": (C.c_int, [C.c_void_p, C.POINTER(Request), C.POINTER(C.c_ulonglong)]),
    "srv_poll": (C.c_int, [C.c_void_p, C.c_ulonglong, C.c_longlong, C.POINTER(C.c_double),
                           C.POINTER(SBStats), C.POINTER(C.c_double)]),
    "srv_stats": (C.c_int, [C.c_void_p, C.POINTER(SrvStats)]),
    "srv_destroy": (None, [C.c_void_p]),
    "kpsb_kernel_launches": (C.c_ulonglong, []),
    "kpsb_gemm_timing": (C.c_int, [C.c_int]),
    "kpsb_gemm_stats": (C.c_int, [C.POINTER(C.c_ulonglong), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "kpsb_timer_stats": (C.c_int, [C.c_int, C.POINTER(C.c_ulonglong), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "kpsb_apply_counts": (C.c_int, [C.POINTER(C.c_ulonglong), C.POINTER(C.c_ulonglong)]),
    "kpsb_conversion_check": (C.c_int, [C.c_ulonglong, C.c_ulonglong, C.POINTER(C.c_ulonglong)]),
    "kpsb_wait_selftest": (C.c_int, [C.c_uint]),
    "kpsb_tuned_variants": (C.c_int, [C.POINTER(C.c_int), C.c_int]),
}


def lib() -> C.CDLL:
    """Loads libkpsb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it first (paper_2410_00233_gb300.build)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return lib().kpsb_last_error().decode()


def _check(fn: str, code: int):
    if code != KPSB_OK:
        raise KpsbError(fn, code, last_error())


def _f64(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _f32(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float32))


def _pd(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _pf(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_float))


class KP:
    """Owning handle of a KP-sum operator (device factors) for n x n images."""

    def __init__(self, ptr: int, n: int | None = None):
        self.ptr = C.c_void_p(ptr)
        self._n = None if n is None else int(n)

    @property
    def n(self) -> int:
        """Image side of the operator (read from the handle once if not known)."""
        if self._n is None:
            self._n = kp_info(self)["n"]
        return self._n

    def close(self):
        if self.ptr and self.ptr.value:
            lib().kp_free(self.ptr)
            self.ptr = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self):
        return kp_info(self)


# The C ABI reads and writes host arrays by the sizes the operator implies, so every host
# array is checked here first: a wrong shape is a ValueError, never an out-of-bounds access.
def _psf2d(psf) -> np.ndarray:
    ps = _f64(psf)
    if ps.ndim != 2 or ps.shape[0] < 1 or ps.shape[1] < 1:
        raise ValueError(f"psf must be a non-empty 2-D array (got shape {ps.shape})")
    return ps


def _image(kp: "KP", a, name: str) -> np.ndarray:
    af = _f64(a)
    n = kp.n
    if af.shape != (n, n):
        raise ValueError(f"{name} must be an {n} x {n} array for this operator (got shape {af.shape})")
    return af


def _check_start(start, n: int, rank_or_tol: float, method: int, p: int):
    """A caller's start is the EGKB start vector y (n^2 entries) or the RSVD test matrix F
    (n^2 x k_p, k_p = k + p with p defaulting to max(2, ceil(k/4)), as the library does)."""
    if start is None:
        return
    if method == RSVD:
        if rank_or_tol < 1.0:
            return  # the library rejects automatic rank with RSVD itself
        k = int(rank_or_tol)
        need = n * n * (k + (int(p) if p > 0 else max(2, (k + 3) // 4)))
    else:
        need = n * n
    if np.size(start) != need:
        raise ValueError(f"start must have {need} entries for this build (got {np.size(start)})")


def _build_opts(p=0, k_min=0, one_sided=False, power_iters=0, seed=0, start=None, stream=0, fp64=False):
    o = BuildOpts()
    o.fp64 = int(bool(fp64))
    o.p, o.k_min, o.one_sided, o.power_iters = int(p), int(k_min), int(bool(one_sided)), int(power_iters)
    o.seed = int(seed)
    keep = None
    if start is not None:
        keep = _f32(start)
        o.start_host = _pf(keep)
    o.stream = C.c_void_p(int(stream)) if stream else None
    return o, keep


def kp_build(psf, n: int, bc: int, rank_or_tol: float, method: int = EGKB, *, p=0, k_min=0,
             one_sided=False, power_iters=0, seed=0, start=None, stream=0, fp64=False) -> KP:
    """TSVD of R(A) + Terms(A_k) (see kp_build in include/kpsb.h); fp64=True: FP64 TSVD."""
    ps = _psf2d(psf)
    _check_start(start, int(n), float(rank_or_tol), int(method), int(p))
    o, keep = _build_opts(p, k_min, one_sided, power_iters, seed, start, stream, fp64)
    out = C.c_void_p()
    _check("kp_build", lib().kp_build(_pd(ps), ps.shape[0], ps.shape[1], int(n), int(bc),
                                      float(rank_or_tol), int(method), C.byref(o), C.byref(out)))
    del keep
    return KP(out.value, n)


def kp_build_dense(A, n: int, rank_or_tol: float, method: int = EGKB, *, p=0, k_min=0, one_sided=False,
                   power_iters=0, seed=0, start=None, stream=0, fp64=False) -> KP:
    """KP sum of a general operator given as an explicit (n^2 x n^2) matrix (see kp_build_dense)."""
    a = _f64(A)
    if a.shape != (n * n, n * n):
        raise ValueError(f"A must be {n * n} x {n * n}")
    _check_start(start, int(n), float(rank_or_tol), int(method), int(p))
    o, keep = _build_opts(p, k_min, one_sided, power_iters, seed, start, stream, fp64)
    out = C.c_void_p()
    _check("kp_build_dense", lib().kp_build_dense(_pd(a), int(n), float(rank_or_tol), int(method), C.byref(o),
                                                  C.byref(out)))
    del keep
    return KP(out.value, n)


def kp_info(kp: KP):
    n, k, kps = C.c_int(), C.c_int(), C.c_int()
    _check("kp_info", lib().kp_info(kp.ptr, C.byref(n), C.byref(k), C.byref(kps), None))
    sig = np.zeros(k.value)
    _check("kp_info", lib().kp_info(kp.ptr, None, None, None, _pd(sig)))
    return dict(n=n.value, k=k.value, kp=kps.value, sigma=sig)


def kp_get_factors(kp: KP):
    inf = kp_info(kp)
    n, k = inf["n"], inf["k"]
    Ax = np.zeros((n * n * k,), dtype=np.float32)
    Ay = np.zeros((n * n * k,), dtype=np.float32)
    sig = np.zeros(k)
    _check("kp_get_factors", lib().kp_get_factors(kp.ptr, _pf(Ax), _pf(Ay), _pd(sig)))
    # term i is the column-major n x n block i
    Ax = Ax.reshape(k, n * n).reshape(k, n, n).transpose(0, 2, 1)
    Ay = Ay.reshape(k, n * n).reshape(k, n, n).transpose(0, 2, 1)
    return np.ascontiguousarray(Ax), np.ascontiguousarray(Ay), sig


def kp_from_factors(Ax, Ay, sigma) -> KP:
    """Handle from k terms Ax[i], Ay[i] (n x n each) and sigma (k)."""
    Ax = np.asarray(Ax, dtype=np.float32)
    Ay = np.asarray(Ay, dtype=np.float32)
    if Ax.ndim != 3 or Ax.shape[1] != Ax.shape[2] or Ay.shape != Ax.shape:
        raise ValueError(f"Ax and Ay must both be k x n x n (got {Ax.shape} and {Ay.shape})")
    k, n, _ = Ax.shape
    if np.shape(sigma) != (k,):
        raise ValueError(f"sigma must have k = {k} entries (got shape {np.shape(sigma)})")
    ax = np.ascontiguousarray(Ax.transpose(0, 2, 1)).reshape(-1)  # column-major blocks
    ay = np.ascontiguousarray(Ay.transpose(0, 2, 1)).reshape(-1)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    out = C.c_void_p()
    _check("kp_from_factors", lib().kp_from_factors(n, k, _pf(ax), _pf(ay), _pd(sg), C.byref(out)))
    return KP(out.value, n)


def kp_dense_blur(psf, n: int, bc: int) -> KP:
    """Handle of the explicit blurring operator A (n^2 x n^2 FP64 on the device, n <= 128)."""
    pf = _psf2d(psf)
    out = C.c_void_p()
    _check("kp_dense_blur", lib().kp_dense_blur(_pd(pf), pf.shape[0], pf.shape[1], int(n), int(bc), C.byref(out)))
    return KP(out.value, n)


def kp_apply(kp: KP, X, transpose: int = 0, prec: int = P_FP64) -> np.ndarray:
    """Y = sum_i sigma_i Ay_i X Ax_i^T (transpose = 0) or its adjoint, X an n x n array."""
    Xf = _image(kp, X, "X")
    Y = np.zeros_like(Xf, order="F")
    _check("kp_apply", lib().kp_apply(kp.ptr, _pd(Xf), _pd(Y), int(transpose), int(prec)))
    return Y


def kp_apply_dev(kp: KP, X_ptr: int, Y_ptr: int, transpose: int = 0, prec: int = P_FP64, stream=0):
    _check("kp_apply_dev", lib().kp_apply_dev(kp.ptr, C.c_void_p(X_ptr), C.c_void_p(Y_ptr), int(transpose),
                                              int(prec), C.c_void_p(int(stream)) if stream else None))


def _sb_opts(beta=0.0, tau_sb=0.0, tau_cgls=0.0, i_max=0, fixed_inner=False, prec=P_FP64,
             threshold_rule=THR_EXACT, stream=0, sub_batches=0) -> SBOpts:
    o = SBOpts()
    o.beta, o.tau_sb, o.tau_cgls = float(beta), float(tau_sb), float(tau_cgls)
    o.i_max, o.fixed_inner, o.prec, o.threshold_rule = int(i_max), int(bool(fixed_inner)), int(prec), int(threshold_rule)
    o.stream = C.c_void_p(int(stream)) if stream else None
    o.sub_batches = int(sub_batches)
    return o


@dataclass
class Stats:
    l_end: int
    iota_total: int
    rc_sb: float
    status: int


def _stats(s: SBStats) -> Stats:
    return Stats(s.l_end, s.iota_total, s.rc_sb, s.status)


def sb_solve(kp: KP, b, mu: float, lam: float, tv: int, iters: int, **opts):
    """Split Bregman deblurring on host arrays; returns (x, Stats)."""
    bf = _image(kp, b, "b")
    x = np.zeros_like(bf, order="F")
    st = SBStats()
    o = _sb_opts(**opts)
    _check("sb_solve", lib().sb_solve(kp.ptr, _pd(bf), float(mu), float(lam), int(tv), int(iters),
                                      C.byref(o), _pd(x), C.byref(st)))
    return x, _stats(st)


def sb_solve_dev(kp: KP, b_ptr: int, x_ptr: int, mu: float, lam: float, tv: int, iters: int, **opts):
    st = SBStats()
    o = _sb_opts(**opts)
    _check("sb_solve_dev", lib().sb_solve_dev(kp.ptr, C.c_void_p(b_ptr), float(mu), float(lam), int(tv),
                                              int(iters), C.byref(o), C.c_void_p(x_ptr), C.byref(st)))
    return _stats(st)


def kp_build_batched(problems) -> list:
    """problems: list of dicts with psf, n, bc, rank_or_tol, method and build options."""
    arr = (Problem * len(problems))()
    keep = []
    for i, pr in enumerate(problems):
        ps = _psf2d(pr["psf"])
        _check_start(pr.get("start"), int(pr["n"]), float(pr["rank_or_tol"]), int(pr.get("method", EGKB)),
                     int(pr.get("p", 0)))
        keep.append(ps)
        o, k2 = _build_opts(pr.get("p", 0), pr.get("k_min", 0), pr.get("one_sided", False),
                            pr.get("power_iters", 0), pr.get("seed", 0), pr.get("start"),
                            fp64=pr.get("fp64", False))
        keep.append(k2)
        arr[i].psf = _pd(ps)
        arr[i].s0, arr[i].s1 = ps.shape
        arr[i].n, arr[i].bc = int(pr["n"]), int(pr["bc"])
        arr[i].rank_or_tol = float(pr["rank_or_tol"])
        arr[i].method = int(pr.get("method", EGKB))
        arr[i].opts = o
    outs = (C.c_void_p * len(problems))()
    code = lib().kp_build_batched(len(problems), arr, outs)
    # every non-NULL handle is the caller's, also when another problem failed
    kps = [KP(outs[i], int(pr["n"])) if outs[i] else None for i, pr in enumerate(problems)]
    if code != KPSB_OK:
        err = KpsbError("kp_build_batched", code, last_error())
        for kp in kps:
            if kp is not None:
                kp.close()
        raise err
    return kps


def sb_solve_batched(jobs, on_device: bool = False, **opts):
    """jobs: list of dicts with kp, b, mu, lam, tv, iters (and beta).  Host mode: b are
    arrays and the results are returned; device mode: b and x are device pointers."""
    arr = (SBJob * len(jobs))()
    stats = (SBStats * len(jobs))()
    keep, outs = [], []
    for i, j in enumerate(jobs):
        arr[i].kp = j["kp"].ptr
        if on_device:
            arr[i].b, arr[i].x = j["b"], j["x"]
        else:
            bf = _image(j["kp"], j["b"], f"jobs[{i}]['b']")
            xf = np.zeros_like(bf, order="F")
            keep.append(bf)
            outs.append(xf)
            arr[i].b, arr[i].x = bf.ctypes.data, xf.ctypes.data
        arr[i].mu, arr[i].lambda_ = float(j["mu"]), float(j["lam"])
        arr[i].beta = float(j.get("beta", 0.0))
        arr[i].tv, arr[i].iters = int(j["tv"]), int(j["iters"])
        arr[i].stats = C.pointer(stats[i])
    o = _sb_opts(**opts)
    _check("sb_solve_batched", lib().sb_solve_batched(len(jobs), arr, int(bool(on_device)), C.byref(o)))
    st = [_stats(stats[i]) for i in range(len(jobs))]
    return (st if on_device else (outs, st))


def kp_blur_dev(psf_ptr: int, s0: int, s1: int, n: int, bc: int, X_ptr: int, B_ptr: int,
                transpose: int = 0, stream=0):
    _check("kp_blur_dev", lib().kp_blur_dev(C.c_void_p(psf_ptr), s0, s1, n, bc, C.c_void_p(X_ptr),
                                            C.c_void_p(B_ptr), int(transpose),
                                            C.c_void_p(int(stream)) if stream else None))


def kp_ra_apply_dev(psf_ptr: int, s0: int, s1: int, n: int, bc: int, V_ptr: int, ldv: int, nb: int,
                    U_ptr: int, ldu: int, transpose: int = 0, stream=0):
    _check("kp_ra_apply_dev", lib().kp_ra_apply_dev(C.c_void_p(psf_ptr), s0, s1, n, bc, C.c_void_p(V_ptr),
                                                    ldv, nb, C.c_void_p(U_ptr), ldu, int(transpose),
                                                    C.c_void_p(int(stream)) if stream else None))


def kp_ra_apply_noalloc_dev(psf_ptr: int, s0: int, s1: int, n: int, bc: int, V_ptr: int, ldv: int,
                            nb: int, U_ptr: int, ldu: int, transpose: int = 0, stream=0):
    """kp_ra_apply_dev with library-owned fixed scratch (no device allocation in the call)."""
    _check("kp_ra_apply_noalloc_dev", lib().kp_ra_apply_noalloc_dev(
        C.c_void_p(psf_ptr), s0, s1, n, bc, C.c_void_p(V_ptr), ldv, nb, C.c_void_p(U_ptr), ldu,
        int(transpose), C.c_void_p(int(stream)) if stream else None))


def kp_ra_materialize_dev(psf_ptr: int, s0: int, s1: int, n: int, bc: int, R_ptr: int, stream=0):
    _check("kp_ra_materialize_dev", lib().kp_ra_materialize_dev(
        C.c_void_p(psf_ptr), s0, s1, n, bc, C.c_void_p(R_ptr), C.c_void_p(int(stream)) if stream else None))


class Server:
    """Continuous-batching deblur server (srv_* of include/kpsb.h)."""

    def __init__(self, budget_bytes: int, max_active: int = 64, round_steps: int = 5):
        out = C.c_void_p()
        _check("srv_create", lib().srv_create(int(budget_bytes), int(max_active), int(round_steps),
                                              C.byref(out)))
        self.ptr = out
        self._n = {}

    def submit(self, psf, n, bc, rank_or_tol, b, mu, lam, tv, iters, *, method=EGKB, beta=0.0,
               prec=P_TF32X2, psf_key=0) -> int:
        ps = _psf2d(psf)
        bf = _f64(b)
        if bf.shape != (int(n), int(n)):
            raise ValueError(f"b must be an {int(n)} x {int(n)} array (got shape {bf.shape})")
        r = Request()
        r.psf = _pd(ps)
        r.s0, r.s1 = ps.shape
        r.n, r.bc, r.rank_or_tol, r.method = int(n), int(bc), float(rank_or_tol), int(method)
        r.b = _pd(bf)
        r.mu, r.lambda_, r.beta = float(mu), float(lam), float(beta)
        r.tv, r.iters, r.prec, r.psf_key = int(tv), int(iters), int(prec), int(psf_key)
        rid = C.c_ulonglong()
        _check("srv_submit", lib().srv_submit(self.ptr, C.byref(r), C.byref(rid)))
        self._n[rid.value] = int(n)
        return rid.value

    def poll(self, rid: int, timeout_us: int = -1):
        """(x, Stats, latency_s) when done, None on timeout; raises if the request failed."""
        n = self._n[rid]
        x = np.zeros((n, n), order="F")
        st = SBStats()
        lat = C.c_double()
        code = lib().srv_poll(self.ptr, C.c_ulonglong(rid), int(timeout_us), _pd(x), C.byref(st), C.byref(lat))
        if code == -4:
            return None
        self._n.pop(rid, None)
        _check("srv_poll", code)
        return x, _stats(st), lat.value

    def stats(self) -> dict:
        st = SrvStats()
        _check("srv_stats", lib().srv_stats(self.ptr, C.byref(st)))
        return {f: getattr(st, f) for f, _ in SrvStats._fields_}

    def close(self):
        if self.ptr and self.ptr.value:
            lib().srv_destroy(self.ptr)
            self.ptr = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kpsb_kernel_launches() -> int:
    return int(lib().kpsb_kernel_launches())


def kpsb_gemm_timing(enable: bool):
    _check("kpsb_gemm_timing", lib().kpsb_gemm_timing(int(bool(enable))))


def kpsb_gemm_stats():
    """(launches, milliseconds, algorithmic flops) of the recorded KP GEMM applies."""
    L, ms, fl = C.c_ulonglong(), C.c_double(), C.c_double()
    _check("kpsb_gemm_stats", lib().kpsb_gemm_stats(C.byref(L), C.byref(ms), C.byref(fl)))
    return int(L.value), float(ms.value), float(fl.value)


TIMER_NAMES = ("kp_apply", "cgls_zz", "cgls_x", "cgls_f", "cgls_w", "sb_outer")
# TSVD timer categories: (launches = calls, ms, algorithmic bytes)
TSVD_TIMERS = {"ra_products": 6, "cgs2": 7, "svqb2": 8, "egkb_block": 9}


def kpsb_timer_stats(category: int):
    """(launches, milliseconds, flops) of one timer category (index into TIMER_NAMES)."""
    L, ms, fl = C.c_ulonglong(), C.c_double(), C.c_double()
    _check("kpsb_timer_stats", lib().kpsb_timer_stats(int(category), C.byref(L), C.byref(ms), C.byref(fl)))
    return int(L.value), float(ms.value), float(fl.value)


def kpsb_apply_counts():
    """(problem-applies, sum of k n^3) performed since the last kpsb_gemm_timing(True)."""
    pa, kn3 = C.c_ulonglong(), C.c_ulonglong()
    _check("kpsb_apply_counts", lib().kpsb_apply_counts(C.byref(pa), C.byref(kn3)))
    return int(pa.value), int(kn3.value)


def kpsb_conversion_check(n_random=1 << 26, seed=1):
    """Mismatches of the integer binary32 <-> binary64 conversions against the hardware ones
    (every binary32 value, n_random binary64 values); 0 expected."""
    bad = C.c_ulonglong()
    _check("kpsb_conversion_check", lib().kpsb_conversion_check(C.c_ulonglong(n_random), C.c_ulonglong(seed),
                                                                C.byref(bad)))
    return int(bad.value)


def kpsb_small_svd(A):
    Af = _f64(A)
    m, nc = Af.shape
    U = np.zeros((m, nc), order="F")
    S = np.zeros(nc)
    V = np.zeros((nc, nc), order="F")
    sw = C.c_int()
    _check("kpsb_small_svd", lib().kpsb_small_svd(m, nc, _pd(Af), _pd(U), _pd(S), _pd(V), C.byref(sw)))
    return U, S, V, sw.value


def kpsb_wait_selftest(limit_us: int = 50):
    """Runs the bounded-wait self-test; raises KpsbError (code -4, ETIMEOUT) when the wait ran
    out as designed."""
    _check("kpsb_wait_selftest", lib().kpsb_wait_selftest(int(limit_us)))


VARIANT_NAMES = {0: "two-stage", 1: "fused 64-column", 2: "fused 32-column", 3: "resident"}


def kpsb_tuned_variants():
    """The autotuner's choices so far: list of dicts (n, prec, kmax, bucket, ext, shared, variant)."""
    cnt = lib().kpsb_tuned_variants(None, 0)
    buf = (C.c_int * (7 * max(1, cnt)))()
    cnt = lib().kpsb_tuned_variants(buf, cnt)
    keys = ("n", "prec", "kmax", "bucket", "ext", "shared", "variant")
    return [dict(zip(keys, buf[7 * i:7 * i + 7])) for i in range(cnt)]
