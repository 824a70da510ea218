"""ctypes binding of libexpm.so: argument marshalling only."""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libexpm.so")

EXPM_FP64 = 0
EXPM_MIXED_F32X2 = 1
EXPM_MIXED_FP32 = 2
EXPM_MIXED_TF32X3 = 3
EXPM_MIXED_BF16X3 = 4
EXPM_FLAG_SKIP_FINAL_RESIDUAL = 1

STATUS = {0: "EXPM_OK", 1: "EXPM_EINVAL", 2: "EXPM_ENOMEM", 3: "EXPM_EGROWTH", 4: "EXPM_ENOCONV",
          5: "EXPM_ETIMEOUT", 6: "EXPM_EAGAIN", 7: "EXPM_ECUDA", 8: "EXPM_ENOTFOUND", 9: "EXPM_ENOTSUP"}


class ExpmError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")


class expm_opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("tol", ctypes.c_double), ("max_refine", ctypes.c_int),
                ("t", ctypes.c_double), ("shift_c", ctypes.c_double), ("growth_max", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("flags", ctypes.c_int)]


class expm_op_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_int64), ("d", ctypes.c_void_p), ("e", ctypes.c_void_p),
                ("e_is_complex", ctypes.c_int), ("A", ctypes.c_void_p), ("lda", ctypes.c_int),
                ("a_is_complex", ctypes.c_int)]


EXPM_OP_TRIDIAG = 1
EXPM_OP_DENSE = 2


class expm_info(ctypes.Structure):
    _fields_ = [("refine_iters_max", ctypes.c_int), ("growth_max_seen", ctypes.c_double),
                ("resid_rel_max", ctypes.c_double), ("status_worst", ctypes.c_int)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(library_path):
        raise ImportError(f"{library_path} is missing: build it with "
                          "`python paper_2306_16778_gb300/build.py` (nvcc, sm_103a)")
    L = ctypes.CDLL(library_path)
    vp, i, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    dp = ctypes.POINTER(ctypes.c_double)
    L.expm_opts_default.argtypes = [ctypes.POINTER(expm_opts)]
    L.expm_opts_default.restype = None
    L.expm_status_string.argtypes = [i]
    L.expm_status_string.restype = ctypes.c_char_p
    L.expm_last_error.argtypes = []
    L.expm_last_error.restype = ctypes.c_char_p
    L.expm_coeffs.argtypes = [i, dp, dp]
    L.expm_coeffs.restype = i
    L.expm_plan_create.argtypes = [dp, dp, i, ctypes.POINTER(vp)]
    L.expm_plan_create.restype = i
    L.expm_plan_destroy.argtypes = [vp]
    L.expm_plan_destroy.restype = i
    L.expm_apply_laplacian2d.argtypes = [vp, i, i, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, vp, i, i, vp, ctypes.POINTER(expm_opts),
                                         ctypes.POINTER(expm_info)]
    L.expm_apply_laplacian2d.restype = i
    L.expm_apply_dense_reduced.argtypes = [vp, i, vp, i, i, vp, i, i, i, vp, i, ctypes.POINTER(expm_opts),
                                           ctypes.POINTER(expm_info)]
    L.expm_apply_dense_reduced.restype = i
    L.expm_apply_dense_full.argtypes = [vp, i, vp, i, i, vp, i, ctypes.POINTER(expm_opts), ctypes.POINTER(expm_info)]
    L.expm_apply_dense_full.restype = i
    L.expm_apply_tridiag.argtypes = [vp, i64, vp, vp, i, vp, i, i, vp, ctypes.POINTER(expm_opts),
                                     ctypes.POINTER(expm_info)]
    L.expm_apply_tridiag.restype = i
    L.expm_apply_dense.argtypes = [vp, i, vp, i, i, vp, i, i, i, vp, i, ctypes.POINTER(expm_opts),
                                   ctypes.POINTER(expm_info)]
    L.expm_apply_dense.restype = i
    L.expm_apply_tridiag_noalloc.argtypes = [vp, i64, vp, vp, i, vp, i, i, vp, ctypes.POINTER(expm_opts),
                                             ctypes.POINTER(expm_info)]
    L.expm_apply_tridiag_noalloc.restype = i
    L.expm_apply_batched.argtypes = [vp, i, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(vp), i,
                                     ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int), i, ctypes.POINTER(vp),
                                     ctypes.POINTER(expm_opts), ctypes.POINTER(expm_info)]
    L.expm_apply_batched.restype = i
    L.expm_batched_capture.argtypes = [vp, i, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(vp), i,
                                       ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int), i, ctypes.POINTER(vp),
                                       ctypes.POINTER(expm_opts), i, ctypes.POINTER(vp)]
    L.expm_batched_capture.restype = i
    L.expm_batched_replay.argtypes = [vp, vp, ctypes.POINTER(expm_info)]
    L.expm_batched_replay.restype = i
    L.expm_batched_graph_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(ctypes.c_size_t),
                                          ctypes.POINTER(ctypes.c_double)]
    L.expm_batched_graph_info.restype = i
    ip, dp = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    L.expm_batched_graph_buckets.argtypes = [vp, i, ip, ip, ip, dp, dp]
    L.expm_batched_graph_buckets.restype = i
    L.expm_batched_graph_destroy.argtypes = [vp]
    L.expm_batched_graph_destroy.restype = i
    u64 = ctypes.c_uint64
    L.expm_server_create.argtypes = [ctypes.c_size_t, i, ctypes.POINTER(vp)]
    L.expm_server_create.restype = i
    L.expm_server_register_op.argtypes = [vp, ctypes.POINTER(expm_op_desc), ctypes.POINTER(u64)]
    L.expm_server_register_op.restype = i
    L.expm_server_submit.argtypes = [vp, u64, vp, vp, i, i, vp, ctypes.POINTER(expm_opts), ctypes.POINTER(u64)]
    L.expm_server_submit.restype = i
    L.expm_server_poll.argtypes = [vp, u64, ctypes.POINTER(expm_info), ctypes.POINTER(ctypes.c_double)]
    L.expm_server_poll.restype = i
    L.expm_server_destroy.argtypes = [vp]
    L.expm_server_destroy.restype = i
    L.expm_server_set_queue_limit.argtypes = [vp, i]
    L.expm_server_set_queue_limit.restype = i
    L.expm_queue_create.argtypes = [vp, i, i, i, ctypes.POINTER(expm_opts), i, i, ctypes.c_double, ctypes.POINTER(vp)]
    L.expm_queue_create.restype = i
    L.expm_queue_submit.argtypes = [vp, i, vp, i, vp, i, vp, i, ctypes.c_double, ctypes.c_double,
                                    ctypes.POINTER(u64)]
    L.expm_queue_submit.restype = i
    L.expm_queue_poll.argtypes = [vp, u64, ctypes.POINTER(expm_info)]
    L.expm_queue_poll.restype = i
    L.expm_queue_state.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(u64), ctypes.POINTER(i)]
    L.expm_queue_state.restype = i
    L.expm_queue_destroy.argtypes = [vp]
    L.expm_queue_destroy.restype = i
    for hook in ("expm_internal_server_fail_next_factor", "expm_internal_server_workers_alive"):
        getattr(L, hook).argtypes = [vp]
        getattr(L, hook).restype = i
    L.expm_internal_server_stop_worker.argtypes = [vp, i]
    L.expm_internal_server_stop_worker.restype = i
    L.expm_profile_enable.argtypes = [vp, i]
    L.expm_profile_enable.restype = i
    L.expm_profile_read.argtypes = [vp, i, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(ctypes.c_double)]
    L.expm_profile_read.restype = i
    return L


lib = _load()


def _check(status: int, where: str) -> None:
    if status != 0:
        raise ExpmError(status, where, lib.expm_last_error().decode())


def _ptr(x) -> int:
    """Raw data pointer of a torch tensor or numpy array (must be contiguous)."""
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported buffer type {type(x)}")


def _is_complex(x) -> bool:
    if hasattr(x, "is_complex"):
        return bool(x.is_complex())
    return bool(np.iscomplexobj(x))


def _default_stream(*bufs) -> int:
    for b in bufs:
        if hasattr(b, "is_cuda") and b.is_cuda:
            import torch
            return torch.cuda.current_stream(b.device).cuda_stream
    return 0


def make_opts(prec=EXPM_FP64, t=1.0, shift_c=0.0, stream=None, tol=None, max_refine=None,
              growth_max=None) -> expm_opts:
    o = expm_opts()
    lib.expm_opts_default(ctypes.byref(o))
    o.prec = int(prec)
    o.t = float(t)
    o.shift_c = float(shift_c)
    if tol is not None:
        o.tol = float(tol)
    if max_refine is not None:
        o.max_refine = int(max_refine)
    if growth_max is not None:
        o.growth_max = float(growth_max)
    o.stream = stream
    return o


def expm_coeffs(degree: int) -> tuple[np.ndarray, np.ndarray]:
    """(poles_ri, residues_ri), each 2*degree float64: lambda_k = -theta_k and w_k = a_k."""
    p = np.zeros(2 * degree)
    r = np.zeros(2 * degree)
    _check(lib.expm_coeffs(int(degree), p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           r.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "expm_coeffs")
    return p, r


class Plan:
    """Owns an ``expm_plan`` (pole data resident on the current CUDA device)."""

    def __init__(self, poles_ri=None, residues_ri=None, degree: int | None = None):
        if poles_ri is None:
            poles_ri, residues_ri = expm_coeffs(int(degree))
        poles_ri = np.ascontiguousarray(poles_ri, dtype=np.float64)
        residues_ri = np.ascontiguousarray(residues_ri, dtype=np.float64)
        if degree is None:
            degree = poles_ri.size // 2
        self.degree = int(degree)
        self._h = ctypes.c_void_p()
        _check(lib.expm_plan_create(poles_ri.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    residues_ri.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    self.degree, ctypes.byref(self._h)), "expm_plan_create")

    @property
    def handle(self):
        return self._h

    def close(self) -> None:
        if self._h:
            lib.expm_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def expm_apply_tridiag_noalloc(plan: Plan, d, e, V, Y, prec=EXPM_FP64, t=1.0, shift_c=0.0,
                               stream=None) -> expm_info:
    """As ``expm_apply_tridiag`` but with no device allocation: scratch comes from a
    fixed array inside the library (see include/expm.h).  Device buffers only."""
    N = int(d.shape[0])
    r = int(V.shape[1]) if len(V.shape) == 2 else 1
    if stream is None:
        stream = _default_stream(d, e, V, Y)
    o = make_opts(prec, t, shift_c, stream)
    info = expm_info()
    _check(lib.expm_apply_tridiag_noalloc(plan.handle, N, _ptr(d), _ptr(e), int(_is_complex(e)), _ptr(V), r,
                                          int(_is_complex(V)), _ptr(Y), ctypes.byref(o), ctypes.byref(info)),
           "expm_apply_tridiag_noalloc")
    return info


def expm_profile_enable(plan: Plan, on: bool = True) -> None:
    """Bracket every kernel launch of ``plan`` with CUDA events (resets counters)."""
    _check(lib.expm_profile_enable(plan.handle, int(bool(on))), "expm_profile_enable")


def expm_profile_read(plan: Plan) -> dict:
    """{kernel name: (launches, total device ms)} since the last enable."""
    out = {}
    k = 0
    while True:
        name = ctypes.c_char_p()
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        st = lib.expm_profile_read(plan.handle, k, ctypes.byref(name), ctypes.byref(n), ctypes.byref(ms))
        if st == 8:                       # EXPM_ENOTFOUND: past the last kernel
            return out
        _check(st, "expm_profile_read")
        out[name.value.decode()] = (int(n.value), float(ms.value))
        k += 1


def expm_apply_dense(plan: Plan, A, V, Y, prec=EXPM_FP64, t=1.0, shift_c=0.0, stream=None, tol=None,
                     max_refine=None, growth_max=None, check=True) -> expm_info:
    """Y = e^c R_n(tA - cI) V for a dense Hermitian A (n x n) and V (n x k); see include/expm.h.

    With ``check=False`` EXPM_EGROWTH / EXPM_ENOCONV are returned in ``info.status_worst``
    instead of raised."""
    n = int(A.shape[0])
    k = int(V.shape[1]) if len(V.shape) == 2 else 1
    if stream is None:
        stream = _default_stream(A, V, Y)
    o = make_opts(prec, t, shift_c, stream, tol, max_refine, growth_max)
    info = expm_info()
    st = lib.expm_apply_dense(plan.handle, n, _ptr(A), n, int(_is_complex(A)), _ptr(V), k, k, int(_is_complex(V)),
                              _ptr(Y), k, ctypes.byref(o), ctypes.byref(info))
    if check or st not in (3, 4):
        _check(st, "expm_apply_dense")
    return info


def expm_apply_dense_full(plan: Plan, A, Y, prec=EXPM_FP64, t=1.0, shift_c=0.0, stream=None, tol=None,
                          max_refine=None, growth_max=None, check=True) -> expm_info:
    """Y = e^c R_n(tA - cI), the full matrix (n x n; real for real A, complex128 for complex A)."""
    n = int(A.shape[0])
    if stream is None:
        stream = _default_stream(A, Y)
    o = make_opts(prec, t, shift_c, stream, tol, max_refine, growth_max)
    info = expm_info()
    st = lib.expm_apply_dense_full(plan.handle, n, _ptr(A), n, int(_is_complex(A)), _ptr(Y), n, ctypes.byref(o),
                                   ctypes.byref(info))
    if st != 0 and not (not check and st in (3, 4)):
        _check(st, "expm_apply_dense_full")
    return info


def expm_apply_dense_reduced(plan: Plan, A, V, Y, prec=EXPM_FP64, t=1.0, shift_c=0.0, stream=None, tol=None,
                             max_refine=None, flags=0, want_info=True, check=True):
    """Y = e^c R_n(tA - cI) V through the reduction of A to real tridiagonal form (device
    tensors; see include/expm.h).  ``prec`` selects the tridiagonal solves."""
    n = int(A.shape[0])
    k = int(V.shape[1]) if len(V.shape) == 2 else 1
    if stream is None:
        stream = _default_stream(A, V, Y)
    o = make_opts(prec, t, shift_c, stream, tol, max_refine)
    o.flags = int(flags)
    info = expm_info() if want_info else None
    st = lib.expm_apply_dense_reduced(plan.handle, n, _ptr(A), n, int(_is_complex(A)), _ptr(V), k, k,
                                      int(_is_complex(V)), _ptr(Y), k, ctypes.byref(o),
                                      ctypes.byref(info) if info is not None else None)
    if st != 0 and not (not check and st == 4):
        _check(st, "expm_apply_dense_reduced")
    return info


def expm_apply_laplacian2d(plan: Plan, dx: int, dy: int, ax: float, bx: float, ay: float, by: float, V, Y,
                           prec=EXPM_FP64, t=1.0, shift_c=0.0, stream=None, tol=None, max_refine=None, flags=0,
                           want_info=True, check=True):
    """Y = e^c R_n(tA - cI) V for A = I (x) tridiag(ax, bx, ax) + tridiag(ay, by, ay) (x) I on a
    dx x dy grid (row iy * dx + ix); V, Y device tensors of dx*dy rows (see include/expm.h)."""
    r = int(V.shape[1]) if len(V.shape) == 2 else 1
    if stream is None:
        stream = _default_stream(V, Y)
    o = make_opts(prec, t, shift_c, stream, tol, max_refine)
    o.flags = int(flags)
    info = expm_info() if want_info else None
    st = lib.expm_apply_laplacian2d(plan.handle, int(dx), int(dy), float(ax), float(bx), float(ay), float(by), _ptr(V),
                                    r, int(_is_complex(V)), _ptr(Y), ctypes.byref(o),
                                    ctypes.byref(info) if info is not None else None)
    if st != 0 and not (not check and st == 4):
        _check(st, "expm_apply_laplacian2d")
    return info


def expm_apply_batched(plan: Plan, As, Vs, Ys, prec=EXPM_FP64, t=1.0, shift_c=0.0, stream=None, tol=None,
                       max_refine=None, growth_max=None, check=True):
    """Y_i = e^c R_n(tA_i - cI) V_i for lists of device tensors (see include/expm.h).
    Returns the list of per-instance expm_info."""
    cnt = len(As)
    n_arr = (ctypes.c_int * cnt)(*[int(a.shape[0]) for a in As])
    k_arr = (ctypes.c_int * cnt)(*[int(v.shape[1]) if len(v.shape) == 2 else 1 for v in Vs])
    a_arr = (ctypes.c_void_p * cnt)(*[_ptr(a) for a in As])
    v_arr = (ctypes.c_void_p * cnt)(*[_ptr(v) for v in Vs])
    y_arr = (ctypes.c_void_p * cnt)(*[_ptr(y) for y in Ys])
    if stream is None:
        stream = _default_stream(*As[:1])
    o = make_opts(prec, t, shift_c, stream, tol, max_refine, growth_max)
    infos = (expm_info * max(cnt, 1))()
    st = lib.expm_apply_batched(plan.handle, cnt, n_arr, a_arr, int(_is_complex(As[0])) if cnt else 0, v_arr, k_arr,
                                int(_is_complex(Vs[0])) if cnt else 0, y_arr, ctypes.byref(o), infos)
    if check or st not in (3, 4):
        _check(st, "expm_apply_batched")
    return list(infos)[:cnt]


def expm_apply_tridiag(plan: Plan, d, e, V, Y, prec=EXPM_FP64, t=1.0, shift_c=0.0, stream=None, tol=None,
                       max_refine=None, flags=0, want_info=True, check=True):
    """Y = e^c R_n(tT - cI) V for the Hermitian tridiagonal T = (d, e); see include/expm.h.

    Returns the ``expm_info`` (or None with ``want_info=False``, which keeps the
    EXPM_MIXED_FP32 path asynchronous).  With ``check=False`` EXPM_ENOCONV is left in
    ``info.status_worst`` instead of raising."""
    N = int(d.shape[0])
    r = int(V.shape[1]) if len(V.shape) == 2 else 1
    if stream is None:
        stream = _default_stream(d, e, V, Y)
    o = make_opts(prec, t, shift_c, stream, tol, max_refine)
    o.flags = int(flags)
    info = expm_info() if want_info else None
    st = lib.expm_apply_tridiag(plan.handle, N, _ptr(d), _ptr(e), int(_is_complex(e)), _ptr(V), r,
                                int(_is_complex(V)), _ptr(Y), ctypes.byref(o),
                                ctypes.byref(info) if info is not None else None)
    if st != 0 and not (not check and st == 4):
        _check(st, "expm_apply_tridiag")
    return info


class BatchGraph:
    """A captured batched evaluation (expm_batched_capture): replay() runs the whole batch
    with one graph launch over the same tensors.  scheme=-1 autotunes the bucket scheme."""

    def __init__(self, plan: Plan, As, Vs, Ys, prec=EXPM_FP64, t=1.0, shift_c=0.0, tol=None, max_refine=None,
                 growth_max=None, scheme=-1):
        cnt = len(As)
        n_arr = (ctypes.c_int * cnt)(*[int(a.shape[0]) for a in As])
        k_arr = (ctypes.c_int * cnt)(*[int(v.shape[1]) if len(v.shape) == 2 else 1 for v in Vs])
        a_arr = (ctypes.c_void_p * cnt)(*[_ptr(a) for a in As])
        v_arr = (ctypes.c_void_p * cnt)(*[_ptr(v) for v in Vs])
        y_arr = (ctypes.c_void_p * cnt)(*[_ptr(y) for y in Ys])
        o = make_opts(prec, t, shift_c, None, tol, max_refine, growth_max)
        self._h = ctypes.c_void_p()
        self.count = cnt
        self._keep = (As, Vs, Ys, plan)        # the graph reads and writes these tensors
        _check(lib.expm_batched_capture(plan.handle, cnt, n_arr, a_arr, int(_is_complex(As[0])), v_arr, k_arr,
                                        int(_is_complex(Vs[0])), y_arr, ctypes.byref(o), int(scheme),
                                        ctypes.byref(self._h)), "expm_batched_capture")

    def replay(self, stream=None, want_info=False, check=True):
        if stream is None:
            stream = _default_stream(*self._keep[0][:1])
        infos = (expm_info * self.count)() if want_info else None
        st = lib.expm_batched_replay(self._h, stream, infos)
        if st != 0 and not (not check and st in (3, 4)):
            _check(st, "expm_batched_replay")
        return list(infos) if want_info else None

    def info(self) -> dict:
        sc, groups, nbytes = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        ms = (ctypes.c_double * 3)()
        _check(lib.expm_batched_graph_info(self._h, ctypes.byref(sc), ctypes.byref(groups), ctypes.byref(nbytes), ms),
               "expm_batched_graph_info")
        return {"scheme": sc.value, "launch_groups": groups.value, "device_bytes": nbytes.value,
                "ms_per_scheme": list(ms)}

    def buckets(self) -> list:
        """Per launch group of the graph: padded order, instances, the trailing-update tile
        shape in use (0: 128 x 64, 1: 64 x 64) and the factorization ms timed with each."""
        cnt = lib.expm_batched_graph_buckets(self._h, 0, None, None, None, None, None)
        if cnt < 0:
            raise RuntimeError("expm_batched_graph_buckets: no graph")
        cint, cdbl = ctypes.c_int * max(cnt, 1), ctypes.c_double * max(cnt, 1)
        order, ninst, tile, m0, m1 = cint(), cint(), cint(), cdbl(), cdbl()
        lib.expm_batched_graph_buckets(self._h, cnt, order, ninst, tile, m0, m1)
        return [{"order": order[j], "ninst": ninst[j], "tile": tile[j], "ms_tile": (m0[j], m1[j])}
                for j in range(cnt)]

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib.expm_batched_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Queue:
    """Device-fed work queue of small dense evaluations (expm_queue_*): a persistent
    kernel evaluates each submitted request (n <= 64) as it is published; poll() returns
    None while pending, else (status, info)."""

    def __init__(self, plan: "Plan", a_is_complex=False, k=1, v_is_complex=False, prec=EXPM_FP64, tol=None,
                 max_refine=None, growth_max=None, capacity=256, max_clusters=0, idle_ms=1000.0):
        o = make_opts(prec, tol=tol, max_refine=max_refine, growth_max=growth_max)
        self._h = ctypes.c_void_p()
        _check(lib.expm_queue_create(plan.handle, int(bool(a_is_complex)), int(k), int(bool(v_is_complex)),
                                     ctypes.byref(o), int(capacity), int(max_clusters), float(idle_ms),
                                     ctypes.byref(self._h)), "expm_queue_create")
        self.k = int(k)

    def submit(self, A, V, Y, t=1.0, shift_c=0.0):
        """Returns the ticket, or None when the ring is full (EXPM_EAGAIN)."""
        n = int(A.shape[0])
        tk = ctypes.c_uint64()
        st = lib.expm_queue_submit(self._h, n, _ptr(A), n, _ptr(V), self.k, _ptr(Y), self.k, float(t), float(shift_c),
                                   ctypes.byref(tk))
        if st == 6:                       # EXPM_EAGAIN
            return None
        _check(st, "expm_queue_submit")
        return int(tk.value)

    def poll(self, ticket: int):
        info = expm_info()
        st = lib.expm_queue_poll(self._h, int(ticket), ctypes.byref(info))
        if st == 6:                       # EXPM_EAGAIN: pending
            return None
        if st not in (0, 3, 4):           # OK, EGROWTH, ENOCONV carry a result
            _check(st, "expm_queue_poll")
        return st, info

    def state(self) -> dict:
        run, last, launches, clusters = ctypes.c_int(), ctypes.c_int(), ctypes.c_uint64(), ctypes.c_int()
        _check(lib.expm_queue_state(self._h, ctypes.byref(run), ctypes.byref(last), ctypes.byref(launches),
                                    ctypes.byref(clusters)), "expm_queue_state")
        return {"running": bool(run.value), "last_exit": last.value, "launches": int(launches.value),
                "clusters": clusters.value}

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib.expm_queue_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owns an ``expm_server``: continuous-batching exp(tA)V requests (include/expm.h)."""

    def __init__(self, hbm_budget_bytes: int, max_inflight: int = 4):
        self._h = ctypes.c_void_p()
        _check(lib.expm_server_create(int(hbm_budget_bytes), int(max_inflight), ctypes.byref(self._h)),
               "expm_server_create")
        self._keep = {}

    def register_tridiag(self, d, e) -> int:
        desc = expm_op_desc(EXPM_OP_TRIDIAG, int(d.shape[0]), _ptr(d), _ptr(e), int(_is_complex(e)), None, 0, 0)
        oid = ctypes.c_uint64()
        _check(lib.expm_server_register_op(self._h, ctypes.byref(desc), ctypes.byref(oid)), "expm_server_register_op")
        return int(oid.value)

    def register_dense(self, A) -> int:
        n = int(A.shape[0])
        desc = expm_op_desc(EXPM_OP_DENSE, n, None, None, 0, _ptr(A), n, int(_is_complex(A)))
        oid = ctypes.c_uint64()
        _check(lib.expm_server_register_op(self._h, ctypes.byref(desc), ctypes.byref(oid)), "expm_server_register_op")
        return int(oid.value)

    def submit(self, op_id: int, plan: "Plan", V, Y, prec=EXPM_FP64, t=1.0, shift_c=0.0, tol=None,
               max_refine=None, flags=0) -> int:
        """Queue a request; V and Y must stay alive until poll() reports it finished."""
        k = int(V.shape[1]) if len(V.shape) == 2 else 1
        o = make_opts(prec, t, shift_c, None, tol, max_refine)
        o.flags = int(flags)
        tk = ctypes.c_uint64()
        _check(lib.expm_server_submit(self._h, int(op_id), plan.handle, _ptr(V), k, int(_is_complex(V)), _ptr(Y),
                                      ctypes.byref(o), ctypes.byref(tk)), "expm_server_submit")
        self._keep[int(tk.value)] = (V, Y, plan)
        return int(tk.value)

    def set_queue_limit(self, max_queue: int) -> None:
        _check(lib.expm_server_set_queue_limit(self._h, int(max_queue)), "expm_server_set_queue_limit")

    def poll(self, ticket: int):
        """None while pending, else (status, expm_info, timestamps[4])."""
        info = expm_info()
        ts = (ctypes.c_double * 4)()
        st = lib.expm_server_poll(self._h, int(ticket), ctypes.byref(info), ts)
        if st == 6:                 # EXPM_EAGAIN: pending
            return None
        self._keep.pop(int(ticket), None)
        return st, info, list(ts)

    def close(self) -> None:
        if self._h:
            lib.expm_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
