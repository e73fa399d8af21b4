"""ctypes binding of libhz.so (include/hz.h).  Argument marshalling only:
every step of the solver runs in the CUDA library.

Device buffers may be passed as any object with ``data_ptr()`` (a torch
tensor on the problem's device, float64 or complex128, contiguous) or as a
raw integer address.  Streams may be a ``torch.cuda.Stream`` or an integer
cudaStream_t (``None`` = legacy default stream).
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libhz.so")

HZ_OK, HZ_ERR_INVALID_ARG, HZ_ERR_OOM, HZ_ERR_CUDA, HZ_ERR_NOT_CONVERGED = 0, 1, 2, 3, 4
HZ_ERR_DIVERGED, HZ_ERR_TIMEOUT, HZ_ERR_BUSY, HZ_ERR_NOT_FOUND, HZ_ERR_INTERNAL, HZ_ERR_UNSUPPORTED = 5, 6, 7, 8, 9, 10
HZ_FP64, HZ_FP32_REFINE, HZ_FP16_TRIAL, HZ_BF16_TRIAL = 0, 1, 2, 3
HZ_OUTER_GMRES, HZ_OUTER_PLAIN, HZ_OUTER_RGMRES = 0, 1, 2
HZ_REFINE_DEFECT, HZ_REFINE_FGMRES = 0, 1
HZ_WAVE_SPEED, HZ_OMEGA, HZ_SOURCE, HZ_BOUNDARY, HZ_TRANSMISSION, HZ_NODE_COORDS = 0, 1, 2, 3, 4, 5

STATUS_NAMES = {0: "HZ_OK", 1: "HZ_ERR_INVALID_ARG", 2: "HZ_ERR_OOM", 3: "HZ_ERR_CUDA", 4: "HZ_ERR_NOT_CONVERGED",
                5: "HZ_ERR_DIVERGED", 6: "HZ_ERR_TIMEOUT", 7: "HZ_ERR_BUSY", 8: "HZ_ERR_NOT_FOUND",
                9: "HZ_ERR_INTERNAL", 10: "HZ_ERR_UNSUPPORTED"}


class HzError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class hz_solve_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("tol", C.c_double), ("max_sweeps", C.c_int32), ("outer", C.c_int32),
                ("gmres_restart", C.c_int32), ("wh_iters", C.c_int32), ("wh_tol", C.c_double),
                ("nt_override", C.c_int32), ("cfl", C.c_double), ("inner_tol", C.c_double),
                ("max_refine", C.c_int32), ("autotune", C.c_int32), ("wh_adaptive", C.c_int32),
                ("pack", C.c_int32), ("graphs", C.c_int32), ("gs_passes", C.c_int32),
                ("wh_warm", C.c_int32), ("refine", C.c_int32), ("refine_restart", C.c_int32)]


class hz_solve_report(C.Structure):
    _fields_ = [("sweeps", C.c_int32), ("refinements", C.c_int32), ("nt", C.c_int32), ("wh_iters_max", C.c_int32),
                ("rel_residual", C.c_double), ("seconds", C.c_double), ("dof_updates", C.c_int64),
                ("gmres_iters", C.c_int32), ("sweep_variant", C.c_int32), ("sweep_shape", C.c_int32),
                ("sweep_seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def library_path():
    return _LIB_PATH


def load():
    """Loads libhz.so; raises ImportError if the CUDA library was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"CUDA library not built: {_LIB_PATH} is missing (run __graft_entry__.build())")
    lib = C.CDLL(_LIB_PATH)
    vp, i32, i64, u64, d, dp = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double, C.POINTER(C.c_double)
    sigs = {
        "hz_default_opts": (None, [C.POINTER(hz_solve_opts)]),
        "hz_last_error": (i32, [C.c_char_p, C.c_size_t]),
        "hz_kernel_launches": (i32, [C.POINTER(u64)]),
        "hz_fma_peak": (i32, [i32, i32, dp, dp]),
        "hz_mesh_create": (i32, [d, d, d, d, i32, i32, i32, i32, i32, C.POINTER(vp)]),
        "hz_mesh_num_nodes": (i32, [vp, C.POINTER(i64)]),
        "hz_mesh_node_coords": (i32, [vp, dp]),
        "hz_mesh_destroy": (None, [vp]),
        "hz_problem_create": (i32, [vp, i32, C.POINTER(vp)]),
        "hz_problem_set": (i32, [vp, i32, dp, i64]),
        "hz_problem_set_device": (i32, [vp, i32, vp, i64, vp]),
        "hz_problem_destroy": (None, [vp]),
        "hz_problem_nt": (i32, [vp, d, C.POINTER(i32)]),
        "hz_solve": (i32, [vp, C.POINTER(hz_solve_opts), dp, C.POINTER(hz_solve_report)]),
        "hz_solve_device": (i32, [vp, C.POINTER(hz_solve_opts), vp, C.POINTER(hz_solve_report), vp]),
        "hz_solve_batch": (i32, [C.POINTER(vp), i32, C.POINTER(hz_solve_opts), i32, C.POINTER(dp),
                                 C.POINTER(hz_solve_report), C.POINTER(i32)]),
        "hz_lambda_size": (i32, [vp, C.POINTER(i64)]),
        "hz_prepare": (i32, [vp, i32, vp]),
        "hz_sweep": (i32, [vp, i32, i32, i32, d, vp, vp, vp, vp, vp]),
        "hz_sweep_from": (i32, [vp, i32, i32, i32, d, vp, vp, vp, vp, vp, vp]),
        "hz_sweep_rect": (i32, [vp, i32, i32, i32, d, i32, i32, i32, i32, vp, vp, vp, vp, vp]),
        "hz_lambda_gather": (i32, [vp, vp, i32, vp, vp, vp]),
        "hz_lambda_scatter": (i32, [vp, vp, i32, vp, vp, vp]),
        "hz_sweep_packed": (i32, [C.POINTER(vp), i32, C.POINTER(i32), i32, C.POINTER(vp), C.POINTER(vp),
                                  C.POINTER(vp), C.POINTER(vp), vp]),
        "hz_rhs": (i32, [vp, vp, vp]),
        "hz_residual": (i32, [vp, vp, vp, vp, vp, vp]),
        "hz_assemble_add": (i32, [vp, vp, vp, vp]),
        "hz_residual_noalloc": (i32, [vp, d, vp, vp, vp, vp, vp, vp]),
        "hz_server_create": (i32, [i32, u64, C.POINTER(vp)]),
        "hz_server_submit": (i32, [vp, vp, C.POINTER(hz_solve_opts), C.POINTER(u64)]),
        "hz_server_poll": (i32, [vp, u64, i32, dp, C.POINTER(hz_solve_report), C.POINTER(i32)]),
        "hz_server_stats": (i32, [vp, dp, dp, dp, C.POINTER(u64)]),
        "hz_server_destroy": (None, [vp]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_names():
    """Names of the C functions this binding expects libhz.so to export."""
    return ["hz_default_opts", "hz_last_error", "hz_kernel_launches", "hz_mesh_create", "hz_mesh_num_nodes", "hz_mesh_node_coords",
            "hz_mesh_destroy", "hz_problem_create", "hz_problem_set", "hz_problem_set_device", "hz_problem_destroy",
            "hz_problem_nt", "hz_solve", "hz_solve_device", "hz_solve_batch", "hz_lambda_size", "hz_prepare", "hz_sweep", "hz_sweep_from",
            "hz_sweep_rect", "hz_lambda_gather", "hz_lambda_scatter",
            "hz_sweep_packed", "hz_rhs",
            "hz_residual", "hz_residual_noalloc", "hz_fma_peak", "hz_assemble_add", "hz_server_create", "hz_server_submit", "hz_server_poll",
            "hz_server_stats", "hz_server_destroy"]


def hz_last_error():
    buf = C.create_string_buffer(1024)
    load().hz_last_error(buf, len(buf))
    return buf.value.decode(errors="replace")


def hz_fma_peak(precision, iters):
    """Measured FMA rate of the current device: (TFLOP/s, ms of the timed launch)."""
    tf, ms = C.c_double(), C.c_double()
    _check(load().hz_fma_peak(precision, iters, C.byref(tf), C.byref(ms)))
    return tf.value, ms.value


def hz_kernel_launches():
    n = C.c_uint64()
    load().hz_kernel_launches(C.byref(n))
    return n.value


def _check(status, allow=(HZ_OK,)):
    if status not in allow:
        raise HzError(status, hz_last_error())
    return status


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return C.c_void_p(x)
    if hasattr(x, "data_ptr"):
        if hasattr(x, "is_contiguous") and not x.is_contiguous():
            raise ValueError("device buffer must be contiguous")
        return C.c_void_p(x.data_ptr())
    raise TypeError(f"cannot pass {type(x)} as a device pointer")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return C.c_void_p(s)
    return C.c_void_p(s.cuda_stream)


def _host_f64(a, n_values):
    arr = np.ascontiguousarray(np.asarray(a))
    if np.iscomplexobj(arr):
        arr = np.ascontiguousarray(arr.astype(np.complex128)).view(np.float64)
    else:
        arr = np.ascontiguousarray(arr, dtype=np.float64)
    return arr


# ------------------------------------------------------------------ API --
def hz_default_opts(**overrides):
    o = hz_solve_opts()
    load().hz_default_opts(C.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def hz_mesh_create(x0, x1, y0, y1, nx, ny, degree, sub_nx, sub_ny):
    h = C.c_void_p()
    _check(load().hz_mesh_create(x0, x1, y0, y1, nx, ny, degree, sub_nx, sub_ny, C.byref(h)))
    return h


def hz_mesh_num_nodes(mesh):
    n = C.c_int64()
    _check(load().hz_mesh_num_nodes(mesh, C.byref(n)))
    return n.value


def hz_mesh_node_coords(mesh):
    n = hz_mesh_num_nodes(mesh)
    xy = np.empty((n, 2), np.float64)
    _check(load().hz_mesh_node_coords(mesh, xy.ctypes.data_as(C.POINTER(C.c_double))))
    return xy


def hz_mesh_destroy(mesh):
    load().hz_mesh_destroy(mesh)


def hz_problem_create(mesh, device=0):
    h = C.c_void_p()
    _check(load().hz_problem_create(mesh, device, C.byref(h)))
    return h


def hz_problem_set(pr, field, data):
    """data: numpy array (real for HZ_WAVE_SPEED / HZ_OMEGA / HZ_TRANSMISSION, complex for
    HZ_SOURCE / HZ_BOUNDARY; HZ_NODE_COORDS: real (n, 2) or 2n values x, y per node)."""
    arr = np.atleast_1d(np.asarray(data))
    if field in (HZ_SOURCE, HZ_BOUNDARY):
        count = arr.size
        buf = np.ascontiguousarray(arr.astype(np.complex128).ravel()).view(np.float64)
    else:
        count = arr.size
        buf = np.ascontiguousarray(arr.astype(np.float64).ravel())
    _check(load().hz_problem_set(pr, field, buf.ctypes.data_as(C.POINTER(C.c_double)), count))


def hz_problem_set_device(pr, field, tensor, count, stream=None):
    _check(load().hz_problem_set_device(pr, field, _ptr(tensor), count, _stream(stream)))


def hz_problem_destroy(pr):
    load().hz_problem_destroy(pr)


def hz_problem_nt(pr, cfl=0.9):
    nt = C.c_int32()
    _check(load().hz_problem_nt(pr, cfl, C.byref(nt)))
    return nt.value


def hz_solve(pr, opts=None, n=None):
    """Returns (status, u complex ndarray (n,), report dict); raises on hard errors."""
    if opts is None:
        opts = hz_default_opts()
    if n is None:
        raise ValueError("n (number of nodes) is required")
    u = np.empty(2 * n, np.float64)
    rep = hz_solve_report()
    st = load().hz_solve(pr, C.byref(opts), u.ctypes.data_as(C.POINTER(C.c_double)), C.byref(rep))
    _check(st, (HZ_OK, HZ_ERR_NOT_CONVERGED))
    return st, u.view(np.complex128), rep.as_dict()


def hz_solve_device(pr, opts, u_dev, stream=None):
    rep = hz_solve_report()
    st = load().hz_solve_device(pr, C.byref(opts), _ptr(u_dev), C.byref(rep), _stream(stream))
    _check(st, (HZ_OK, HZ_ERR_NOT_CONVERGED))
    return st, rep.as_dict()


def hz_solve_batch(problems, ns, opts=None, max_concurrent=0, want_u=True):
    """problems: list of handles; ns: their node counts.  Returns (status,
    list of per-problem statuses, list of u arrays or None, list of report dicts)."""
    if opts is None:
        opts = hz_default_opts()
    k = len(problems)
    arr = (C.c_void_p * k)(*[p.value if isinstance(p, C.c_void_p) else p for p in problems])
    us = [np.empty(2 * n, np.float64) for n in ns] if want_u else None
    uptr = (C.POINTER(C.c_double) * k)(*[u.ctypes.data_as(C.POINTER(C.c_double)) for u in us]) if want_u else None
    reps = (hz_solve_report * k)()
    sts = (C.c_int32 * k)()
    st = load().hz_solve_batch(arr, k, C.byref(opts), max_concurrent, uptr, reps, sts)
    _check(st, (HZ_OK, HZ_ERR_NOT_CONVERGED))
    return st, list(sts), ([u.view(np.complex128) for u in us] if want_u else None), [r.as_dict() for r in reps]


def hz_lambda_size(pr):
    n = C.c_int64()
    _check(load().hz_lambda_size(pr, C.byref(n)))
    return n.value


def hz_prepare(pr, nt, stream=None):
    _check(load().hz_prepare(pr, nt, _stream(stream)))


def hz_sweep(pr, precision, nt, wh_iters, wh_tol, lam_in, lam_out, rhs=None, u_sub=None, stream=None):
    _check(load().hz_sweep(pr, precision, nt, wh_iters, wh_tol, _ptr(lam_in), _ptr(lam_out), _ptr(rhs), _ptr(u_sub),
                           _stream(stream)))


def hz_sweep_from(pr, precision, nt, wh_iters, wh_tol, lam_in, lam_out, rhs, u0, u_sub=None, stream=None):
    _check(load().hz_sweep_from(pr, precision, nt, wh_iters, wh_tol, _ptr(lam_in), _ptr(lam_out), _ptr(rhs), _ptr(u0),
                                _ptr(u_sub), _stream(stream)))


def hz_sweep_rect(pr, precision, nt, wh_iters, wh_tol, rect, lam_in, lam_out, rhs=None, u_sub=None, stream=None):
    """Rank-local sweep of the subdomain rectangle rect = (sx0, sy0, sw, sh)."""
    sx0, sy0, sw, sh = (int(v) for v in rect)
    _check(load().hz_sweep_rect(pr, precision, nt, wh_iters, wh_tol, sx0, sy0, sw, sh, _ptr(lam_in), _ptr(lam_out),
                                _ptr(rhs), _ptr(u_sub), _stream(stream)))


def hz_lambda_gather(pr, slots, count, lam, buf, stream=None):
    """buf[k] = lambda slot slots[k] = (l, e) (device int32 pairs)."""
    _check(load().hz_lambda_gather(pr, _ptr(slots), int(count), _ptr(lam), _ptr(buf), _stream(stream)))


def hz_lambda_scatter(pr, slots, count, buf, lam, stream=None):
    """lambda slot slots[k] = (l, e) = buf[k]."""
    _check(load().hz_lambda_scatter(pr, _ptr(slots), int(count), _ptr(buf), _ptr(lam), _stream(stream)))


def hz_sweep_packed(problems, nts, wh_iters, lam_in, lam_out, rhs=None, u_sub=None, stream=None):
    """One packed FP32 sweep of several problems (lists of per-problem device
    buffers; rhs / u_sub entries may be None, or the whole list None)."""
    k = len(problems)

    def arr(xs):
        if xs is None:
            return None
        return (C.c_void_p * k)(*[(_ptr(x).value if x is not None else None) for x in xs])

    prs = (C.c_void_p * k)(*[p.value if isinstance(p, C.c_void_p) else p for p in problems])
    ntv = (C.c_int32 * k)(*nts)
    _check(load().hz_sweep_packed(prs, k, ntv, wh_iters, arr(lam_in), arr(lam_out), arr(rhs), arr(u_sub),
                                  _stream(stream)))


def hz_rhs(pr, b, stream=None):
    _check(load().hz_rhs(pr, _ptr(b), _stream(stream)))


def hz_residual(pr, b, u, r, norms2=None, stream=None):
    _check(load().hz_residual(pr, _ptr(b), _ptr(u), _ptr(r), _ptr(norms2), _stream(stream)))


def hz_residual_noalloc(mesh, omega, c, b, u, r, norms2, stream=None):
    """Residual without device allocation; every array is the caller's."""
    _check(load().hz_residual_noalloc(mesh, omega, _ptr(c), _ptr(b), _ptr(u), _ptr(r), _ptr(norms2),
                                      _stream(stream)))


def hz_assemble_add(pr, u_sub, u, stream=None):
    _check(load().hz_assemble_add(pr, _ptr(u_sub), _ptr(u), _stream(stream)))


def hz_server_create(device=0, hbm_budget_bytes=150 << 30):
    h = C.c_void_p()
    _check(load().hz_server_create(device, hbm_budget_bytes, C.byref(h)))
    return h


def hz_server_submit(srv, pr, opts=None):
    if opts is None:
        opts = hz_default_opts()
    t = C.c_uint64()
    _check(load().hz_server_submit(srv, pr, C.byref(opts), C.byref(t)))
    return t.value


def hz_server_poll(srv, ticket, timeout_ms=-1, n=None):
    """Returns (done, status, u or None, report dict)."""
    u = np.empty(2 * n, np.float64) if n else None
    rep = hz_solve_report()
    done = C.c_int32()
    up = u.ctypes.data_as(C.POINTER(C.c_double)) if u is not None else None
    st = load().hz_server_poll(srv, ticket, timeout_ms, up, C.byref(rep), C.byref(done))
    if not done.value:
        _check(st, (HZ_OK, HZ_ERR_TIMEOUT))
        return False, st, None, None
    _check(st, (HZ_OK, HZ_ERR_NOT_CONVERGED))
    return True, st, (u.view(np.complex128) if u is not None else None), rep.as_dict()


def hz_server_stats(srv):
    p50, p99, sps = C.c_double(), C.c_double(), C.c_double()
    mem = C.c_uint64()
    _check(load().hz_server_stats(srv, C.byref(p50), C.byref(p99), C.byref(sps), C.byref(mem)))
    return {"p50_ms": p50.value, "p99_ms": p99.value, "solves_per_s": sps.value, "hbm_in_use": mem.value}


def hz_server_destroy(srv):
    load().hz_server_destroy(srv)
