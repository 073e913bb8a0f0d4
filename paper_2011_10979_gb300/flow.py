"""Thin Python binding of the C ABI in include/tvl1flow.h (libtvl1flow.so).

Argument marshalling only: every step of the solver runs in the library's CUDA kernels.  Device
memory and streams come from PyTorch (tensors on a CUDA device, the current torch stream).  The
functions keep the C names.  There is no fallback: if the library is missing or fails to load,
every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtvl1flow.so")
_lib = None

OF_OK, OF_EINVAL, OF_ENOMEM, OF_ECUDA, OF_ETIMEOUT, OF_ENUMERIC, OF_EBUSY = range(7)
OF_PADMM_I, OF_PADMM_II, OF_PDR, OF_CP = 0, 1, 2, 3
OF_PREC_FP32, OF_PREC_FP16, OF_PREC_BF16 = 0, 1, 2
OF_ENGINE_FUSED, OF_ENGINE_PLAIN, OF_ENGINE_STREAM, OF_ENGINE_RESIDENT, OF_ENGINE_PERSISTENT = 0, 1, 2, 3, 4

EXPORTS = ("of_default_params", "of_create", "of_destroy", "of_last_error", "of_arena_bytes",
           "of_solve_kernel_count", "of_rows_per_warp", "of_resident_clusters", "of_persistent_selftest", "of_l2_bandwidth", "of_solve",
           "of_solve_host", "of_solve_batch", "of_pyr_down", "of_upsample", "of_derivatives",
           "of_warp_linearise", "of_admm_iterate", "of_admm_iterate_noalloc", "of_pdr_iterate", "of_cp_iterate",
           "of_fields_bytes", "of_energy",
           "of_server_start", "of_server_submit", "of_server_poll", "of_server_stop")


class OfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("status %d: %s" % (status, msg))
        self.status = status


class of_params(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("lambda_", ctypes.c_float), ("beta", ctypes.c_float),
                ("c", ctypes.c_float), ("a", ctypes.c_float), ("a_tilde", ctypes.c_float),
                ("r", ctypes.c_float), ("rho", ctypes.c_float), ("sigma", ctypes.c_float),
                ("tau", ctypes.c_float), ("gs_sweeps", ctypes.c_int), ("eta", ctypes.c_float),
                ("levels", ctypes.c_int), ("warps", ctypes.c_int), ("iters", ctypes.c_int),
                ("tol", ctypes.c_double), ("precision", ctypes.c_int), ("fp32_last_warp", ctypes.c_int),
                ("fp32_flow", ctypes.c_int),
                ("engine", ctypes.c_int), ("out_level", ctypes.c_int), ("cp_tau", ctypes.c_float),
                ("cp_sigma", ctypes.c_float), ("a_tilde_mode", ctypes.c_int), ("rows_per_warp", ctypes.c_int),
                ("c_adapt_iters", ctypes.c_int)]


class of_stats(ctypes.Structure):
    _fields_ = [("iters_run", ctypes.c_longlong), ("residual", ctypes.c_double), ("energy", ctypes.c_double),
                ("dual_value", ctypes.c_double), ("ms", ctypes.c_float), ("c", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_FP = ctypes.POINTER(ctypes.c_float)


class of_fields(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("w", "u", "v", "p1", "p2", "q11", "q12", "q21", "q22", "s",
                                               "wb", "ub", "vb")]


def lib():
    """Loads libtvl1flow.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libtvl1flow.so is not built; run paper_2011_10979_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, f, sz, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_size_t, ctypes.c_double
        P = ctypes.POINTER
        sig = {
            "of_default_params": (None, [P(of_params)]),
            "of_create": (i, [P(vp), i, sz]),
            "of_destroy": (None, [vp]),
            "of_last_error": (ctypes.c_char_p, [vp]),
            "of_arena_bytes": (sz, [i, i, P(of_params)]),
            "of_solve_kernel_count": (ctypes.c_longlong, [vp, i, i, P(of_params)]),
            "of_rows_per_warp": (i, [vp, i, P(i), P(i), P(of_params), P(i)]),
            "of_resident_clusters": (i, [P(i), P(i)]),
            "of_persistent_selftest": (i, [i, i, i, i, d, P(i), P(i)]),
            "of_l2_bandwidth": (i, [sz, i, P(d)]),
            "of_solve": (i, [vp, vp, vp, i, i, i, P(of_params), vp, vp, vp, i, vp, P(of_stats)]),
            "of_solve_host": (i, [vp, vp, vp, i, i, P(of_params), vp, vp, vp, vp, P(of_stats)]),
            "of_solve_batch": (i, [vp, i, P(vp), P(vp), P(i), P(i), P(i), P(of_params), P(vp), P(vp), P(vp),
                                   P(i), vp, P(of_stats)]),
            "of_pyr_down": (i, [vp, i, i, i, vp, i, i, i, f, vp, vp]),
            "of_upsample": (i, [vp, i, i, i, vp, i, i, i, f, vp]),
            "of_derivatives": (i, [vp, i, i, i, vp, vp, vp]),
            "of_warp_linearise": (i, [vp, vp, vp, vp, vp, vp, i, i, i, f, vp, vp, vp, vp, vp]),
            "of_admm_iterate": (i, [of_fields, vp, vp, vp, i, i, i, f, P(of_params), i, vp, P(d), vp]),
            "of_admm_iterate_noalloc": (i, [of_fields, vp, vp, vp, i, i, i, f, P(of_params), i, P(d), vp]),
            "of_pdr_iterate": (i, [of_fields, vp, vp, vp, i, i, i, P(of_params), i, vp, P(d), vp]),
            "of_cp_iterate": (i, [of_fields, vp, vp, vp, i, i, i, P(of_params), i, vp, P(d), vp]),
            "of_fields_bytes": (sz, [i, i]),
            "of_energy": (i, [vp, vp, vp, vp, vp, vp, vp, i, i, i, f, f, P(d), P(d), vp]),
            "of_server_start": (i, [vp, P(of_params), sz, i]),
            "of_server_submit": (i, [vp, vp, vp, i, i, P(ctypes.c_uint64)]),
            "of_server_poll": (i, [vp, ctypes.c_uint64, vp, vp, P(of_stats), P(i)]),
            "of_server_stop": (i, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status, ctx=None):
    if status != OF_OK:
        raise OfError(status, lib().of_last_error(ctx).decode())


def default_params(**kw) -> of_params:
    p = of_params()
    lib().of_default_params(ctypes.byref(p))
    names = {n for n, _ in of_params._fields_}
    for k, v in kw.items():
        k = "lambda_" if k in ("lam", "lambda") else k
        if k not in names:
            raise TypeError("unknown solver parameter %r" % k)
        setattr(p, k, v)
    return p


def out_size(H, W, params):
    """Output size at params.out_level (1 x 1 when out_level is out of range: the C layer
    rejects such parameters before touching the outputs)."""
    sz = level_sizes(H, W, params.eta, max(1, params.levels))
    return sz[params.out_level] if 0 <= params.out_level < len(sz) else (1, 1)


def level_sizes(H, W, eta, levels):
    import math
    hs, ws = [H], [W]
    for _ in range(1, levels):
        hs.append(max(1, int(math.floor(hs[-1] * eta + 0.5))))
        ws.append(max(1, int(math.floor(ws[-1] * eta + 0.5))))
    return list(zip(hs, ws))


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """Owns an of_ctx (device arena + cached CUDA graphs)."""

    def __init__(self, device: int = 0, hbm_budget: int = 0):
        self.h = ctypes.c_void_p()
        check(lib().of_create(ctypes.byref(self.h), device, hbm_budget))
        self.device = device

    def close(self):
        if self.h:
            lib().of_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def of_solve_kernel_count(ctx: Context, H, W, params: of_params) -> int:
    """Kernel launches in one solve's graph (captures the graph if needed)."""
    n = lib().of_solve_kernel_count(ctx.h, int(H), int(W), ctypes.byref(params))
    if n < 0:
        raise OfError(OF_EINVAL, lib().of_last_error(ctx.h).decode())
    return int(n)


def of_rows_per_warp(ctx: Context, sizes, params: of_params) -> list:
    """Strip height of the streaming ADMM kernel per pyramid level (0 = that level does not run
    on it) for a solve of the pairs of `sizes` [(H, W), ...]; tunes the layout first when
    params.rows_per_warp is -1."""
    n = len(sizes)
    Hs = (ctypes.c_int * n)(*[int(h) for h, _ in sizes])
    Ws = (ctypes.c_int * n)(*[int(w) for _, w in sizes])
    rows = (ctypes.c_int * max(1, params.levels))()
    check(lib().of_rows_per_warp(ctx.h, n, Hs, Ws, ctypes.byref(params), rows), ctx.h)
    return list(rows)[:params.levels]


def of_resident_clusters() -> tuple:
    """(CTAs per cluster, clusters the device runs at once) of the level-resident engine."""
    nc, act = ctypes.c_int(0), ctypes.c_int(0)
    check(lib().of_resident_clusters(ctypes.byref(nc), ctypes.byref(act)))
    return nc.value, act.value


def of_persistent_selftest(H, W, iters, withhold, wait_ms) -> tuple:
    """(timed_out, segments) of the persistent engine's bounded-wait self-test."""
    to, nseg = ctypes.c_int(0), ctypes.c_int(0)
    check(lib().of_persistent_selftest(H, W, iters, withhold, float(wait_ms), ctypes.byref(to), ctypes.byref(nseg)))
    return to.value, nseg.value


def of_l2_bandwidth(nbytes: int, passes: int) -> float:
    """GB/s of the L2-only streaming probe over a working set of `nbytes`."""
    g = ctypes.c_double(0.0)
    check(lib().of_l2_bandwidth(nbytes, passes, ctypes.byref(g)))
    return g.value


def of_solve(ctx: Context, I0, I1, params: of_params, want_w=False, stats=True, stream=None):
    """I0, I1: 2-D float32 CUDA tensors (row pitch = stride(0)).  Returns (u, v, w|None, stats|None)
    at level params.out_level."""
    import torch
    assert I0.is_cuda and I0.dtype == torch.float32 and I0.dim() == 2 and I0.stride(1) == 1
    assert I1.shape == I0.shape and I1.stride() == I0.stride() and I1.dtype == torch.float32
    H, W = I0.shape
    h, w = out_size(H, W, params)
    u = torch.empty((h, w), dtype=torch.float32, device=I0.device)
    v = torch.empty_like(u)
    wo = torch.empty_like(u) if want_w else None
    st = of_stats()
    check(lib().of_solve(ctx.h, _ptr(I0), _ptr(I1), H, W, I0.stride(0), ctypes.byref(params), _ptr(u), _ptr(v),
                         _ptr(wo), w, _stream(stream), ctypes.byref(st) if stats else None), ctx.h)
    return u, v, wo, (st.as_dict() if stats else None)


def of_solve_host(ctx: Context, I0, I1, params: of_params, stats=True, stream=None):
    """I0, I1: C-contiguous float32 numpy arrays on the host.  Returns host (u, v, stats)."""
    import numpy as np
    I0 = np.ascontiguousarray(I0, np.float32)
    I1 = np.ascontiguousarray(I1, np.float32)
    H, W = I0.shape
    h, w = out_size(H, W, params)
    u = np.empty((h, w), np.float32)
    v = np.empty((h, w), np.float32)
    st = of_stats()
    check(lib().of_solve_host(ctx.h, I0.ctypes.data_as(ctypes.c_void_p), I1.ctypes.data_as(ctypes.c_void_p), H, W,
                              ctypes.byref(params), u.ctypes.data_as(ctypes.c_void_p),
                              v.ctypes.data_as(ctypes.c_void_p), None, _stream(stream),
                              ctypes.byref(st) if stats else None), ctx.h)
    return u, v, (st.as_dict() if stats else None)


def of_solve_host_ptrs(ctx: Context, I0_ptr, I1_ptr, H, W, params: of_params, u_ptr, v_ptr, stream=None):
    """Raw-pointer form of of_solve_host (pinned host buffers owned by the caller)."""
    check(lib().of_solve_host(ctx.h, ctypes.c_void_p(I0_ptr), ctypes.c_void_p(I1_ptr), H, W, ctypes.byref(params),
                              ctypes.c_void_p(u_ptr), ctypes.c_void_p(v_ptr), None, _stream(stream), None), ctx.h)


def of_solve_batch(ctx: Context, I0s, I1s, params: of_params, stats=True, stream=None):
    import torch
    n = len(I0s)
    VP = ctypes.c_void_p * n
    IA = ctypes.c_int * n
    us, vs = [], []
    for a in I0s:
        H, W = a.shape
        h, w = out_size(H, W, params)
        us.append(torch.empty((h, w), dtype=torch.float32, device=a.device))
        vs.append(torch.empty((h, w), dtype=torch.float32, device=a.device))
    st = (of_stats * n)()
    check(lib().of_solve_batch(ctx.h, n, VP(*[a.data_ptr() for a in I0s]), VP(*[a.data_ptr() for a in I1s]),
                               IA(*[a.shape[0] for a in I0s]), IA(*[a.shape[1] for a in I0s]),
                               IA(*[a.stride(0) for a in I0s]), ctypes.byref(params), VP(*[x.data_ptr() for x in us]),
                               VP(*[x.data_ptr() for x in vs]), None, IA(*[x.stride(0) for x in us]),
                               _stream(stream), st if stats else None), ctx.h)
    return us, vs, ([s.as_dict() for s in st] if stats else None)


# ---------------------------------------------------------------------- step-level entry points
def of_pyr_down(fine, Hc, Wc, eta, stream=None):
    import torch
    Hf, Wf = fine.shape
    coarse = torch.empty((Hc, Wc), dtype=torch.float32, device=fine.device)
    scratch = torch.empty((2, Hf, fine.stride(0)), dtype=torch.float32, device=fine.device)
    check(lib().of_pyr_down(_ptr(fine), Hf, Wf, fine.stride(0), _ptr(coarse), Hc, Wc, coarse.stride(0), eta,
                            _ptr(scratch), _stream(stream)))
    return coarse


def of_upsample(coarse, Hf, Wf, scale, stream=None):
    import torch
    Hc, Wc = coarse.shape
    fine = torch.empty((Hf, Wf), dtype=torch.float32, device=coarse.device)
    check(lib().of_upsample(_ptr(coarse), Hc, Wc, coarse.stride(0), _ptr(fine), Hf, Wf, fine.stride(0), scale,
                            _stream(stream)))
    return fine


def of_derivatives(I, stream=None):
    import torch
    H, W = I.shape
    Ix, Iy = torch.empty_like(I), torch.empty_like(I)
    check(lib().of_derivatives(_ptr(I), H, W, I.stride(0), _ptr(Ix), _ptr(Iy), _stream(stream)))
    return Ix, Iy


def of_warp_linearise(I0, I1, I1x, I1y, u0, v0, beta, stream=None):
    import torch
    H, W = I0.shape
    Ix, Iy, It = torch.empty_like(I0), torch.empty_like(I0), torch.empty_like(I0)
    ms = torch.zeros(1, dtype=torch.float32, device=I0.device)
    check(lib().of_warp_linearise(_ptr(I0), _ptr(I1), _ptr(I1x), _ptr(I1y), _ptr(u0), _ptr(v0), H, W, I0.stride(0),
                                  beta, _ptr(Ix), _ptr(Iy), _ptr(It), _ptr(ms), _stream(stream)))
    return Ix, Iy, It, ms


def _fields(state: dict) -> of_fields:
    f = of_fields()
    for name, _ in of_fields._fields_:
        t = state.get(name)
        setattr(f, name, None if t is None else t.data_ptr())
    return f


def of_admm_iterate(state: dict, Ix, Iy, It, a_tilde, params: of_params, iters, want_res=True, stream=None):
    """In place on the FP32 CUDA tensors of `state` (keys w u v p1 p2 q11 q12 q21 q22 s)."""
    import torch
    H, W = Ix.shape
    scratch = torch.empty(lib().of_fields_bytes(H, Ix.stride(0)), dtype=torch.uint8, device=Ix.device)
    res = ctypes.c_double(0.0)
    check(lib().of_admm_iterate(_fields(state), _ptr(Ix), _ptr(Iy), _ptr(It), H, W, Ix.stride(0), a_tilde,
                                ctypes.byref(params), iters, _ptr(scratch), ctypes.byref(res) if want_res else None,
                                _stream(stream)))
    return res.value


def of_pdr_iterate(state: dict, Ix, Iy, It, params: of_params, iters, want_res=True, stream=None):
    import torch
    H, W = Ix.shape
    scratch = torch.empty(lib().of_fields_bytes(H, Ix.stride(0)), dtype=torch.uint8, device=Ix.device)
    res = ctypes.c_double(0.0)
    check(lib().of_pdr_iterate(_fields(state), _ptr(Ix), _ptr(Iy), _ptr(It), H, W, Ix.stride(0),
                               ctypes.byref(params), iters, _ptr(scratch), ctypes.byref(res) if want_res else None,
                               _stream(stream)))
    return res.value


def of_cp_iterate(state: dict, Ix, Iy, It, params: of_params, iters, want_res=True, stream=None):
    import torch
    H, W = Ix.shape
    scratch = torch.empty(lib().of_fields_bytes(H, Ix.stride(0)), dtype=torch.uint8, device=Ix.device)
    res = ctypes.c_double(0.0)
    check(lib().of_cp_iterate(_fields(state), _ptr(Ix), _ptr(Iy), _ptr(It), H, W, Ix.stride(0),
                              ctypes.byref(params), iters, _ptr(scratch), ctypes.byref(res) if want_res else None,
                              _stream(stream)))
    return res.value


def of_energy(w, u, v, s, Ix, Iy, It, beta, lam, stream=None):
    H, W = u.shape
    e, d = ctypes.c_double(), ctypes.c_double()
    check(lib().of_energy(_ptr(w), _ptr(u), _ptr(v), _ptr(s), _ptr(Ix), _ptr(Iy), _ptr(It), H, W, u.stride(0), beta,
                          lam, ctypes.byref(e), ctypes.byref(d), _stream(stream)))
    return e.value, d.value


# ---------------------------------------------------------------------- serving loop
def of_server_start(ctx: Context, params: of_params, hbm_budget: int = 0, max_active: int = 8):
    check(lib().of_server_start(ctx.h, ctypes.byref(params), hbm_budget, max_active), ctx.h)


def of_server_submit(ctx: Context, I0, I1) -> int:
    """I0, I1: host float32 arrays (H x W).  Returns the request id."""
    import numpy as np
    I0 = np.ascontiguousarray(I0, np.float32)
    I1 = np.ascontiguousarray(I1, np.float32)
    H, W = I0.shape
    rid = ctypes.c_uint64(0)
    check(lib().of_server_submit(ctx.h, I0.ctypes.data_as(ctypes.c_void_p), I1.ctypes.data_as(ctypes.c_void_p), H, W,
                                 ctypes.byref(rid)), ctx.h)
    return rid.value


def of_server_poll(ctx: Context, rid: int, shape):
    """Returns None while the request runs, else (u, v, latency_ms) as host arrays; raises the
    request's error status if it failed."""
    import numpy as np
    h, w = shape
    u = np.empty((h, w), np.float32)
    v = np.empty((h, w), np.float32)
    st = of_stats()
    done = ctypes.c_int(0)
    check(lib().of_server_poll(ctx.h, ctypes.c_uint64(rid), u.ctypes.data_as(ctypes.c_void_p),
                               v.ctypes.data_as(ctypes.c_void_p), ctypes.byref(st), ctypes.byref(done)), ctx.h)
    return (u, v, st.ms) if done.value else None


def of_server_stop(ctx: Context):
    check(lib().of_server_stop(ctx.h), ctx.h)
