"""FP64 CPU oracle for the TV-L1 optical-flow solvers of Sun, Tai & Yuan (arXiv 2011.10979).

TEST INFRASTRUCTURE ONLY.  This package is the independent reference the CUDA library is
checked against.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product package never does.  The arithmetic lives in
``tvl1_oracle.c`` (plain C, double precision, single thread); this module only builds it with
gcc and marshals numpy arrays through ctypes.

Parity status per function (the pins live in ``tests/test_oracle_*.py``):
  grad / div ............ pinned (exact adjointness, ||grad||^2 <= 8, closed forms)
  proj_p / proj_q / proj_s pinned (projection invariants, brute-force nearest point)
  prox_l1 ............... pinned (brute-force minimisation of the prox objective)
  srbgs ................. pinned (red-black GS property, convergence to a direct sparse solve)
  admm_step ............. pinned (subproblem optimality, special cases, strong duality)
  pdr_step .............. pinned (same minimum as ADMM, dual certificate, SRBGS limit)
  admm_step, per-pixel a~ pinned (s-subproblem solution with the diagonal preconditioner;
                          same certified minimum)
  cp_step (ALG1) ........ pinned (dual step = projection, primal step = prox optimality,
                          same certified minimum as ADMM at a fixed linearisation)
  gauss_smooth .......... pinned (scipy.ndimage.gaussian_filter1d with half-sample reflection,
                          impulse responses at the border and inside)
  downsample / upsample . pinned (that smoothing, then scipy.ndimage.map_coordinates at the
                          pixel centres; constants, ramps, size ratios)
  derivatives ........... pinned (numpy.gradient inside, halved one-sided differences at the border)
  warp_linearise ........ pinned (map_coordinates at the displaced positions; identities)
  solve (schedule) ...... pinned (a 1 x 1 pair solved by hand for every method across levels and
                          warps; a two-level pair equal to the composition of the pinned steps,
                          with planted schedule mistakes shown to fail; out_level = a one-level
                          solve of the downsampled pair; known-flow recovery).  The absolute
                          flow values on the paper's own sequences stay unpinned (the data sets
                          are not available).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tvl1_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_tvl1.so")
_lib = None

METHOD_PADMM_I = 0   # rpADMMI (pADMM when r = 1; Zach-pADMM when beta = 0 and r = 1)
METHOD_PADMM_II = 1  # rpADMMII
METHOD_PDR = 2       # pDR with red-black symmetric Gauss-Seidel
METHOD_CP = 3        # ALG1: the primal-dual method of Chambolle and Pock (Sec. 4)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction) into an in-tree .so."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("lam", ctypes.c_double), ("beta", ctypes.c_double),
                ("c", ctypes.c_double), ("a", ctypes.c_double), ("a_tilde", ctypes.c_double),
                ("r", ctypes.c_double), ("rho", ctypes.c_double), ("sigma", ctypes.c_double),
                ("tau", ctypes.c_double), ("gs_sweeps", ctypes.c_int), ("eta", ctypes.c_double),
                ("levels", ctypes.c_int), ("warps", ctypes.c_int), ("iters", ctypes.c_int),
                ("tol", ctypes.c_double), ("out_level", ctypes.c_int), ("cp_tau", ctypes.c_double),
                ("cp_sigma", ctypes.c_double), ("a_tilde_mode", ctypes.c_int), ("c_adapt_iters", ctypes.c_int)]


class _Stats(ctypes.Structure):
    _fields_ = [("iters_run", ctypes.c_longlong), ("residual", ctypes.c_double),
                ("energy", ctypes.c_double), ("dual_value", ctypes.c_double),
                ("c_final", ctypes.c_double), ("adapt_margin", ctypes.c_double)]


@dataclass
class Params:
    """Solver parameters; defaults are the paper's Sec. 4 settings (pADMM, c = 0.05, a = 8)."""
    method: int = METHOD_PADMM_I
    lam: float = 0.05
    beta: float = 0.05
    c: float = 0.05
    a: float = 8.0
    a_tilde: float = 0.0
    r: float = 1.0
    rho: float = 1.9
    sigma: float = 2.0
    tau: float = 0.4
    gs_sweeps: int = 1
    eta: float = 0.5
    levels: int = 3
    warps: int = 5
    iters: int = 50
    tol: float = 0.0
    out_level: int = 0
    cp_tau: float = 0.1      # ALG1 dual step (Sec. 4)
    cp_sigma: float = 1.25   # ALG1 primal step 1 / (8 cp_tau) (Sec. 4, reading of the step rule)
    a_tilde_mode: int = 0    # 0: a~ = max M_s per warp (Prop. 3.1); 1: per-pixel a~_ij = M_s(ij)
    c_adapt_iters: int = 0   # 0: fixed steps; K: balancing of c (pDR: sigma / tau) in each level's first K iterations

    def _c(self) -> _Params:
        return _Params(self.method, self.lam, self.beta, self.c, self.a, self.a_tilde, self.r,
                       self.rho, self.sigma, self.tau, self.gs_sweeps, self.eta, self.levels,
                       self.warps, self.iters, self.tol, self.out_level, self.cp_tau, self.cp_sigma,
                       self.a_tilde_mode, self.c_adapt_iters)


_D = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        i, d, sz = ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        PP = ctypes.POINTER(_D)
        sig = {
            "orc_grad": (None, [i, i, _D, _D, _D]),
            "orc_div": (None, [i, i, _D, _D, _D]),
            "orc_proj_p": (None, [sz, _D, _D]),
            "orc_proj_q": (None, [sz, _D, _D, _D, _D]),
            "orc_proj_s": (None, [sz, _D, d]),
            "orc_prox_l1": (None, [sz, _D, _D, _D, _D, _D, _D, d, d, d]),
            "orc_srbgs": (None, [i, i, _D, _D, d, i]),
            "orc_level_size": (i, [i, d]),
            "orc_gauss_smooth": (None, [i, i, _D, _D, d]),
            "orc_downsample": (None, [i, i, _D, i, i, _D, d]),
            "orc_upsample": (None, [i, i, _D, i, i, _D, d]),
            "orc_derivatives": (None, [i, i, _D, _D, _D]),
            "orc_warp_linearise": (d, [i, i, _D, _D, _D, _D, _D, _D, d, _D, _D, _D]),
            "orc_energy": (d, [i, i, _D, _D, _D, _D, _D, _D, d, d]),
            "orc_dual_value": (d, [sz, _D, _D]),
            "orc_admm_step_flat": (d, [i, i, PP, _D, _D, _D, d, ctypes.POINTER(_Params)]),
            "orc_pdr_step_flat": (d, [i, i, PP, _D, _D, _D, ctypes.POINTER(_Params)]),
            "orc_cp_step_flat": (d, [i, i, PP, _D, _D, _D, ctypes.POINTER(_Params)]),
            "orc_inner_flat": (ctypes.c_longlong, [i, i, PP, _D, _D, _D, d, ctypes.POINTER(_Params), i, _D]),
            "orc_solve": (i, [i, i, _D, _D, ctypes.POINTER(_Params), _D, _D, _D, ctypes.POINTER(_Stats)]),
            "orc_adapt_rule": (d, [d, d, d]),
            "orc_adapt_residuals_flat": (d, [i, i, PP, PP, _D, _D, d, d, ctypes.POINTER(_Params), _D, _D]),
            "orc_inner_adapt_flat": (ctypes.c_longlong, [i, i, PP, _D, _D, _D, d, ctypes.POINTER(_Params), i, i,
                                                         _D, _D, _D]),
            "orc_pdr_adapt_residuals_flat": (d, [i, i, PP, PP, d, d, ctypes.POINTER(_Params), _D, _D]),
            "orc_inner_adapt_pdr_flat": (ctypes.c_longlong, [i, i, PP, _D, _D, _D, ctypes.POINTER(_Params), i, i,
                                                             _D, _D, _D]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


# ---------------------------------------------------------------------------- operators
def grad(f):
    f = _f64(f)
    H, W = f.shape
    gx, gy = np.empty_like(f), np.empty_like(f)
    lib().orc_grad(H, W, _p(f), _p(gx), _p(gy))
    return gx, gy


def div(px, py):
    px, py = _f64(px), _f64(py)
    H, W = px.shape
    d = np.empty_like(px)
    lib().orc_div(H, W, _p(px), _p(py), _p(d))
    return d


def proj_p(p1, p2):
    p1, p2 = _f64(p1).copy(), _f64(p2).copy()
    lib().orc_proj_p(p1.size, _p(p1), _p(p2))
    return p1, p2


def proj_q(q11, q12, q21, q22):
    q = [_f64(x).copy() for x in (q11, q12, q21, q22)]
    lib().orc_proj_q(q[0].size, *[_p(x) for x in q])
    return tuple(q)


def proj_s(s, lam):
    s = _f64(s).copy()
    lib().orc_proj_s(s.size, _p(s), lam)
    return s


def prox_l1(zw, zu, zv, Ix, Iy, It, beta, lam, sigma):
    z = [_f64(x).copy() for x in (zw, zu, zv)]
    dat = [_f64(x) for x in (Ix, Iy, It)]
    lib().orc_prox_l1(z[0].size, *[_p(x) for x in z], *[_p(x) for x in dat], beta, lam, sigma)
    return tuple(z)


def srbgs(x, b, st, sweeps):
    x, b = _f64(x).copy(), _f64(b)
    H, W = x.shape
    lib().orc_srbgs(H, W, _p(x), _p(b), st, sweeps)
    return x


# ---------------------------------------------------------------------------- pyramid / warp
def level_size(n, eta):
    return lib().orc_level_size(n, eta)


def level_sizes(H, W, eta, levels):
    hs, ws = [H], [W]
    for _ in range(1, levels):
        hs.append(level_size(hs[-1], eta))
        ws.append(level_size(ws[-1], eta))
    return list(zip(hs, ws))


def gauss_smooth(img, eta):
    img = _f64(img)
    H, W = img.shape
    out = np.empty_like(img)
    lib().orc_gauss_smooth(H, W, _p(img), _p(out), eta)
    return out


def downsample(img, Hc, Wc, eta):
    img = _f64(img)
    H, W = img.shape
    out = np.empty((Hc, Wc), np.float64)
    lib().orc_downsample(H, W, _p(img), Hc, Wc, _p(out), eta)
    return out


def upsample(field, Hf, Wf, scale):
    field = _f64(field)
    Hc, Wc = field.shape
    out = np.empty((Hf, Wf), np.float64)
    lib().orc_upsample(Hc, Wc, _p(field), Hf, Wf, _p(out), scale)
    return out


def derivatives(img):
    img = _f64(img)
    H, W = img.shape
    Ix, Iy = np.empty_like(img), np.empty_like(img)
    lib().orc_derivatives(H, W, _p(img), _p(Ix), _p(Iy))
    return Ix, Iy


def warp_linearise(I0, I1, I1x, I1y, u0, v0, beta):
    """Returns (Ix, Iy, It, max M_s)."""
    arrs = [_f64(x) for x in (I0, I1, I1x, I1y, u0, v0)]
    H, W = arrs[0].shape
    Ix, Iy, It = (np.empty((H, W), np.float64) for _ in range(3))
    ms = lib().orc_warp_linearise(H, W, *[_p(x) for x in arrs], beta, _p(Ix), _p(Iy), _p(It))
    return Ix, Iy, It, ms


# ---------------------------------------------------------------------------- solver state
STATE_FIELDS = ("w", "u", "v", "p1", "p2", "q11", "q12", "q21", "q22", "s", "wb", "ub", "vb")


@dataclass
class State:
    """ADMM: multipliers (w, u, v) and duals p, q, s.  pDR: X = (w, u, v), Xbar = (wb, ub, vb),
    ybar = (p, q)."""
    arrays: dict = field(default_factory=dict)

    @classmethod
    def zeros(cls, H, W):
        return cls({k: np.zeros((H, W), np.float64) for k in STATE_FIELDS})

    def copy(self):
        return State({k: v.copy() for k, v in self.arrays.items()})

    def __getitem__(self, k):
        return self.arrays[k]

    def __setitem__(self, k, v):
        self.arrays[k] = _f64(v).copy()

    def _ptrs(self):
        for k in STATE_FIELDS:
            a = self.arrays[k]
            if not (a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]):
                self.arrays[k] = _f64(a).copy()
        return (_D * 13)(*[_p(self.arrays[k]) for k in STATE_FIELDS])


def admm_step(state: State, Ix, Iy, It, a_tilde, params: Params) -> float:
    """One rpADMMI / rpADMMII iteration in place; returns ||A s + B y||^2 after the step."""
    dat = [_f64(x) for x in (Ix, Iy, It)]
    H, W = dat[0].shape
    P = params._c()
    return lib().orc_admm_step_flat(H, W, state._ptrs(), *[_p(x) for x in dat], a_tilde, ctypes.byref(P))


def pdr_step(state: State, Ix, Iy, It, params: Params) -> float:
    """One pDR iteration in place; returns ||X^{k+1} - X^k||^2."""
    dat = [_f64(x) for x in (Ix, Iy, It)]
    H, W = dat[0].shape
    P = params._c()
    return lib().orc_pdr_step_flat(H, W, state._ptrs(), *[_p(x) for x in dat], ctypes.byref(P))


def cp_step(state: State, Ix, Iy, It, params: Params) -> float:
    """One ALG1 (primal-dual) iteration in place; returns ||X^{k+1} - X^k||^2."""
    dat = [_f64(x) for x in (Ix, Iy, It)]
    H, W = dat[0].shape
    P = params._c()
    return lib().orc_cp_step_flat(H, W, state._ptrs(), *[_p(x) for x in dat], ctypes.byref(P))


def inner(state: State, Ix, Iy, It, a_tilde, params: Params, iters: int):
    """`iters` inner iterations (with the tol stopping test); returns (iters_run, residual)."""
    dat = [_f64(x) for x in (Ix, Iy, It)]
    H, W = dat[0].shape
    P = params._c()
    res = ctypes.c_double(0.0)
    n = lib().orc_inner_flat(H, W, state._ptrs(), *[_p(x) for x in dat], a_tilde, ctypes.byref(P),
                             iters, ctypes.byref(res))
    return int(n), res.value


def adapt_residuals(prev: State, cur: State, Ix, Iy, a_tilde, c, params: Params):
    """Norms (||r||, ||d||) of the constraint and dual residuals of the ADMM step prev -> cur taken
    with step c (the residual-balancing extension)."""
    dat = [_f64(x) for x in (Ix, Iy)]
    H, W = dat[0].shape
    P = params._c()
    rn, dn = ctypes.c_double(0.0), ctypes.c_double(0.0)
    lib().orc_adapt_residuals_flat(H, W, prev._ptrs(), cur._ptrs(), *[_p(x) for x in dat], a_tilde, c,
                                   ctypes.byref(P), ctypes.byref(rn), ctypes.byref(dn))
    return rn.value, dn.value


def adapt_rule(c, r_norm, d_norm):
    """The balancing rule: c doubled when ||r|| > 10 ||d||, halved when ||d|| > 10 ||r||."""
    return lib().orc_adapt_rule(c, r_norm, d_norm)


def inner_adapt(state: State, Ix, Iy, It, a_tilde, params: Params, iters: int, window: int, c: float):
    """A level's first warp under the adaptive step; returns (iters_run, residual, c, margin)."""
    dat = [_f64(x) for x in (Ix, Iy, It)]
    H, W = dat[0].shape
    P = params._c()
    res, cc, mg = ctypes.c_double(0.0), ctypes.c_double(c), ctypes.c_double(float("inf"))
    n = lib().orc_inner_adapt_flat(H, W, state._ptrs(), *[_p(x) for x in dat], a_tilde, ctypes.byref(P), iters,
                                   window, ctypes.byref(cc), ctypes.byref(mg), ctypes.byref(res))
    return int(n), res.value, cc.value, mg.value


def pdr_adapt_residuals(prev: State, cur: State, sigma, tau, params: Params):
    """pDR's balancing residuals of the step prev -> cur taken with (sigma, tau): the primal change
    ||X^{k+1} - X^k|| / sigma and the dual change ||ybar^{k+1} - ybar^k|| / tau."""
    H, W = prev["u"].shape
    P = params._c()
    rx, ry = ctypes.c_double(0.0), ctypes.c_double(0.0)
    lib().orc_pdr_adapt_residuals_flat(H, W, prev._ptrs(), cur._ptrs(), sigma, tau, ctypes.byref(P),
                                       ctypes.byref(rx), ctypes.byref(ry))
    return rx.value, ry.value


def inner_adapt_pdr(state: State, Ix, Iy, It, params: Params, iters: int, window: int, theta: float = 1.0):
    """A level's first warp of pDR under the adaptive steps; returns (iters_run, residual, theta,
    margin)."""
    dat = [_f64(x) for x in (Ix, Iy, It)]
    H, W = dat[0].shape
    P = params._c()
    res, th, mg = ctypes.c_double(0.0), ctypes.c_double(theta), ctypes.c_double(float("inf"))
    n = lib().orc_inner_adapt_pdr_flat(H, W, state._ptrs(), *[_p(x) for x in dat], ctypes.byref(P), iters, window,
                                       ctypes.byref(th), ctypes.byref(mg), ctypes.byref(res))
    return int(n), res.value, th.value, mg.value


def energy(w, u, v, Ix, Iy, It, beta, lam):
    arrs = [_f64(x) for x in (w, u, v, Ix, Iy, It)]
    H, W = arrs[0].shape
    return lib().orc_energy(H, W, *[_p(x) for x in arrs], beta, lam)


def dual_value(It, s):
    It, s = _f64(It), _f64(s)
    return lib().orc_dual_value(It.size, _p(It), _p(s))


def solve(I0, I1, params: Params):
    """Whole schedule.  Returns (u, v, w, stats) at level params.out_level."""
    I0, I1 = _f64(I0), _f64(I1)
    H, W = I0.shape
    sizes = level_sizes(H, W, params.eta, params.levels)
    h, w = sizes[params.out_level]
    u, v, wo = (np.zeros((h, w), np.float64) for _ in range(3))
    st = _Stats()
    P = params._c()
    rc = lib().orc_solve(H, W, _p(I0), _p(I1), ctypes.byref(P), _p(u), _p(v), _p(wo), ctypes.byref(st))
    if rc != 0:
        raise ValueError("oracle rejected the parameters")
    stats = dict(iters_run=st.iters_run, residual=st.residual, energy=st.energy, dual_value=st.dual_value,
                 c_final=st.c_final, adapt_margin=st.adapt_margin)
    return u, v, wo, stats
