"""CPU checks of the C ABI: the library loads, exports every function include/tvl1flow.h
declares, and validates arguments before touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_2011_10979_gb300 import build, flow

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return flow.lib()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(of_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 20
    for n in sorted(names):
        assert hasattr(L, n), n
    assert set(flow.EXPORTS) == names


def test_default_params_are_the_papers(L):
    p = flow.default_params()
    assert (p.method, p.c, p.a, p.r, p.sigma, p.tau, p.gs_sweeps) == (0, pytest.approx(0.05), 8.0, 1.0, 2.0,
                                                                      pytest.approx(0.4), 1)
    assert p.rho == pytest.approx(1.9) and p.beta == pytest.approx(0.05) and p.eta == 0.5


def test_arena_bytes_and_validation_without_gpu(L):
    p = flow.default_params(levels=5, warps=10, iters=100)
    n = L.of_arena_bytes(480, 640, ctypes.byref(p))
    assert 20e6 < n < 200e6
    for bad in (dict(levels=0), dict(eta=1.0), dict(lam=0.0), dict(r=1.7), dict(out_level=5)):
        q = flow.default_params(**{"levels": 5, **bad})
        assert L.of_arena_bytes(480, 640, ctypes.byref(q)) == 0
    assert L.of_arena_bytes(0, 640, ctypes.byref(p)) == 0
    side = 32768    # OF_MAX_SIDE in include/tvl1flow.h
    assert L.of_arena_bytes(side, 8, ctypes.byref(p)) > 0 and L.of_arena_bytes(8, side, ctypes.byref(p)) > 0
    for H, W in ((side + 1, 8), (8, side + 1)):
        assert L.of_arena_bytes(H, W, ctypes.byref(p)) == 0
        assert b"[1, 32768]" in L.of_last_error(None)
    st = L.of_solve(None, None, None, 10, 10, 10, ctypes.byref(p), None, None, None, 10, None, None)
    assert st == flow.OF_EINVAL
    assert b"ctx" in L.of_last_error(None)


def test_rows_per_warp_validation_without_gpu(L):
    """The strip-height field takes -1 (autotune), 0 (built-in rule) or one of the kernel's heights;
    a set height can be the lowest, so the partial-sum slots grow to its block count."""
    base = L.of_arena_bytes(480, 640, ctypes.byref(flow.default_params(levels=5)))
    for ok in (-1, 0, 1, 2, 8, 32):
        q = flow.default_params(levels=5, rows_per_warp=ok)
        n = L.of_arena_bytes(480, 640, ctypes.byref(q))
        assert n >= base if ok else n == base
    for bad in (-2, 3, 4, 16, 64):
        q = flow.default_params(levels=5, rows_per_warp=bad)
        assert L.of_arena_bytes(480, 640, ctypes.byref(q)) == 0
        assert b"rows_per_warp" in L.of_last_error(None)
    rows = (ctypes.c_int * 5)()
    H = (ctypes.c_int * 1)(480)
    st = L.of_rows_per_warp(None, 1, H, H, ctypes.byref(flow.default_params(levels=5)), rows)
    assert st == flow.OF_EINVAL


def _golden_params():
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", "sec4_parameters.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, value = line.split()[:2]
                out[name] = float(value)
    return out


def test_defaults_match_the_printed_sec4_settings(L):
    """The library's defaults and each method's settings against the values Sec. 4 prints
    (tests/golden/sec4_parameters.txt).  ALG1's primal step reads the garbled rule as
    1 / (L^2 tau)."""
    g = _golden_params()
    p = flow.default_params()
    assert p.c == pytest.approx(g["c"]) and p.r == pytest.approx(g["r_padmm"])
    assert p.rho == pytest.approx(g["rho_rpadmm2"])
    assert p.sigma == pytest.approx(g["pdr_sigma"]) and p.tau == pytest.approx(g["pdr_tau"])
    assert p.cp_tau == pytest.approx(g["alg1_tau"])
    assert p.cp_sigma == pytest.approx(1.0 / (g["alg1_L2"] * g["alg1_tau"]))
    assert p.beta == pytest.approx(g["beta"]) and p.a == pytest.approx(g["a"])
    # rpADMMI's printed relaxation lies inside the range the library accepts, (0, (1 + sqrt 5) / 2)
    q = flow.default_params(levels=5, r=g["r_rpadmm1"])
    assert L.of_arena_bytes(480, 640, ctypes.byref(q)) > 0
    q = flow.default_params(levels=5, beta=g["beta_alt"])
    assert L.of_arena_bytes(480, 640, ctypes.byref(q)) > 0


def test_fields_bytes_covers_every_width_up_to_the_pitch(L):
    """The step-level scratch holds 19 planes, then one FP64 partial sum per block of the engine
    in use, then the device scalars.  Its size may depend on (H, pitch) only, so the partial sums
    must be sized for the most blocks any width W <= pitch launches: 1-row strips of 29 columns
    and 4 rows per block for the fused ADMM kernel.  H = 97, pitch = 2929 is a case where the
    strip height picked at W = pitch (8 rows) launches fewer blocks than the one at W = 2900."""
    for H, pitch in ((97, 2929), (1, 1), (480, 640), (3, 4096), (689, 640)):
        plane = -(-(H * pitch * 4) // 256) * 256
        blocks = -(-pitch // 29) * -(-H // 4)
        need = 19 * plane + -(-(blocks * 8) // 256) * 256 + 64
        assert L.of_fields_bytes(H, pitch) >= need, (H, pitch)
    assert L.of_fields_bytes(0, 5) == 0 and L.of_fields_bytes(5, 0) == 0


def test_adaptive_step_validation_without_gpu(L):
    """c_adapt_iters: 0 (the fixed steps) or a positive multiple of 10; ADMM methods and pDR with one
    sweep, on the fused engines only."""
    assert flow.default_params().c_adapt_iters == 0
    for ok in (0, 10, 30, 1000):
        for m in (flow.OF_PADMM_I, flow.OF_PADMM_II, flow.OF_PDR):
            q = flow.default_params(levels=5, c_adapt_iters=ok, method=m)
            assert L.of_arena_bytes(480, 640, ctypes.byref(q)) > 0
    for bad in (dict(c_adapt_iters=-10), dict(c_adapt_iters=15), dict(c_adapt_iters=20, method=flow.OF_PDR, gs_sweeps=2),
                dict(c_adapt_iters=20, method=flow.OF_CP), dict(c_adapt_iters=20, engine=flow.OF_ENGINE_PLAIN)):
        q = flow.default_params(levels=5, **bad)
        assert L.of_arena_bytes(480, 640, ctypes.byref(q)) == 0, bad
        assert b"c_adapt_iters" in L.of_last_error(None)
    with pytest.raises(TypeError):
        flow.default_params(c_adapt=20)
