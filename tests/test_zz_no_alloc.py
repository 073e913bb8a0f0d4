"""GPU test of of_admm_iterate_noalloc, the allocation-free form of the fused ADMM iteration.

It serves callers that cannot allocate device memory (code under an allocator it does not own,
regions where cudaMalloc would synchronise or is forbidden, runtimes that own every device byte):
instead of a caller-provided scratch buffer it uses the library's static 32 MiB device array.
Its fields must match of_admm_iterate with a torch-allocated scratch buffer, within the
iteration tolerance of the parity tests, on two calls in a row -- the static array keeps the
previous call's contents, which must not leak into the next call.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2011_10979_gb300 import build, flow  # noqa: E402

FIELDS = ("w", "u", "v", "p1", "p2", "q11", "q12", "q21", "q22", "s")
TOL = 1e-4   # the iteration tolerance of tests/test_gpu_parity.py


def _state(H, W, rng, lam, beta):
    def ball(k):
        x = rng.normal(size=(k, H, W))
        return x / np.maximum(1.0, np.sqrt((x * x).sum(0)))
    p, q = ball(2), ball(4)
    st = dict(p1=p[0], p2=p[1], q11=q[0], q12=q[1], q21=q[2], q22=q[3], s=rng.uniform(-lam, lam, (H, W)),
              w=rng.normal(size=(H, W)), u=rng.normal(size=(H, W)), v=rng.normal(size=(H, W)))
    if beta == 0.0:
        st["w"] = st["p1"] = st["p2"] = None
    return st


def _noalloc(fields, Ix, Iy, It, a_tilde, params, iters):
    H, W = Ix.shape
    res = ctypes.c_double(0.0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = flow.lib().of_admm_iterate_noalloc(flow._fields(fields), Ix.data_ptr(), Iy.data_ptr(), It.data_ptr(), H, W,
                                            Ix.stride(0), ctypes.c_float(a_tilde), ctypes.byref(params), iters,
                                            ctypes.byref(res), stream)
    flow.check(st)
    return res.value


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return flow.lib()


LIMIT = 32 << 20   # the static array's size, as the header states


def _pitched(a, pitch):
    """A CUDA FP32 copy of the H x W array `a` whose rows are `pitch` elements apart."""
    H, W = a.shape
    buf = torch.full((H, pitch), float("nan"), dtype=torch.float32, device="cuda")
    buf[:, :W] = torch.from_numpy(a.astype(np.float32)).cuda()
    return buf[:, :W]


def _largest_rows_under_limit(lib, pitch):
    H = 1
    while lib.of_fields_bytes(H + 1, pitch) <= LIMIT:
        H += 1
    return H


def test_noalloc_matches_scratch_entry_point_on_two_calls(lib):
    H_edge = _largest_rows_under_limit(lib, 640)
    cases = [(100, 130, 130, 0.05, 0, 1.0, 31, 1),      # rpADMMI (pADMM), beta > 0, odd count
             (480, 640, 640, 0.0, 1, 1.0, 20, 2),       # rpADMMII, beta = 0 model, the 640 x 480 level
             (97, 2900, 2929, 0.05, 0, 1.618, 9, 3),    # padded rows: the strip height at W differs from pitch
             (H_edge, 640, 640, 0.05, 0, 1.0, 6, 4)]    # the layout's last bytes at the end of the array
    for H, W, pitch, beta, method, r, iters, seed in cases:
        assert lib.of_fields_bytes(H, pitch) <= LIMIT
        rng = np.random.default_rng(seed)
        lam = 0.3
        st = _state(H, W, rng, lam, beta)
        Ix, Iy, It = (_pitched(rng.normal(size=(H, W)) * s, pitch) for s in (0.4, 0.4, 0.2))
        at = float((beta ** 2 + Ix.double() ** 2 + Iy.double() ** 2).max()) + 1e-3
        P = flow.default_params(method=method, lam=lam, beta=beta, r=r, rho=1.9)
        ref = {k: (None if a is None else _pitched(a, pitch)) for k, a in st.items()}
        got = {k: (None if a is None else _pitched(a, pitch)) for k, a in st.items()}
        r_ref = flow.of_admm_iterate(ref, Ix, Iy, It, at, P, iters)
        r_got = _noalloc(got, Ix, Iy, It, at, P, iters)
        torch.cuda.synchronize()
        for k in FIELDS:
            if ref[k] is None:
                continue
            err = float((ref[k] - got[k]).abs().max())
            assert err <= TOL, (H, W, k, err)
            assert torch.isnan(got[k].as_strided((H, pitch - W), (pitch, 1), W)).all() if pitch > W else True
        assert abs(r_ref - r_got) <= 1e-6 * max(abs(r_ref), 1.0)


def test_noalloc_rejects_fields_beyond_the_static_scratch(lib):
    x = torch.zeros((1, 1), device="cuda")
    f = {k: x for k in FIELDS}
    P = flow.default_params()
    res = ctypes.c_double(0.0)
    H_edge = _largest_rows_under_limit(lib, 640)
    for H, W in ((2000, 2000), (H_edge + 1, 640)):   # far over, and one row over the limit
        assert lib.of_fields_bytes(H, W) > LIMIT
        st = lib.of_admm_iterate_noalloc(flow._fields(f), x.data_ptr(), x.data_ptr(), x.data_ptr(), H, W, W,
                                         ctypes.c_float(1.0), ctypes.byref(P), 1, ctypes.byref(res), None)
        assert st == flow.OF_EINVAL
        assert b"32 MiB" in lib.of_last_error(None)
