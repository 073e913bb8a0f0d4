"""GPU tests of the serving loop: continuous batching of requests of different sizes, every step
advancing all admitted requests by one warp of their current pyramid level with the inner
iterations of all of them in shared launches.  Each request's result must be bitwise the one of the
same pair solved alone (through the loop or by of_solve), admission must respect the HBM budget,
non-finite inputs must be reported, and stopping must not hang."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2011_10979_gb300 import flow, synth  # noqa: E402


@pytest.fixture(scope="module")
def pairs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = [synth.sinusoid_pair(seed=s) for s in range(2)]
    out += [synth.random_affine_rect_pair(H, W, 10 + k) for k, (H, W) in enumerate([(120, 160), (97, 131), (240, 320)])]
    return out


def _wait(ctx, ids, shapes, timeout=120.0):
    res = {}
    t0 = time.time()
    while len(res) < len(ids):
        for rid, shp in zip(ids, shapes):
            if rid in res:
                continue
            r = flow.of_server_poll(ctx, rid, shp)
            if r is not None:
                res[rid] = r
        assert time.time() - t0 < timeout, "serving loop did not finish in time"
        time.sleep(0.002)
    return res


def test_results_identical_alone_and_in_the_mix(pairs):
    P = flow.default_params(lam=2.0, levels=3, warps=3, iters=30)
    alone = flow.Context(0)
    ref = [flow.of_solve_host(alone, p.I0, p.I1, P)[:2] for p in pairs]
    alone.close()
    ctx = flow.Context(0)
    flow.of_server_start(ctx, P, 0, 3)
    try:
        # the mix: every pair twice, interleaved, submitted while earlier requests run
        order = list(range(len(pairs))) * 2
        ids, shapes = [], []
        for k in order:
            ids.append(flow.of_server_submit(ctx, pairs[k].I0, pairs[k].I1))
            shapes.append(pairs[k].I0.shape)
            time.sleep(0.001)
        res = _wait(ctx, ids, shapes)
        for rid, k in zip(ids, order):
            u, v, ms = res[rid]
            assert np.array_equal(u, ref[k][0]) and np.array_equal(v, ref[k][1])
            assert ms > 0
    finally:
        flow.of_server_stop(ctx)
        ctx.close()


@pytest.mark.parametrize("prec", [flow.OF_PREC_FP32, flow.OF_PREC_BF16])
def test_mixed_sizes_up_to_1920x1080_alone_and_in_the_mix(prec):
    """Requests of five sizes (up to 1920 x 1080) arriving while others run, some at coarse levels
    while others are at fine ones; BF16 duals with the FP32 last warp switch groups mid-mix.  Every
    flow equals the request's own of_solve bitwise, and its run through the loop alone."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sizes = [(240, 320), (1080, 1920), (64, 96), (436, 1024), (480, 640)]
    reqs = [synth.layered_pair(h, w, seed=60 + k, max_shift=20.0, sigma=0.01) for k, (h, w) in enumerate(sizes)]
    P = flow.default_params(lam=5.0, levels=5, warps=3, iters=20, precision=prec, fp32_flow=1, fp32_last_warp=1)
    ctx = flow.Context(0)
    ref = [flow.of_solve_host(ctx, r.I0, r.I1, P)[:2] for r in reqs]
    flow.of_server_start(ctx, P, 0, 8)
    try:
        alone = []
        for r in reqs[:2]:
            rid = flow.of_server_submit(ctx, r.I0, r.I1)
            alone.append(_wait(ctx, [rid], [r.I0.shape])[rid])
        order = [0, 1, 2, 3, 4, 2, 0, 4, 1, 3]
        ids = []
        for k in order:
            ids.append(flow.of_server_submit(ctx, reqs[k].I0, reqs[k].I1))
            time.sleep(0.003)
        res = _wait(ctx, ids, [reqs[k].I0.shape for k in order], timeout=300.0)
        for rid, k in zip(ids, order):
            u, v, _ = res[rid]
            assert np.array_equal(u, ref[k][0]) and np.array_equal(v, ref[k][1]), sizes[k]
        for k in range(2):
            assert np.array_equal(alone[k][0], ref[k][0]) and np.array_equal(alone[k][1], ref[k][1])
    finally:
        flow.of_server_stop(ctx)
        ctx.close()


def test_non_finite_request_is_reported_and_the_others_finish(pairs):
    P = flow.default_params(lam=2.0, levels=3, warps=2, iters=10)
    ctx = flow.Context(0)
    flow.of_server_start(ctx, P, 0, 4)
    try:
        bad = pairs[0].I0.copy()
        bad[5, 7] = np.nan
        rb = flow.of_server_submit(ctx, bad, pairs[0].I1)
        rg = flow.of_server_submit(ctx, pairs[1].I0, pairs[1].I1)
        res = _wait(ctx, [rg], [pairs[1].I0.shape])
        assert np.isfinite(res[rg][0]).all()
        t0 = time.time()
        while True:
            try:
                r = flow.of_server_poll(ctx, rb, bad.shape)
            except flow.OfError as e:
                assert e.status == flow.OF_ENUMERIC
                break
            assert r is None and time.time() - t0 < 60
            time.sleep(0.002)
    finally:
        flow.of_server_stop(ctx)
        ctx.close()


def test_admission_respects_the_budget(pairs):
    P = flow.default_params(lam=2.0, levels=3, warps=2, iters=10)
    big = pairs[-1]
    need = flow.lib().of_arena_bytes(big.I0.shape[0], big.I0.shape[1], flow.default_params(lam=2.0, levels=3, warps=2,
                                                                                             iters=10))
    ctx = flow.Context(0)
    # a budget that fits one large request at a time, but not two
    flow.of_server_start(ctx, P, int(need * 1.5), 4)
    try:
        ids = [flow.of_server_submit(ctx, big.I0, big.I1) for _ in range(3)]
        res = _wait(ctx, ids, [big.I0.shape] * 3)
        assert len(res) == 3
        # a request larger than the whole budget fails cleanly
        huge = np.zeros((2000, 2000), np.float32)
        rid = flow.of_server_submit(ctx, huge, huge)
        t0 = time.time()
        while True:
            try:
                r = flow.of_server_poll(ctx, rid, (2000, 2000))
            except flow.OfError as e:
                assert e.status == flow.OF_ENOMEM
                break
            assert r is None and time.time() - t0 < 30
            time.sleep(0.002)
    finally:
        flow.of_server_stop(ctx)
        ctx.close()


def test_stop_with_queued_requests(pairs):
    P = flow.default_params(lam=2.0, levels=3, warps=2, iters=10)
    ctx = flow.Context(0)
    flow.of_server_start(ctx, P, 0, 1)
    for _ in range(6):
        flow.of_server_submit(ctx, pairs[-1].I0, pairs[-1].I1)
    t0 = time.time()
    flow.of_server_stop(ctx)
    assert time.time() - t0 < 60
    with pytest.raises(flow.OfError):
        flow.of_server_submit(ctx, pairs[0].I0, pairs[0].I1)
    ctx.close()
