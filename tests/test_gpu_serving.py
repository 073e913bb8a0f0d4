"""GPU tests of batched solves through the serving loop (continuous batching of requests of
different sizes).  Each request's result must be bitwise the one of the same pair solved alone,
admission must respect the HBM budget, and stopping must not hang."""
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
