"""The one-launch pDR kernel (one symmetric Gauss-Seidel sweep, 32 x 32 output tiles with their
halo staged in shared memory, ping-pong buffers) against the engines it replaces on streamed
levels.  Every stage rounds as the per-kernel engine does, so the flows are bitwise those of the
literal plain engine (R B B R, in place, one kernel per half-sweep), of the level-resident engine
and of the stage-by-stage solver of the serving loop (which keeps the per-kernel engine)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2011_10979_gb300 import flow, synth  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = flow.Context(0)
    yield c
    c.close()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.mark.parametrize("H,W", [(1, 1), (1, 70), (70, 1), (31, 33), (97, 131), (203, 333), (480, 640)])
@pytest.mark.parametrize("beta", [0.05, 0.0])
@pytest.mark.parametrize("tol", [0.0, 3e-3])
def test_tile_kernel_equals_the_plain_engine(ctx, H, W, beta, tol):
    """One level, every iteration on the streaming engines: bitwise the literal plain engine (FP32),
    on tiles with ragged right and bottom edges and degenerate sizes; the same iteration count
    under the stopping rule."""
    pr = synth.random_affine_rect_pair(H, W, 7 + H) if min(H, W) > 8 else synth.Pair(
        np.random.default_rng(H + W).random((H, W)).astype(np.float32),
        np.random.default_rng(H + W + 1).random((H, W)).astype(np.float32), None, None)
    out = []
    for eng in (flow.OF_ENGINE_STREAM, flow.OF_ENGINE_PLAIN):
        P = flow.default_params(method=flow.OF_PDR, lam=2.0, beta=beta, levels=1, warps=2, iters=23, tol=tol,
                                engine=eng)
        u, v, w, st = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), P, want_w=True)
        out.append((u, v, w, st))
    (u0, v0, w0, s0), (u1, v1, w1, s1) = out
    assert torch.equal(u0, u1) and torch.equal(v0, v1) and torch.equal(w0, w1)
    assert s0["iters_run"] == s1["iters_run"]
    assert s0["residual"] == pytest.approx(s1["residual"], rel=1e-5, abs=1e-12)


@pytest.mark.parametrize("prec,fp32_flow", [(0, 1), (2, 1), (2, 0), (1, 0)])
def test_tile_kernel_equals_the_resident_engine_on_every_storage(ctx, prec, fp32_flow):
    """A 150 x 150 level fits the level-resident engine: the same solve streamed (tile kernel) and
    resident, in FP32 and 16-bit storage (X rounded to its storage type after every half-sweep)."""
    pr = synth.random_affine_rect_pair(150, 150, 4)
    out = []
    for eng in (flow.OF_ENGINE_STREAM, flow.OF_ENGINE_RESIDENT):
        P = flow.default_params(method=flow.OF_PDR, lam=2.0, levels=2, warps=2, iters=21, precision=prec,
                                fp32_flow=fp32_flow, engine=eng)
        u, v, _, st = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), P)
        out.append((u, v, st))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


def test_batch_of_uneven_pairs_equals_single_solves(ctx):
    pairs = [synth.random_affine_rect_pair(H, W, 11 + k) for k, (H, W) in enumerate([(240, 320), (97, 131), (130, 100),
                                                                                    (480, 640)])]
    P = flow.default_params(method=flow.OF_PDR, lam=2.0, levels=3, warps=2, iters=15)
    us, vs, _ = flow.of_solve_batch(ctx, [cu(p.I0) for p in pairs], [cu(p.I1) for p in pairs], P)
    for k, p in enumerate(pairs):
        u, v, _, _ = flow.of_solve(ctx, cu(p.I0), cu(p.I1), P)
        assert torch.equal(us[k], u) and torch.equal(vs[k], v), k


def test_serving_loop_per_kernel_engine_equals_the_tile_kernel(ctx):
    """The serving loop's stage solver runs pDR on the per-kernel engine (in place); of_solve runs
    the tile kernel: the flows are bitwise equal."""
    reqs = [synth.random_affine_rect_pair(H, W, 21 + H) for H, W in [(240, 320), (97, 131)]]
    P = flow.default_params(method=flow.OF_PDR, lam=2.0, levels=3, warps=2, iters=12)
    ref = [flow.of_solve_host(ctx, r.I0, r.I1, P)[:2] for r in reqs]
    srv = flow.Context(0)
    flow.of_server_start(srv, P, 0, 4)
    try:
        ids = [flow.of_server_submit(srv, r.I0, r.I1) for r in reqs]
        got, t0 = {}, time.time()
        while len(got) < len(ids):
            for rid, r in zip(ids, reqs):
                if rid not in got:
                    res = flow.of_server_poll(srv, rid, r.I0.shape)
                    if res is not None:
                        got[rid] = res
            assert time.time() - t0 < 120
            time.sleep(0.002)
        for rid, (u, v) in zip(ids, ref):
            assert np.array_equal(got[rid][0], u) and np.array_equal(got[rid][1], v)
    finally:
        flow.of_server_stop(srv)
        srv.close()


def test_tile_kernel_against_the_oracle(ctx, orc):
    """Three levels of a 203 x 333 pair (the two finer ones streamed) against the FP64 oracle: the
    EPE bar, and the flow bitwise that of the literal plain engine, so any larger single-pixel
    deviation is the method's FP32 behaviour (recorded for pDR at 640x480 in
    test_gpu_schedules), not the kernel's."""
    pr = synth.random_affine_rect_pair(203, 333, 9)
    kw = dict(method=2, lam=5.0, levels=3, warps=3, iters=30)
    u, v, _, st = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), flow.default_params(**kw))
    up, vp, _, _ = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), flow.default_params(engine=flow.OF_ENGINE_PLAIN, **kw))
    assert torch.equal(u, up) and torch.equal(v, vp)
    ru, rv, _, rst = orc.solve(pr.I0, pr.I1, orc.Params(**kw))
    u, v = u.cpu().double().numpy(), v.cpu().double().numpy()
    print("max|du| %.2e max|dv| %.2e" % (np.abs(u - ru).max(), np.abs(v - rv).max()))
    assert np.hypot(u - ru, v - rv).mean() <= 1e-2
    assert st["iters_run"] == rst["iters_run"]
