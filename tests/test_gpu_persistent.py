"""GPU tests of the persistent ADMM engine (OF_ENGINE_PERSISTENT): one launch per warp of a level
runs every inner iteration, its warps synchronising with their neighbouring segments through
device counters.  Every pixel runs the streaming kernel's arithmetic, so whole solves must be
bitwise equal to the streaming engine's (which the parity tests check against the FP64 oracle);
the stopping test sums the residual in another grouping, so with a tolerance the iteration counts
may differ in rare cases and the flows are compared with the oracle instead.  The bounded waits
are tested with a segment that never publishes its progress."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2011_10979_gb300 import flow, synth  # noqa: E402

VARIANTS = {
    "padmm": dict(method=0, r=1.0),
    "rpadmm1": dict(method=0, r=1.618),
    "rpadmm2": dict(method=1, rho=1.9),
    "zach": dict(method=0, r=1.0, beta=0.0),
    "padmm_pp": dict(method=0, r=1.0, a_tilde_mode=1),
}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = flow.Context(0)
    yield c
    c.close()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _pair(H, W, seed):
    return synth.sinusoid_pair() if (H, W) == (48, 64) else synth.random_affine_rect_pair(H, W, seed)


@pytest.mark.parametrize("name", list(VARIANTS))
@pytest.mark.parametrize("H,W", [(48, 64), (130, 100), (240, 320), (480, 640)])
def test_persistent_equals_streaming_bitwise(ctx, name, H, W):
    pr = _pair(H, W, 11)
    kw = dict(lam=2.0, levels=3, warps=2, iters=23, **VARIANTS[name])
    P_stream = flow.default_params(engine=flow.OF_ENGINE_STREAM, **kw)
    P_pers = flow.default_params(engine=flow.OF_ENGINE_PERSISTENT, **kw)
    a = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), P_stream)
    b = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), P_pers)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert a[3]["iters_run"] == b[3]["iters_run"]
    assert b[3]["residual"] == pytest.approx(a[3]["residual"], rel=1e-5)
    assert b[3]["energy"] == pytest.approx(a[3]["energy"], rel=1e-12)
    # the persistent levels are not on the streaming kernel
    assert all(r == 0 for r in flow.of_rows_per_warp(ctx, [(H, W)], P_pers))


@pytest.mark.parametrize("prec,fp32_flow", [(flow.OF_PREC_FP16, 1), (flow.OF_PREC_BF16, 1), (flow.OF_PREC_BF16, 0)])
def test_persistent_16bit_storage_equals_streaming(ctx, prec, fp32_flow):
    pr = synth.affine_rect_pair(240, 320, seed=4)
    kw = dict(lam=5.0, levels=4, warps=3, iters=17, precision=prec, fp32_flow=fp32_flow, fp32_last_warp=1)
    a = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), flow.default_params(engine=flow.OF_ENGINE_STREAM, **kw))
    b = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), flow.default_params(engine=flow.OF_ENGINE_PERSISTENT, **kw))
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def _batch():
    return [synth.random_affine_rect_pair(h, w, 30 + k) for k, (h, w) in
            enumerate([(64, 96), (240, 320), (37, 53), (130, 100), (436, 1024), (1, 1), (480, 640), (9, 200)])]


@pytest.mark.parametrize("prec", [flow.OF_PREC_FP32, flow.OF_PREC_BF16])
@pytest.mark.parametrize("name", ["padmm", "rpadmm2", "zach"])
def test_persistent_batch_equals_single_and_streaming(ctx, prec, name):
    """Uneven pairs in one persistent launch per level and warp: bitwise the single-pair solves of
    the same engine and the streaming engine's batch."""
    pairs = _batch()
    kw = dict(lam=2.0, levels=4, warps=2, iters=20, precision=prec, **VARIANTS[name])
    Pp = flow.default_params(engine=flow.OF_ENGINE_PERSISTENT, **kw)
    Ps = flow.default_params(engine=flow.OF_ENGINE_STREAM, **kw)
    up, vp, stp = flow.of_solve_batch(ctx, [cu(p.I0) for p in pairs], [cu(p.I1) for p in pairs], Pp)
    us, vs, sts = flow.of_solve_batch(ctx, [cu(p.I0) for p in pairs], [cu(p.I1) for p in pairs], Ps)
    for k, p in enumerate(pairs):
        su, sv, _, sst = flow.of_solve(ctx, cu(p.I0), cu(p.I1), Pp)
        assert torch.equal(up[k], su) and torch.equal(vp[k], sv), k
        assert torch.equal(up[k], us[k]) and torch.equal(vp[k], vs[k]), k
        assert stp[k]["iters_run"] == sst["iters_run"] == sts[k]["iters_run"]


@pytest.mark.parametrize("batched", [False, True])
def test_persistent_stopping_rule_against_the_oracle(ctx, orc, batched):
    """tol > 0: the in-kernel stopping test (pair barriers every 10 iterations) against the oracle's
    schedule; the iteration counts may differ by the FP32/FP64 residual at a check, so the bar is
    the end-point error, and the counts must stay within one check per warp."""
    pr = synth.sinusoid_pair()
    kw = dict(lam=5.0, levels=3, warps=5, iters=200, tol=3e-3)
    P = flow.default_params(engine=flow.OF_ENGINE_PERSISTENT, **kw)
    if batched:
        other = synth.random_affine_rect_pair(130, 100, 5)
        us, vs, sts = flow.of_solve_batch(ctx, [cu(pr.I0), cu(other.I0)], [cu(pr.I1), cu(other.I1)], P)
        u, v, st = us[0], vs[0], sts[0]
    else:
        u, v, _, st = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), P)
    ru, rv, _, rst = orc.solve(pr.I0, pr.I1, orc.Params(**kw))
    u, v = u.double().cpu().numpy(), v.double().cpu().numpy()
    epe = float(np.hypot(u - ru, v - rv).mean())
    assert st["iters_run"] < 3 * 5 * 200 and st["iters_run"] % 10 == 0
    assert abs(st["iters_run"] - rst["iters_run"]) <= 10 * 3 * 5
    assert epe <= 1e-2, epe
    assert st["residual"] < 3e-3 * 1.0001


def test_persistent_schedule_against_the_oracle(ctx, orc):
    pr = synth.sinusoid_pair()
    kw = dict(lam=0.05, levels=3, warps=5, iters=50)
    u, v, _, st = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), flow.default_params(engine=flow.OF_ENGINE_PERSISTENT, **kw))
    ru, rv, _, rst = orc.solve(pr.I0, pr.I1, orc.Params(**kw))
    u, v = u.double().cpu().numpy(), v.double().cpu().numpy()
    assert np.abs(u - ru).max() <= 1e-3 and np.abs(v - rv).max() <= 1e-3
    assert float(np.hypot(u - ru, v - rv).mean()) <= 1e-2
    assert st["iters_run"] == rst["iters_run"]


def test_bounded_wait_runs_out_and_the_device_stays_usable(ctx):
    """A segment that never publishes its progress: its neighbours' waits run out after the bound
    (50 ms here), the launch ends with its timeout flag set and the device keeps working."""
    to, nseg = flow.of_persistent_selftest(480, 640, 3, -1, 2000.0)
    assert to == 0 and nseg > 100
    to, _ = flow.of_persistent_selftest(480, 640, 3, nseg // 2, 50.0)
    assert to == 1
    to, _ = flow.of_persistent_selftest(480, 640, 3, 0, 50.0)
    assert to == 1
    pr = synth.sinusoid_pair()
    u, v, _, st = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), flow.default_params(engine=flow.OF_ENGINE_PERSISTENT))
    assert bool(torch.isfinite(u).all()) and np.isfinite(st["energy"])
