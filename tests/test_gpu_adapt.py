"""GPU parity of the opt-in adaptive ADMM step (residual balancing of c in the first
c_adapt_iters iterations of every level's first warp, frozen afterwards) against the FP64
oracle, through the C ABI.

Every balancing test is a decision between doubling, halving and keeping c; both sides take it
from their own residual norms (FP32 fields with FP64 sums here, FP64 in the oracle), so each
fixture first checks that the oracle's decisions were at least 1% from a tie.  The step the solve
ends with (a power-of-two multiple of c) must then be the oracle's, and the flows meet the
whole-schedule bar (max |du|, |dv| <= 1e-3 px, EPE <= 1e-2 px)."""
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


def np64(t):
    return t.detach().cpu().double().numpy()


METHODS = {"padmm": dict(method=0, r=1.0), "rpadmm1": dict(method=0, r=1.618), "rpadmm2": dict(method=1, rho=1.9),
           "zach": dict(method=0, r=1.0, beta=0.0), "padmm_pp": dict(method=0, r=1.0, a_tilde_mode=1)}
ENGINES = {"fused": flow.OF_ENGINE_FUSED, "stream": flow.OF_ENGINE_STREAM, "persistent": flow.OF_ENGINE_PERSISTENT}
MARGIN = 0.01


def _both(ctx, orc, pr, kw, engine=flow.OF_ENGINE_FUSED, **gpu_kw):
    P = flow.default_params(engine=engine, **kw, **gpu_kw)
    u, v, _, st = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), P)
    ru, rv, _, rst = orc.solve(pr.I0, pr.I1, orc.Params(**kw))
    return np64(u), np64(v), st, ru, rv, rst


def _check(u, v, st, ru, rv, rst, c0):
    assert rst["adapt_margin"] > MARGIN, "fixture too close to a balancing tie: %g" % rst["adapt_margin"]
    assert rst["c_final"] != c0, "the fixture must move c"
    assert st["c"] == pytest.approx(rst["c_final"], rel=1e-6)
    du, dv = np.abs(u - ru), np.abs(v - rv)
    epe = float(np.hypot(u - ru, v - rv).mean())
    assert du.max() <= 1e-3 and dv.max() <= 1e-3 and epe <= 1e-2, (du.max(), dv.max(), epe)
    assert st["iters_run"] == rst["iters_run"]


@pytest.mark.parametrize("engine", list(ENGINES))
@pytest.mark.parametrize("name", list(METHODS))
@pytest.mark.parametrize("c0", [50.0, 0.0005])
def test_adaptive_step_matches_the_oracle(ctx, orc, name, engine, c0):
    """The 64 x 48 sinusoid pair, 3 levels x 3 warps x 40 iterations with a 30-iteration window,
    from a step 1000 times too large and 100 times too small."""
    pr = synth.sinusoid_pair()
    kw = dict(lam=5.0, levels=3, warps=3, iters=40, c=c0, c_adapt_iters=30, **METHODS[name])
    _check(*_both(ctx, orc, pr, kw, ENGINES[engine]), c0)


@pytest.mark.parametrize("H,W,levels", [(97, 131, 3), (203, 333, 2), (480, 640, 5)])
def test_adaptive_step_on_multi_tile_levels(ctx, orc, H, W, levels):
    """Levels that span several strips and blocks with ragged right and bottom edges, up to the
    640 x 480 workload's five levels (the coarse ones level-resident after the window)."""
    pr = synth.random_affine_rect_pair(H, W, 31 + H)
    kw = dict(lam=5.0, levels=levels, warps=2, iters=30, c=20.0, c_adapt_iters=20)
    _check(*_both(ctx, orc, pr, kw), 20.0)


def test_engines_give_the_same_flow_and_step(ctx):
    """The window runs on the streaming kernel whatever the engine; the rest of each warp on the
    level's engine, which computes every pixel alike: flows and the final step are bitwise equal."""
    pr = synth.random_affine_rect_pair(150, 210, 5)
    out = []
    for eng in ENGINES.values():
        P = flow.default_params(lam=5.0, levels=4, warps=2, iters=40, c=0.002, c_adapt_iters=20, engine=eng)
        u, v, _, st = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), P)
        out.append((u, v, st["c"]))
    for u, v, c in out[1:]:
        assert torch.equal(u, out[0][0]) and torch.equal(v, out[0][1]) and c == out[0][2]


def test_window_of_zero_is_the_fixed_step(ctx):
    pr = synth.sinusoid_pair()
    P0 = flow.default_params(lam=5.0)
    u0, v0, _, s0 = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), P0)
    assert s0["c"] == pytest.approx(0.05)
    # a window longer than the warp: every iteration of each level's first warp is in it
    P = flow.default_params(lam=5.0, levels=3, warps=2, iters=25, c=5.0, c_adapt_iters=60)
    u, v, _, st = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), P)
    assert st["iters_run"] == 3 * 2 * 25 and st["c"] != 5.0


def test_adaptive_step_with_the_stopping_test(ctx, orc):
    """tol > 0: the test starts after the window; the iteration counts agree with the oracle to
    within one test period per warp, exactly when the decisions agree."""
    pr = synth.sinusoid_pair()
    kw = dict(lam=5.0, levels=3, warps=3, iters=200, c=50.0, c_adapt_iters=30, tol=3e-3)
    u, v, st, ru, rv, rst = _both(ctx, orc, pr, kw)
    assert rst["adapt_margin"] > MARGIN
    assert st["c"] == pytest.approx(rst["c_final"], rel=1e-6)
    assert st["iters_run"] < 3 * 3 * 200
    assert abs(st["iters_run"] - rst["iters_run"]) <= 30
    if st["iters_run"] == rst["iters_run"]:
        assert np.hypot(u - ru, v - rv).mean() <= 1e-2


BF16_ADAPT = pytest.mark.xfail(strict=True, reason="EPE 1.5e-2 px > 1e-2: each multiplier step adds c x (BF16 "
                                                   "rounding of s), and the balanced c ends far above 0.05")


@pytest.mark.parametrize("prec", [pytest.param(flow.OF_PREC_BF16, marks=BF16_ADAPT), flow.OF_PREC_FP16])
def test_adaptive_step_with_16bit_duals(ctx, orc, prec):
    """16-bit duals and data with the flow in FP32: the balancing residuals come from the stored
    16-bit duals, so the fixture asks for a 10% margin; the step must match and the flow meet the
    16-bit storage bar (EPE <= 1e-2 px).  FP16 meets it; BF16 does not (measured EPE 1.5e-2 px):
    the multiplier update moves the flow by r c (A s + B y), so the rounding of the stored s
    (8-bit mantissa, |s| up to lambda) enters the flow scaled by c, and from c = 50 the balanced
    step stays well above the paper's 0.05.  Recorded as a strict expected failure."""
    pr = synth.sinusoid_pair()
    kw = dict(lam=5.0, levels=3, warps=5, iters=50, c=50.0, c_adapt_iters=30)
    u, v, st, ru, rv, rst = _both(ctx, orc, pr, kw, precision=prec, fp32_flow=1, fp32_last_warp=1)
    assert rst["adapt_margin"] > 0.1
    assert st["c"] == pytest.approx(rst["c_final"], rel=1e-6)
    assert np.hypot(u - ru, v - rv).mean() <= 1e-2


def test_adaptive_step_is_rejected_where_it_does_not_apply(ctx):
    pr = synth.sinusoid_pair()
    I0, I1 = cu(pr.I0), cu(pr.I1)
    for kw in (dict(c_adapt_iters=15), dict(c_adapt_iters=-10), dict(c_adapt_iters=20, method=flow.OF_PDR, gs_sweeps=2),
               dict(c_adapt_iters=20, method=flow.OF_CP), dict(c_adapt_iters=20, engine=flow.OF_ENGINE_PLAIN)):
        with pytest.raises(flow.OfError) as e:
            flow.of_solve(ctx, I0, I1, flow.default_params(**kw))
        assert e.value.status == flow.OF_EINVAL, kw
    P = flow.default_params(c_adapt_iters=20)
    with pytest.raises(flow.OfError) as e:
        flow.of_solve_batch(ctx, [I0, I0], [I1, I1], P)
    assert e.value.status == flow.OF_EINVAL
    with pytest.raises(flow.OfError) as e:
        flow.of_server_start(ctx, P, 0, 2)
    assert e.value.status == flow.OF_EINVAL


# ------------------------------------------------------------------ pDR: sigma and tau, sigma tau fixed
@pytest.mark.parametrize("engine", ["fused", "stream"])
@pytest.mark.parametrize("kw", [dict(sigma=32.0, tau=0.025), dict(sigma=0.125, tau=6.4),
                                dict(sigma=2.0, tau=0.4, beta=0.0)])
def test_pdr_adaptive_steps_match_the_oracle(ctx, orc, engine, kw):
    """pDR from a sigma / tau ratio far too large, far too small and the paper's: the window runs on
    the one-launch tile kernel, the rest of each warp on the level's engine (level-resident on the
    coarse levels with the fused engine).  The final sigma must be the oracle's (each decision at
    least 1% from a tie) and the flows meet the schedule bar."""
    pr = synth.sinusoid_pair()
    P = dict(method=2, lam=5.0, levels=3, warps=3, iters=40, c_adapt_iters=30, **kw)
    u, v, st, ru, rv, rst = _both(ctx, orc, pr, P, ENGINES[engine])
    assert rst["adapt_margin"] > MARGIN, rst["adapt_margin"]
    assert st["c"] == pytest.approx(rst["c_final"], rel=1e-6)
    du, dv = np.abs(u - ru), np.abs(v - rv)
    assert du.max() <= 1e-3 and dv.max() <= 1e-3 and np.hypot(u - ru, v - rv).mean() <= 1e-2
    assert st["iters_run"] == rst["iters_run"]


def test_pdr_adaptive_engines_agree_bitwise(ctx):
    pr = synth.random_affine_rect_pair(150, 210, 5)
    out = []
    for eng in (flow.OF_ENGINE_FUSED, flow.OF_ENGINE_STREAM, flow.OF_ENGINE_RESIDENT):
        P = flow.default_params(method=flow.OF_PDR, lam=5.0, levels=3, warps=2, iters=40, sigma=32.0, tau=0.025,
                                c_adapt_iters=20, engine=eng)
        u, v, _, st = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), P)
        out.append((u, v, st["c"]))
    for u, v, c in out[1:]:
        assert torch.equal(u, out[0][0]) and torch.equal(v, out[0][1]) and c == out[0][2]
