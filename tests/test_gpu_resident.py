"""Level-resident engine: one thread-block cluster per pair keeps a pyramid level in shared memory
and runs all inner iterations of a warp (rpADMMI / rpADMMII / Zach, Sec. 3.1.1, with the stopping
rule) in one launch.  It evaluates the same per-pixel expressions as the streaming engine (one
kernel per iteration) and rounds the state to the storage type where the streaming engine's stores
do, so the flows agree bit for bit in every storage precision; against the FP64 oracle it meets
the same bounds as the streaming engine."""
import numpy as np
import pytest
import torch

from paper_2011_10979_gb300 import flow, synth

pytestmark = pytest.mark.gpu

METHODS = {
    "padmm": dict(method=0, r=1.0),
    "rpadmm1": dict(method=0, r=1.618),
    "rpadmm2": dict(method=1, rho=1.9),
    "zach": dict(method=0, r=1.0, beta=0.0),
    "alg1": dict(method=3),
    "alg1_beta0": dict(method=3, beta=0.0),
    "pdr": dict(method=2),
    "pdr_beta0_2sweeps": dict(method=2, beta=0.0, gs_sweeps=2),
}
FUSED, STREAM, RESIDENT = flow.OF_ENGINE_FUSED, flow.OF_ENGINE_STREAM, flow.OF_ENGINE_RESIDENT


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = flow.Context(0)
    yield c
    c.close()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _both(ctx, pr, **kw):
    out = []
    for eng in (RESIDENT, STREAM):
        u, v, _, st = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), flow.default_params(engine=eng, **kw))
        out.append((u, v, st))
    return out


@pytest.mark.parametrize("name", list(METHODS))
@pytest.mark.parametrize("tol", [0.0, 3e-3])
@pytest.mark.parametrize("prec,fp32_flow", [(0, 1), (1, 1), (2, 1), (2, 0)])
def test_resident_equals_streaming(ctx, name, tol, prec, fp32_flow):
    """The 64 x 48 pair, 3 levels (every level resident) against the streaming engine, FP32 and
    16-bit storage (the finest level's last warp in FP32, as by default)."""
    pr = synth.sinusoid_pair()
    (u0, v0, s0), (u1, v1, s1) = _both(ctx, pr, lam=2.0, tol=tol, levels=3, warps=3, iters=40, precision=prec,
                                       fp32_flow=fp32_flow, **METHODS[name])
    assert torch.equal(u0, u1) and torch.equal(v0, v1)
    assert s0["iters_run"] == s1["iters_run"]
    assert s0["residual"] == pytest.approx(s1["residual"], rel=1e-5, abs=1e-12)
    assert s0["energy"] == pytest.approx(s1["energy"], rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("H,W", [(1, 1), (1, 200), (200, 1), (3, 200), (17, 33), (30, 40), (120, 160),
                                 (224, 200), (1, 1000)])
@pytest.mark.parametrize("name", ["padmm", "alg1", "pdr"])
def test_resident_shapes(ctx, H, W, name):
    """One level, shapes from a single pixel to the largest bands the shared memory holds (224 x 200:
    14 rows of 200 pixels per CTA plus two ghost rows; one row of 1000 plus ghost rows), rows fewer than the
    cluster's CTAs, single rows and columns."""
    pr = synth.random_affine_rect_pair(H, W, 11)
    (u0, v0, s0), (u1, v1, s1) = _both(ctx, pr, lam=2.0, levels=1, warps=2, iters=25, **METHODS[name])
    assert torch.equal(u0, u1) and torch.equal(v0, v1)
    assert s0["iters_run"] == s1["iters_run"] == 50


@pytest.mark.parametrize("name", ["padmm", "rpadmm2", "zach", "alg1", "pdr"])
def test_resident_vs_oracle_largest_band(ctx, orc, name):
    """The largest level the cluster's shared memory holds (224 x 200; pDR, with 21 planes per
    pixel, 150 x 150), 2 warps x 50 iterations, against the FP64 oracle."""
    H, W = (150, 150) if name == "pdr" else (224, 200)
    pr = synth.random_affine_rect_pair(H, W, 5)
    kw = dict(lam=5.0, levels=1, warps=2, iters=50, **METHODS[name])
    u, v, _, st = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), flow.default_params(engine=RESIDENT, **kw))
    ru, rv, _, rst = orc.solve(pr.I0, pr.I1, orc.Params(**kw))
    u, v = u.cpu().double().numpy(), v.cpu().double().numpy()
    assert np.abs(u - ru).max() <= 1e-3 and np.abs(v - rv).max() <= 1e-3
    assert np.hypot(u - ru, v - rv).mean() <= 1e-2
    assert st["iters_run"] == rst["iters_run"]


@pytest.mark.parametrize("prec", [flow.OF_PREC_FP32, flow.OF_PREC_BF16])
@pytest.mark.parametrize("tol", [0.0, 3e-3])
@pytest.mark.parametrize("engine", [FUSED, RESIDENT])
@pytest.mark.parametrize("name", ["padmm", "alg1", "pdr"])
def test_mixed_batch_equals_single(ctx, prec, tol, engine, name):
    """A batch whose levels are resident for some pairs and streamed for others (320 x 240 is
    above the resident size) equals the single-pair solves bit for bit."""
    pairs = [synth.sinusoid_pair(seed=1), synth.random_affine_rect_pair(240, 320, 3),
             synth.random_affine_rect_pair(120, 160, 4),
             synth.Pair(np.full((1, 1), 0.5, np.float32), np.full((1, 1), 0.25, np.float32), None, None)]
    P = flow.default_params(lam=2.0, precision=prec, tol=tol, levels=3, warps=3, iters=30, engine=engine,
                            **METHODS[name])
    us, vs, sts = flow.of_solve_batch(ctx, [cu(p.I0) for p in pairs], [cu(p.I1) for p in pairs], P)
    for p, u, v, st in zip(pairs, us, vs, sts):
        su, sv, _, sst = flow.of_solve(ctx, cu(p.I0), cu(p.I1), P)
        assert torch.equal(u, su) and torch.equal(v, sv)
        assert st["iters_run"] == sst["iters_run"]


def test_resident_kernel_count(ctx):
    """A resident level launches one kernel per warp; the streaming engine one per inner iteration
    (with a pinned strip height; by the built-in rule and a fixed schedule one per three
    iterations), an iteration count per warp and the final residual sum."""
    P = flow.default_params(lam=2.0, levels=1, warps=3, iters=100, engine=RESIDENT)
    n_res = flow.of_solve_kernel_count(ctx, 48, 64, P)
    P.engine = STREAM
    P.rows_per_warp = 2
    n_str = flow.of_solve_kernel_count(ctx, 48, 64, P)
    assert n_str - n_res == 3 * (100 + 1 - 1) + 1
    P.rows_per_warp = 0   # 33 launches of three iterations and one single-iteration launch per warp
    assert flow.of_solve_kernel_count(ctx, 48, 64, P) - n_res == 3 * (34 + 1 - 1) + 1
    P.iters = 101  # 33 launches of three and one of two
    P.engine = RESIDENT
    n_res = flow.of_solve_kernel_count(ctx, 48, 64, P)
    P.engine = STREAM
    assert flow.of_solve_kernel_count(ctx, 48, 64, P) - n_res == 3 * (34 + 1 - 1) + 1


def test_large_batch_streams_small_levels(ctx):
    """More eligible pairs than resident clusters run at once: the batch streams the level (one
    work-list launch per iteration) and still equals the single-pair (resident) solves."""
    pairs = [synth.sinusoid_pair(seed=s) for s in range(12)]
    P = flow.default_params(lam=2.0, levels=2, warps=2, iters=20, engine=RESIDENT)
    us, vs, sts = flow.of_solve_batch(ctx, [cu(p.I0) for p in pairs], [cu(p.I1) for p in pairs], P)
    for p, u, v in zip(pairs, us, vs):
        su, sv, _, _ = flow.of_solve(ctx, cu(p.I0), cu(p.I1), P)
        assert torch.equal(u, su) and torch.equal(v, sv)
