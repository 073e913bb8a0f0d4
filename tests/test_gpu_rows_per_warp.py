"""Strip height of the streaming ADMM kernel (rows each warp finishes per inner iteration of
Sec. 3.1.1's rpADMMI / rpADMMII / beta = 0 model) and its autotuner.  The height only changes how
the work is cut into warps, so every height gives bitwise the same flow and the same iteration
counts; only the grouping of the residual's partial sums changes (each lane adds its strip's rows
in FP32, blocks in FP64), so the residual agrees to FP32 rounding.  Each height is also checked
against the FP64 oracle on a level several strips wide and tall, with ragged right and bottom
edges."""
import numpy as np
import pytest
import torch

from paper_2011_10979_gb300 import flow, synth

pytestmark = pytest.mark.gpu

HEIGHTS = (1, 2, 8, 32)
METHODS = {
    "padmm": dict(method=0, r=1.0),
    "rpadmm2": dict(method=1, rho=1.9),
    "zach": dict(method=0, beta=0.0),
    "padmm_pp": dict(method=0, a_tilde_mode=1),
}
STREAM = flow.OF_ENGINE_STREAM


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = flow.Context(0)
    yield c
    c.close()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _solve(ctx, pr, **kw):
    return flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), flow.default_params(**kw))


@pytest.mark.parametrize("prec", [flow.OF_PREC_FP32, flow.OF_PREC_BF16])
@pytest.mark.parametrize("name", list(METHODS))
@pytest.mark.parametrize("H,W", [(1, 1), (3, 200), (17, 33), (45, 61), (130, 250), (480, 640)])
def test_every_height_gives_the_same_flow(ctx, H, W, name, prec):
    """One level per shape on the streaming engine: a single pixel, fewer rows than one strip,
    ragged strips and row groups, and a level 23 strips wide and 480 rows tall."""
    pr = synth.random_affine_rect_pair(H, W, 7)
    kw = dict(lam=2.0, levels=1, warps=2, iters=20, engine=STREAM, precision=prec, **METHODS[name])
    u0, v0, _, s0 = _solve(ctx, pr, rows_per_warp=0, **kw)
    for ty in HEIGHTS:
        u, v, _, st = _solve(ctx, pr, rows_per_warp=ty, **kw)
        assert torch.equal(u, u0) and torch.equal(v, v0), ty
        assert st["iters_run"] == s0["iters_run"] == 40
        assert st["residual"] == pytest.approx(s0["residual"], rel=1e-6, abs=1e-15)
        assert st["energy"] == pytest.approx(s0["energy"], rel=1e-9, abs=1e-15)


@pytest.mark.parametrize("ty", HEIGHTS)
def test_every_height_vs_oracle(ctx, orc, ty):
    """A 150 x 200 level (7 strips, ragged on the right; 150 rows, ragged for every height),
    2 warps x 50 iterations, against the FP64 oracle at the flow tolerance of the solve tests."""
    pr = synth.random_affine_rect_pair(150, 200, 5)
    kw = dict(lam=5.0, levels=1, warps=2, iters=50)
    u, v, _, st = _solve(ctx, pr, engine=STREAM, rows_per_warp=ty, **kw)
    ru, rv, _, rst = orc.solve(pr.I0, pr.I1, orc.Params(**kw))
    u, v = u.cpu().double().numpy(), v.cpu().double().numpy()
    assert np.abs(u - ru).max() <= 1e-3 and np.abs(v - rv).max() <= 1e-3
    assert np.hypot(u - ru, v - rv).mean() <= 1e-2
    assert st["iters_run"] == rst["iters_run"]


@pytest.mark.parametrize("tol", [0.0, 3e-3])
def test_stopping_rule_is_height_independent(ctx, tol):
    """With the stopping test on, every height stops each warp after the same iteration."""
    pr = synth.random_affine_rect_pair(240, 320, 9)
    kw = dict(lam=2.0, levels=2, warps=3, iters=60, tol=tol, engine=STREAM)
    u0, v0, _, s0 = _solve(ctx, pr, rows_per_warp=0, **kw)
    for ty in HEIGHTS + (-1,):
        u, v, _, st = _solve(ctx, pr, rows_per_warp=ty, **kw)
        assert torch.equal(u, u0) and torch.equal(v, v0), ty
        assert st["iters_run"] == s0["iters_run"]


@pytest.mark.parametrize("ty", HEIGHTS + (-1,))
def test_batch_every_height_equals_single(ctx, ty):
    """Batched work-lists built for each height (and the autotuned one) give the single-pair
    flows bit for bit; the 1 x 1 and 64 x 48 pairs run level-resident, the others streamed."""
    pairs = [synth.random_affine_rect_pair(240, 320, 3), synth.sinusoid_pair(seed=1),
             synth.random_affine_rect_pair(130, 250, 4), synth.random_affine_rect_pair(436, 1024, 6),
             synth.Pair(np.full((1, 1), 0.5, np.float32), np.full((1, 1), 0.25, np.float32), None, None)]
    P = flow.default_params(lam=2.0, levels=3, warps=2, iters=20, rows_per_warp=ty)
    us, vs, sts = flow.of_solve_batch(ctx, [cu(p.I0) for p in pairs], [cu(p.I1) for p in pairs], P)
    P0 = flow.default_params(lam=2.0, levels=3, warps=2, iters=20)
    for p, u, v, st in zip(pairs, us, vs, sts):
        su, sv, _, sst = flow.of_solve(ctx, cu(p.I0), cu(p.I1), P0)
        assert torch.equal(u, su) and torch.equal(v, sv)
        assert st["iters_run"] == sst["iters_run"]
    # levels 0 and 1 stream some pairs; on level 2 every pair runs level-resident
    rows = flow.of_rows_per_warp(ctx, [p.I0.shape for p in pairs], P)
    assert rows[0] in HEIGHTS and rows[1] in HEIGHTS and rows[2] == 0
    if ty > 0:
        assert rows == [ty, ty, 0]


def test_autotuned_single_pair(ctx):
    """640 x 480, 5 levels, default engine: the two levels above the resident size are tuned to
    one of the kernel's heights and the three resident levels report 0; the tuned solve equals the
    built-in rule's bit for bit and the tuning is kept by the context.  The built-in rule runs the
    tile kernel (three iterations per launch) on the three levels above 7,000 px (the 160x120
    level included), so it launches fewer kernels."""
    P = flow.default_params(lam=5.0, levels=5, warps=2, iters=10, rows_per_warp=-1)
    rows = flow.of_rows_per_warp(ctx, [(480, 640)], P)
    assert rows[0] in HEIGHTS and rows[1] in HEIGHTS and rows[2:] == [0, 0, 0]
    P0 = flow.default_params(lam=5.0, levels=5, warps=2, iters=10)
    built_in = flow.of_rows_per_warp(ctx, [(480, 640)], P0)
    assert all(r in HEIGHTS for r in built_in[:3]) and built_in[3:] == [0, 0]
    pr = synth.affine_rect_pair()
    u, v, _, st = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), P)
    u0, v0, _, s0 = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), P0)
    assert torch.equal(u, u0) and torch.equal(v, v0)
    assert st["iters_run"] == s0["iters_run"]
    assert flow.of_rows_per_warp(ctx, [(480, 640)], P) == rows
    # levels 0 and 1: 10 iterations in 4 tile launches instead of 10 (2 x 2 x 6 fewer); level 2:
    # 4 tile launches and an iteration count per warp instead of one resident launch (2 x 4 more)
    assert flow.of_solve_kernel_count(ctx, 480, 640, P) == flow.of_solve_kernel_count(ctx, 480, 640, P0) + 24 - 8


def test_rows_report_for_other_kernels(ctx):
    """ALG1 and pDR with two sweeps report the block height of their one-iteration kernels on the
    levels they stream (8 by default) and 0 on the level-resident one (pDR: 160x120; ALG1 streams
    it, its tile kernel being faster there); pDR with one sweep (its one-launch tile kernel), the
    plain engine and levels below out_level report 0."""
    pdr2 = flow.default_params(levels=3, method=flow.OF_PDR, gs_sweeps=2)
    assert flow.of_rows_per_warp(ctx, [(480, 640)], pdr2) == [8, 8, 0]
    assert flow.of_rows_per_warp(ctx, [(480, 640)], flow.default_params(levels=3, method=flow.OF_CP)) == [8, 8, 8]
    assert flow.of_rows_per_warp(ctx, [(480, 640)], flow.default_params(levels=3, method=flow.OF_PDR)) == [0, 0, 0]
    plain = flow.default_params(levels=3, engine=flow.OF_ENGINE_PLAIN)
    assert flow.of_rows_per_warp(ctx, [(480, 640)], plain) == [0, 0, 0]
    rows = flow.of_rows_per_warp(ctx, [(480, 640)], flow.default_params(levels=3, out_level=1, rows_per_warp=8))
    assert rows == [0, 8, 0]
    with pytest.raises(flow.OfError):
        flow.of_rows_per_warp(ctx, [(480, 640)], flow.default_params(rows_per_warp=4))


# ------------------------------------------------------------------ pDR / ALG1 block heights
BLOCK_HEIGHTS = (4, 8, 16)


@pytest.mark.parametrize("method", [2, 3])
@pytest.mark.parametrize("beta", [0.05, 0.0])
def test_pdr_and_alg1_block_heights_give_the_same_flow(ctx, method, beta):
    """The pDR and ALG1 per-iteration kernels run blocks of 32 columns by 4, 8 or 16 rows (the
    autotuner's choice): every height computes every pixel alike, so the flows are bitwise equal,
    on a level with ragged right and bottom edges, single and batched."""
    pr = synth.random_affine_rect_pair(203, 333, 21)
    kw = dict(lam=2.0, levels=2, warps=2, iters=17, method=method, beta=beta, engine=STREAM)
    if method == 2:
        kw["gs_sweeps"] = 2  # one sweep runs the one-launch tile kernel, which has no height
    ref = _solve(ctx, pr, rows_per_warp=0, **kw)
    for h in BLOCK_HEIGHTS + (-1,):
        got = _solve(ctx, pr, rows_per_warp=h, **kw)
        assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1]), h
        assert got[3]["iters_run"] == ref[3]["iters_run"]
    P = flow.default_params(rows_per_warp=-1, **kw)
    rows = flow.of_rows_per_warp(ctx, [pr.I0.shape], P)
    assert all(r in BLOCK_HEIGHTS for r in rows), rows
    pairs = [pr, synth.random_affine_rect_pair(64, 96, 22), synth.random_affine_rect_pair(130, 100, 23)]
    for h in (4, 16, -1):
        Pb = flow.default_params(rows_per_warp=h, **kw)
        us, vs, _ = flow.of_solve_batch(ctx, [cu(p.I0) for p in pairs], [cu(p.I1) for p in pairs], Pb)
        assert torch.equal(us[0], ref[0]) and torch.equal(vs[0], ref[1]), h


def test_block_heights_are_validated_per_method(ctx):
    pr = synth.sinusoid_pair()
    for method, bad in ((2, 2), (3, 32), (0, 4), (1, 16)):
        with pytest.raises(flow.OfError) as e:
            _solve(ctx, pr, method=method, rows_per_warp=bad)
        assert e.value.status == flow.OF_EINVAL
