"""Several ALG1 iterations per launch (k_cp_tile: three, the last launch of a warp two or one;
single pairs with the built-in block height) against one launch per iteration of k_cp (a pinned
block height): the state between the iterations is rounded where k_cp's stores round it, so the
flows are bitwise equal, on tiles with ragged edges, both tile sizes, beta > 0 and beta = 0,
16-bit storage, iteration counts that end a warp with launches of one, two and three iterations,
and with the stopping test."""
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


def _pair(H, W, seed):
    if min(H, W) > 8:
        return synth.random_affine_rect_pair(H, W, seed)
    rng = np.random.default_rng(seed)
    return synth.Pair(rng.random((H, W)).astype(np.float32), rng.random((H, W)).astype(np.float32), None, None)


def _solve(ctx, pr, **kw):
    return flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), flow.default_params(method=flow.OF_CP, **kw), want_w=True)


def _equal(a, b, w=True):
    return torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) and (not w or torch.equal(a[2], b[2]))


@pytest.mark.parametrize("H,W", [(1, 1), (3, 200), (200, 3), (37, 53), (203, 333), (480, 640), (436, 1024)])
@pytest.mark.parametrize("beta", [0.05, 0.0])
@pytest.mark.parametrize("iters", [21, 22, 23, 24])
def test_alg1_iterations_per_launch_equal_single_launches(ctx, H, W, beta, iters):
    pr = _pair(H, W, 7 + W)
    kw = dict(lam=2.0, beta=beta, levels=1, warps=2, iters=iters, engine=flow.OF_ENGINE_STREAM)
    a = _solve(ctx, pr, rows_per_warp=8, **kw)
    b = _solve(ctx, pr, rows_per_warp=0, **kw)
    assert _equal(a, b, w=beta != 0.0)
    assert b[3]["iters_run"] == a[3]["iters_run"] == 2 * iters
    assert b[3]["residual"] == pytest.approx(a[3]["residual"], rel=1e-5, abs=1e-12)
    assert b[3]["energy"] == pytest.approx(a[3]["energy"], rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("prec,fp32_flow", [(1, 1), (2, 1), (2, 0), (1, 0)])
def test_alg1_iterations_per_launch_on_16bit_storage(ctx, prec, fp32_flow):
    pr = synth.affine_rect_pair(240, 320)
    kw = dict(lam=5.0, levels=2, warps=3, iters=30, precision=prec, fp32_flow=fp32_flow, engine=flow.OF_ENGINE_STREAM)
    assert _equal(_solve(ctx, pr, rows_per_warp=8, **kw), _solve(ctx, pr, rows_per_warp=0, **kw))


def test_alg1_whole_solve_against_single_launches(ctx):
    """The bench workload's schedule shape (5 levels) on the 640x480 pair: the default engine (three
    iterations per launch on the streamed levels, level-resident below) against a pinned block
    height (one launch per iteration where not resident)."""
    pr = synth.affine_rect_pair()
    kw = dict(lam=5.0, levels=5, warps=3, iters=41)
    assert _equal(_solve(ctx, pr, **kw), _solve(ctx, pr, rows_per_warp=8, **kw))


@pytest.mark.parametrize("H,W", [(37, 53), (480, 640)])
@pytest.mark.parametrize("iters", [40, 25])
@pytest.mark.parametrize("stop", ["never", "met"])
def test_alg1_stopping_rule_on_the_tile_path(ctx, H, W, iters, stop):
    """tol > 0: launches of 3, 3, 3 and 1 per ten iterations (the tested one on k_cp) against one
    launch per iteration, bitwise, with the same iterations run."""
    pr = _pair(H, W, 3 + H)
    kw = dict(lam=2.0, levels=1, warps=2, iters=iters, engine=flow.OF_ENGINE_STREAM)
    if stop == "never":
        tol = 1e-30
    else:
        tol = _solve(ctx, pr, **dict(kw, warps=1, iters=20, rows_per_warp=8))[3]["residual"] * 1.001
    a = _solve(ctx, pr, rows_per_warp=8, tol=tol, **kw)
    b = _solve(ctx, pr, rows_per_warp=0, tol=tol, **kw)
    assert _equal(a, b)
    assert b[3]["iters_run"] == a[3]["iters_run"]
    assert (a[3]["iters_run"] == 2 * iters) if stop == "never" else (a[3]["iters_run"] < 2 * iters)


def test_alg1_launch_counts(ctx):
    """Forty iterations on one 640x480 level: 14 launches on the tile path (13 of three iterations
    and one of one) against 40 with a pinned block height."""
    P = flow.default_params(method=flow.OF_CP, lam=5.0, levels=1, warps=1, iters=40, engine=flow.OF_ENGINE_STREAM)
    n_tile = flow.of_solve_kernel_count(ctx, 480, 640, P)
    P.rows_per_warp = 8
    n_rows = flow.of_solve_kernel_count(ctx, 480, 640, P)
    assert n_rows - n_tile == 40 - 14
