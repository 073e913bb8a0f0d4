"""Several ADMM inner iterations per launch (k_admm_tile2: three, the last launch of a warp two or
one; single pairs with a fixed schedule and the built-in strip rule) against one launch per
iteration of the row-streaming kernel (a pinned strip height) and the persistent engine: the state
between the iterations is rounded where the streaming kernel's stores round it, so the flows are
bitwise equal, on tiles with ragged edges, both tile sizes, every ADMM variant, 16-bit storage and
iteration counts that end a warp with launches of one, two and three iterations, with and without
the stopping test."""
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


VARIANTS = {"padmm": dict(method=0), "rpadmm1": dict(method=0, r=1.618), "rpadmm2": dict(method=1, rho=1.9),
            "zach": dict(method=0, beta=0.0), "padmm_pp": dict(method=0, a_tilde_mode=1)}


def _pair(H, W, seed):
    if min(H, W) > 8:
        return synth.random_affine_rect_pair(H, W, seed)
    rng = np.random.default_rng(seed)
    return synth.Pair(rng.random((H, W)).astype(np.float32), rng.random((H, W)).astype(np.float32), None, None)


def _solve(ctx, pr, **kw):
    u, v, w, st = flow.of_solve(ctx, cu(pr.I0), cu(pr.I1), flow.default_params(**kw), want_w=True)
    return u, v, w, st


@pytest.mark.parametrize("H,W", [(1, 1), (3, 200), (200, 3), (37, 53), (203, 333), (480, 640), (436, 1024), (1080, 1920)])
@pytest.mark.parametrize("name", list(VARIANTS))
@pytest.mark.parametrize("iters", [21, 22, 23, 24])
def test_iterations_per_launch_equal_single_launches(ctx, H, W, name, iters):
    pr = _pair(H, W, 5 + H)
    kw = dict(lam=2.0, levels=1, warps=2, iters=iters, engine=flow.OF_ENGINE_STREAM, **VARIANTS[name])
    u0, v0, w0, s0 = _solve(ctx, pr, rows_per_warp=2, **kw)
    u1, v1, w1, s1 = _solve(ctx, pr, rows_per_warp=0, **kw)
    assert torch.equal(u0, u1) and torch.equal(v0, v1) and torch.equal(w0, w1)
    assert s1["iters_run"] == s0["iters_run"] == 2 * iters
    assert s1["residual"] == pytest.approx(s0["residual"], rel=1e-5, abs=1e-12)
    assert s1["energy"] == pytest.approx(s0["energy"], rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("prec,fp32_flow", [(1, 1), (2, 1), (2, 0), (1, 0)])
def test_iterations_per_launch_on_16bit_storage(ctx, prec, fp32_flow):
    pr = synth.affine_rect_pair(240, 320)
    kw = dict(lam=5.0, levels=2, warps=3, iters=30, precision=prec, fp32_flow=fp32_flow, engine=flow.OF_ENGINE_STREAM)
    a = _solve(ctx, pr, rows_per_warp=8, **kw)
    b = _solve(ctx, pr, rows_per_warp=0, **kw)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_whole_solve_against_the_persistent_engine(ctx):
    """The bench workload's schedule shape (5 levels) on the 640x480 pair: the default engine (three
    iterations per launch on its two streamed levels, resident below) against the persistent
    engine (every iteration of a warp in one launch, the row-streaming pipeline)."""
    pr = synth.affine_rect_pair()
    kw = dict(lam=5.0, levels=5, warps=3, iters=41)
    a = _solve(ctx, pr, engine=flow.OF_ENGINE_FUSED, **kw)
    b = _solve(ctx, pr, engine=flow.OF_ENGINE_PERSISTENT, **kw)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def _tol_met_at_20(ctx, pr, kw):
    """A tolerance the residual meets at the check after iteration 20 of a one-warp solve (or at
    the one after iteration 10)."""
    k = dict(kw, warps=1, iters=20, rows_per_warp=2)
    return _solve(ctx, pr, **k)[3]["residual"] * 1.001


@pytest.mark.parametrize("H,W", [(37, 53), (203, 333), (480, 640)])
@pytest.mark.parametrize("iters", [40, 25, 27, 23])
@pytest.mark.parametrize("stop", ["never", "met"])
def test_stopping_rule_on_the_tile_path(ctx, H, W, iters, stop):
    """tol > 0 on the several-iterations path (launches of 3, 3, 3 and 1 per ten iterations, the
    warp's last launch a single iteration) against one launch per iteration: bitwise equal flows
    and the same iterations run, whether the test stops a warp early (the tails
    of 25 and 27 iterations leave an odd number of launches, so the stopped state is copied to the
    final buffer) or never."""
    pr = _pair(H, W, 11 + W)
    kw = dict(lam=2.0, levels=1, warps=2, iters=iters, engine=flow.OF_ENGINE_STREAM)
    tol = 1e-30 if stop == "never" else _tol_met_at_20(ctx, pr, kw)
    u0, v0, w0, s0 = _solve(ctx, pr, rows_per_warp=2, tol=tol, **kw)
    u1, v1, w1, s1 = _solve(ctx, pr, rows_per_warp=0, tol=tol, **kw)
    assert torch.equal(u0, u1) and torch.equal(v0, v1) and torch.equal(w0, w1)
    assert s1["iters_run"] == s0["iters_run"]
    # the same state; the partial sums of its residual group the pixels per strip of the kernel
    # that ran the last iteration (pinned 2-row strips against the built-in height)
    assert s1["residual"] == pytest.approx(s0["residual"], rel=1e-6, abs=1e-12)
    if stop == "never":
        assert s0["iters_run"] == 2 * iters
        u2, v2, _, _ = _solve(ctx, pr, rows_per_warp=0, **kw)
        assert torch.equal(u1, u2) and torch.equal(v1, v2)
    else:
        assert s0["iters_run"] < 2 * iters


def test_stopping_rule_launch_counts(ctx):
    """Forty iterations with the stopping test: 16 iteration launches on the tile path against 40
    with a pinned strip height (each with the same four checks)."""
    P = flow.default_params(lam=5.0, levels=1, warps=1, iters=40, engine=flow.OF_ENGINE_STREAM, tol=1e-30)
    n_tile = flow.of_solve_kernel_count(ctx, 480, 640, P)
    P.rows_per_warp = 2
    n_rows = flow.of_solve_kernel_count(ctx, 480, 640, P)
    assert n_rows - n_tile == 40 - 16
