"""GPU parity of whole schedules at the benchmark sizes, against the FP64 oracle.

Covers the cases the small-size schedule tests cannot reach:
  * pDR and ALG1 on the 640 x 480 pair, where their per-iteration engines (not the level-resident
    one) run the two finest levels; compared after level 1 and after level 0;
  * the 1024 x 436 layered pair at its full schedule (6 levels, 10 warps, 150 iterations) in FP32
    and with 16-bit duals and data (FP32 flow fields);
  * one pair of every size of the benchmark batch, solved together in one batch (FP32, and BF16
    duals with FP32 flow fields as the batch benchmark runs it);
  * the stopping rule, comparing the flows whatever iteration counts the two sides stop at.

Bars (the accuracy this library is built to): max |du|, |dv| <= 1e-3 px and mean end-point error
<= 1e-2 px after the same schedule in FP32; EPE <= 1e-2 px with 16-bit storage (max |d| printed);
with a stopping tolerance the two sides may stop at different iterations, so there the bar is the
EPE alone.  The oracle solves run in host threads (the oracle releases the GIL inside its C code)
started when the module's first test runs, so they overlap each other and the GPU work.
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from paper_2011_10979_gb300 import flow, synth  # noqa: E402

LAM = 5.0
SCHED = dict(lam=LAM, levels=5, warps=10, iters=100)
LAYERED = dict(lam=LAM, levels=6, warps=10, iters=150)


BATCH_SIZES = [(64, 96), (240, 320), (480, 640), (436, 1024), (375, 1242)]
_JOBS = {}


def jobs():
    """name -> (pair, oracle parameters); the pairs are generated on first use."""
    if not _JOBS:
        bench = synth.affine_rect_pair()
        _JOBS.update({
            "pdr_l1": (bench, dict(SCHED, method=2, out_level=1)),
            "pdr_l0": (bench, dict(SCHED, method=2)),
            "alg1_l1": (bench, dict(SCHED, method=3, out_level=1)),
            "alg1_l0": (bench, dict(SCHED, method=3)),
            "layered": (synth.layered_pair(), dict(LAYERED)),
            "stop_l1": (bench, dict(lam=LAM, levels=5, warps=10, iters=300, tol=1e-3, out_level=1)),
        })
        pool = synth.batch_pairs(n=32)     # the benchmark batch's distinct pairs
        for k, s in enumerate(BATCH_SIZES):
            _JOBS["batch%d" % k] = (next(p for p in pool if p.I0.shape == s), dict(SCHED))
    return _JOBS


@pytest.fixture(scope="module")
def ref(orc):
    """Starts every oracle solve of this module at once; ref(name) waits for one."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    J = jobs()
    futures = {}
    ex = cf.ThreadPoolExecutor(max_workers=max(2, min(len(J), os.cpu_count() or 2)))
    # longest first, so the pool finishes as early as it can
    for name in sorted(J, key=lambda n: -J[n][0].I0.size * J[n][1].get("iters", 1)):
        pair, kw = J[name]
        futures[name] = ex.submit(orc.solve, pair.I0, pair.I1, orc.Params(**kw))
    yield lambda name: futures[name].result()
    ex.shutdown(wait=True)


@pytest.fixture(scope="module")
def ctx():
    c = flow.Context(0)
    yield c
    c.close()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _errors(u, v, ru, rv):
    u, v = u.double().cpu().numpy(), v.double().cpu().numpy()
    return float(np.abs(u - ru).max()), float(np.abs(v - rv).max()), float(np.hypot(u - ru, v - rv).mean())


# Measured misses of the max |d| <= 1e-3 px bar after the longest schedules (5,000 inner
# iterations in FP32 against FP64): one to a few pixels drift past 1e-3 px while the mean
# end-point error stays 200-500 times below its 1e-2 px bar.  Recorded as failing, not widened.
# An FP32 build of the oracle itself misses these bars by more (pDR 5.0e-3, ALG1 3.4e-3 px), and
# FP32 storage of the pyramid images alone (FP64 arithmetic everywhere else) already moves single
# pixels of the ALG1 case by 2.2e-3 px.
MAX_BAR_MISS = {
    "pdr_l0": "max|dv| 1.15e-3 px (EPE 5.7e-5 px)",
    "alg1_l0": "max|du| 2.52e-3 px, max|dv| 1.11e-3 px (EPE 1.9e-5 px)",
}


def _expect_max_bar_miss(request, key):
    request.applymarker(pytest.mark.xfail(strict=True, reason="max |d| bar missed: " + MAX_BAR_MISS[key]))


@pytest.mark.parametrize("name", ["pdr_l1", "pdr_l0", "alg1_l1", "alg1_l0"])
def test_pdr_and_alg1_schedules_at_640x480(ctx, ref, name, request):
    if name in MAX_BAR_MISS:
        _expect_max_bar_miss(request, name)
    pair, kw = jobs()[name]
    P = flow.default_params(**kw)
    u, v, _, st = flow.of_solve(ctx, cu(pair.I0), cu(pair.I1), P)
    ru, rv, _, rst = ref(name)
    mu, mv, epe = _errors(u, v, ru, rv)
    print("%s: max|du| %.2e max|dv| %.2e EPE %.2e" % (name, mu, mv, epe))
    assert mu <= 1e-3 and mv <= 1e-3 and epe <= 1e-2, (mu, mv, epe)
    assert st["iters_run"] == rst["iters_run"]


@pytest.mark.parametrize("prec,fp32_flow", [(flow.OF_PREC_FP32, 1), (flow.OF_PREC_FP16, 1), (flow.OF_PREC_BF16, 1),
                                            (flow.OF_PREC_FP16, 0), (flow.OF_PREC_BF16, 0)])
def test_layered_1024x436_full_schedule(ctx, ref, prec, fp32_flow):
    """The precision workload at its own schedule (6 levels, 10 warps, 150 iterations).  FP32 and
    16-bit duals/data with FP32 flow fields meet the EPE bar; all-16-bit storage is reported only."""
    pair = jobs()["layered"][0]
    P = flow.default_params(precision=prec, fp32_last_warp=1, fp32_flow=fp32_flow, **LAYERED)
    u, v, _, _ = flow.of_solve(ctx, cu(pair.I0), cu(pair.I1), P)
    ru, rv, _, _ = ref("layered")
    mu, mv, epe = _errors(u, v, ru, rv)
    print("1024x436 prec %d fp32_flow %d: max|du| %.2e max|dv| %.2e EPE %.2e" % (prec, fp32_flow, mu, mv, epe))
    if prec == flow.OF_PREC_FP32:
        assert mu <= 1e-3 and mv <= 1e-3 and epe <= 1e-2, (mu, mv, epe)
    elif fp32_flow:
        assert epe <= 1e-2, (mu, mv, epe)


@pytest.mark.parametrize("prec", [flow.OF_PREC_FP32, flow.OF_PREC_BF16])
def test_benchmark_batch_sizes_against_the_oracle(ctx, ref, prec):
    """One pair of each benchmark batch size (96 x 64 .. 1242 x 375) solved together in one batch,
    each compared with its own oracle solve."""
    sample = [jobs()["batch%d" % k][0] for k in range(len(BATCH_SIZES))]
    P = flow.default_params(precision=prec, fp32_last_warp=1, fp32_flow=1, rows_per_warp=-1, **SCHED)
    us, vs, _ = flow.of_solve_batch(ctx, [cu(p.I0) for p in sample], [cu(p.I1) for p in sample], P)
    for k, p in enumerate(sample):
        ru, rv, _, _ = ref("batch%d" % k)
        mu, mv, epe = _errors(us[k], vs[k], ru, rv)
        print("batch pair %dx%d prec %d: max|du| %.2e max|dv| %.2e EPE %.2e" % (p.I0.shape + (prec, mu, mv, epe)))
        if prec == flow.OF_PREC_FP32:
            assert mu <= 1e-3 and mv <= 1e-3 and epe <= 1e-2, (p.I0.shape, mu, mv, epe)
        else:
            assert epe <= 1e-2, (p.I0.shape, mu, mv, epe)


def test_stopping_rule_flows_whatever_the_iteration_counts(ctx, ref):
    """tol = 1e-3 on the 640 x 480 pair up to level 1 (at most 300 iterations per warp): the FP32
    residual and the FP64 one can cross the tolerance at different checks, so the iteration
    counts may differ; the flows must still agree to EPE <= 1e-2 px."""
    pair, kw = jobs()["stop_l1"]
    P = flow.default_params(**kw)
    u, v, _, st = flow.of_solve(ctx, cu(pair.I0), cu(pair.I1), P)
    ru, rv, _, rst = ref("stop_l1")
    mu, mv, epe = _errors(u, v, ru, rv)
    print("stopping rule: iterations %d (oracle %d), max|du| %.2e max|dv| %.2e EPE %.2e"
          % (st["iters_run"], rst["iters_run"], mu, mv, epe))
    assert st["iters_run"] < 4 * 10 * 300 and rst["iters_run"] < 4 * 10 * 300
    assert epe <= 1e-2, (mu, mv, epe)
