"""GPU checks of the library's guards: scratch sizing, the resident engine's capacity check and
non-finite inputs.  Each test calls through the C ABI."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2011_10979_gb300 import flow, synth  # noqa: E402

FIELDS = ("w", "u", "v", "p1", "p2", "q11", "q12", "q21", "q22", "s", "wb", "ub", "vb")
GUARD = 4096


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = flow.Context(0)
    yield c
    c.close()


def _pitched(a, pitch):
    H, W = a.shape
    buf = torch.zeros((H, pitch), dtype=torch.float32, device="cuda")
    buf[:, :W] = torch.from_numpy(a.astype(np.float32)).cuda()
    return buf[:, :W]


@pytest.mark.parametrize("kind", ["admm", "pdr", "cp"])
@pytest.mark.parametrize("H,W,pitch", [(97, 2900, 2929), (5, 30, 64), (33, 17, 17)])
def test_step_entry_points_stay_inside_a_scratch_of_of_fields_bytes(ctx, kind, H, W, pitch):
    """A scratch buffer of exactly of_fields_bytes(H, pitch) bytes, followed by a guard region: the
    step-level entry points never touch the guard (the partial sums and device scalars sit at the
    end of the layout, sized for every width up to the pitch)."""
    L = flow.lib()
    rng = np.random.default_rng(H + W)
    st = {k: _pitched(rng.normal(size=(H, W)) * 0.3, pitch) for k in FIELDS}
    Ix, Iy, It = (_pitched(rng.normal(size=(H, W)) * s, pitch) for s in (0.4, 0.4, 0.2))
    n = L.of_fields_bytes(H, pitch)
    buf = torch.full((n + GUARD,), 0xA5, dtype=torch.uint8, device="cuda")
    method = {"admm": 0, "pdr": 2, "cp": 3}[kind]
    P = flow.default_params(method=method, lam=0.3, tol=1e-9)   # tol > 0: the stop flag and counters too
    res = ctypes.c_double(0.0)
    args = (flow._fields(st), Ix.data_ptr(), Iy.data_ptr(), It.data_ptr(), H, W, pitch)
    if kind == "admm":
        rc = L.of_admm_iterate(*args, ctypes.c_float(1.0), ctypes.byref(P), 21, ctypes.c_void_p(buf.data_ptr()),
                               ctypes.byref(res), None)
    else:
        fn = L.of_pdr_iterate if kind == "pdr" else L.of_cp_iterate
        rc = fn(*args, ctypes.byref(P), 21, ctypes.c_void_p(buf.data_ptr()), ctypes.byref(res), None)
    flow.check(rc)
    torch.cuda.synchronize()
    assert bool((buf[n:] == 0xA5).all()), "the call wrote past of_fields_bytes"
    assert np.isfinite(res.value)


def test_resident_engine_takes_a_batch_level_only_when_its_clusters_run_at_once(ctx):
    """The capacity comes from cudaOccupancyMaxActiveClusters; a batch level with as many small
    pairs as clusters run at once goes to the resident engine (no streamed strips), one pair more
    sends every pair of the level to the streaming work-list.  Both give the single-pair flows."""
    nc, active = flow.of_resident_clusters()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert nc in (16, 8) and 1 <= active <= sms // nc, (nc, active)
    P = flow.default_params(lam=2.0, levels=1, warps=2, iters=20)
    for n, resident in ((active, True), (active + 1, False)):
        rows = flow.of_rows_per_warp(ctx, [(30, 40)] * n, P)
        assert (rows[0] == 0) == resident, (n, rows)
    pairs = [synth.random_affine_rect_pair(30, 40, 20 + k) for k in range(active + 1)]
    us, vs, _ = flow.of_solve_batch(ctx, [torch.from_numpy(p.I0).cuda() for p in pairs],
                                    [torch.from_numpy(p.I1).cuda() for p in pairs], P)
    su, sv, _, _ = flow.of_solve(ctx, torch.from_numpy(pairs[0].I0).cuda(), torch.from_numpy(pairs[0].I1).cuda(), P)
    assert torch.equal(us[0], su) and torch.equal(vs[0], sv)


@pytest.mark.parametrize("where", ["I0", "I1"])
def test_non_finite_input_is_reported(ctx, where):
    """NaN or Inf pixels give non-finite residuals and energies, which every call that waits for
    its result reports as OF_ENUMERIC (the warp clamps non-finite sample positions to the image,
    so nothing is read out of bounds)."""
    pr = synth.sinusoid_pair()
    I0, I1 = pr.I0.copy(), pr.I1.copy()
    (I0 if where == "I0" else I1)[10, 20] = np.nan
    (I0 if where == "I0" else I1)[3, 5] = np.inf
    P = flow.default_params(lam=2.0, levels=2, warps=2, iters=10)
    with pytest.raises(flow.OfError) as e:
        flow.of_solve(ctx, torch.from_numpy(I0).cuda(), torch.from_numpy(I1).cuda(), P)
    assert e.value.status == flow.OF_ENUMERIC
    with pytest.raises(flow.OfError) as e:
        flow.of_solve_host(ctx, I0, I1, P)
    assert e.value.status == flow.OF_ENUMERIC
    with pytest.raises(flow.OfError) as e:
        flow.of_solve_batch(ctx, [torch.from_numpy(pr.I0).cuda(), torch.from_numpy(I0).cuda()],
                            [torch.from_numpy(pr.I1).cuda(), torch.from_numpy(I1).cuda()], P)
    assert e.value.status == flow.OF_ENUMERIC
    # the context stays usable
    u, v, _, st = flow.of_solve(ctx, torch.from_numpy(pr.I0).cuda(), torch.from_numpy(pr.I1).cuda(), P)
    assert np.isfinite(st["energy"]) and bool(torch.isfinite(u).all())
