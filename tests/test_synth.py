"""CPU checks of the seeded input generators (input generation only, shared by the CUDA path and
the oracle): determinism, value range, and that each ground-truth field is the motion the frames
show, I1(x + u, y + v) = I0(x, y), exactly where the motion is an integer shift (noise off)."""
import numpy as np
import pytest

from paper_2011_10979_gb300 import synth


def test_seeded_and_in_range():
    a, b = synth.sinusoid_pair(seed=3), synth.sinusoid_pair(seed=3)
    assert np.array_equal(a.I0, b.I0) and np.array_equal(a.I1, b.I1)
    assert not np.array_equal(a.I0, synth.sinusoid_pair(seed=4).I0)
    for p in (a, synth.affine_rect_pair(H=60, W=80), synth.layered_pair(H=44, W=100), synth.random_affine_rect_pair(30, 50, 1)):
        for im in (p.I0, p.I1):
            assert im.dtype == np.float32 and im.shape == p.u_true.shape == p.v_true.shape
            assert im.min() >= 0.0 and im.max() <= 1.0


def test_sinusoid_pair_shows_its_motion():
    """Integer motions (2, 0) on the left half and (-1, 1) on the right, no noise: the frame-1
    pixel a frame-0 pixel moves to holds exactly its value."""
    p = synth.sinusoid_pair(sigma=0.0, left=(2.0, 0.0), right=(-1.0, 1.0))
    H, W = p.I0.shape
    assert np.all(p.u_true[:, : W // 2] == 2) and np.all(p.v_true[:, W // 2:] == 1)
    # left half of frame 1: I1(x, y) = f(x - 2, y) = I0(x - 2, y)
    assert np.array_equal(p.I1[:, 2: W // 2], p.I0[:, : W // 2 - 2])
    # right half: I1(x, y) = f(x + 1, y - 1) = I0(x + 1, y - 1)
    assert np.array_equal(p.I1[1:, W // 2: W - 1], p.I0[:-1, W // 2 + 1:])


def test_affine_rect_pair_shows_its_motion():
    """Pure translation (3, -2) of the background and a box moving (6, 4), no noise: background
    pixels away from both box positions and every box pixel land exactly on their values."""
    H, W, bx, by, rw, rh = 60, 80, 20, 15, 16, 12
    p = synth.affine_rect_pair(H=H, W=W, sigma=0.0, rot_deg=0.0, zoom=1.0, shift=(3.0, -2.0), rect=(rw, rh),
                               rect_motion=(6.0, 4.0), rect_pos=(bx, by))
    y, x = np.mgrid[0:H, 0:W]
    box0 = (x >= bx) & (x < bx + rw) & (y >= by) & (y < by + rh)
    assert np.all(p.u_true[box0] == 6) and np.all(p.v_true[box0] == 4)
    assert np.allclose(p.u_true[~box0], 3) and np.allclose(p.v_true[~box0], -2)
    # box: I1(x + 6, y + 4) = I0(x, y)
    assert np.array_equal(p.I1[by + 4: by + 4 + rh, bx + 6: bx + 6 + rw], p.I0[by: by + rh, bx: bx + rw])
    # background: I1(x + 3, y - 2) = I0(x, y) where neither frame's box covers those pixels
    xs, ys = x + 3, y - 2
    ok = ~box0 & (xs < W) & (ys >= 0)
    box1 = lambda X, Y: (X >= bx + 6) & (X < bx + 6 + rw) & (Y >= by + 4) & (Y < by + 4 + rh)
    ok &= ~box1(xs, ys)
    assert ok.sum() > 0.5 * H * W
    assert np.array_equal(p.I1[ys[ok], xs[ok]], p.I0[ok])


def test_layered_pair_motion_bounds():
    """Background rotated 1 degree about the centre; ellipses translated by at most max_shift."""
    p = synth.layered_pair(H=120, W=200, max_shift=10.0)
    H, W = p.I0.shape
    r = np.hypot(W / 2.0, H / 2.0)
    bound = max(10.0, 2 * r * np.sin(np.radians(1.0) / 2) + 1e-6)
    assert np.hypot(p.u_true, p.v_true).max() <= bound


@pytest.mark.parametrize("n", [12])
def test_batch_sizes_and_motion(n):
    ps = synth.batch_pairs(n=n)
    sizes = {p.I0.shape for p in ps}
    assert sizes <= set(synth.BATCH_SIZES) and len(sizes) == len(synth.BATCH_SIZES)
    for p in ps:
        H, W = p.I0.shape
        d = np.hypot(p.u_true, p.v_true)
        # translation <= 7.5 px, box <= 15 px; rotation (2 deg) and zoom (3%) about the centre add
        # at most 0.05 px per px of distance from it
        assert d.max() <= 15.0 + 0.05 * np.hypot(W / 2.0, H / 2.0) + 1e-6


def test_sinusoid_pair_bilinear_rendering():
    from scipy import ndimage
    a = synth.sinusoid_pair()
    assert np.array_equal(a.I1, synth.sinusoid_pair(render="analytic").I1)
    p = synth.sinusoid_pair(render="bilinear")
    H, W = p.I0.shape
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    ys, xs = np.clip(y - p.v_true, 0, H - 1), np.clip(x - p.u_true, 0, W - 1)
    ref = ndimage.map_coordinates(p.I0.astype(np.float64), [ys, xs], order=1, mode="nearest")
    assert np.max(np.abs(p.I1 - ref)) <= 6e-8
    assert np.array_equal(p.u_true, a.u_true) and np.array_equal(p.v_true, a.v_true)
    with pytest.raises(ValueError):
        synth.sinusoid_pair(render="nearest")


def test_batch_pairs_in_workers_equal_serial_and_extend_shorter_batches():
    serial = synth.batch_pairs(n=6)
    pooled = synth.batch_pairs(n=6, workers=2)
    assert [sp[:2] for sp in synth.batch_specs(6)] == [p.I0.shape for p in serial]
    assert synth.batch_specs(4) == synth.batch_specs(6)[:4]
    for a, b in zip(serial, pooled):
        for k in ("I0", "I1", "u_true", "v_true"):
            assert np.array_equal(getattr(a, k), getattr(b, k))


def test_batch_pairs_fall_back_to_threads_without_a_process_pool(monkeypatch):
    import concurrent.futures as cf

    class NoPool:
        def __init__(self, *a, **k):
            raise OSError("no POSIX semaphores here")

    monkeypatch.setattr(cf, "ProcessPoolExecutor", NoPool)
    got = synth.batch_pairs(n=3, workers=2)
    for a, b in zip(synth.batch_pairs(n=3), got):
        assert np.array_equal(a.I0, b.I0) and np.array_equal(a.I1, b.I1)


def test_serving_mix_and_arrivals():
    sizes = synth.serve_sizes(2000)
    frac = {s: sizes.count(s) / len(sizes) for s, _ in synth.SERVE_MIX}
    for s, w in synth.SERVE_MIX:
        assert abs(frac[s] - w) < 0.04
    t = synth.poisson_arrivals(50.0, 20.0)
    assert all(b > a for a, b in zip(t, t[1:])) and t[-1] < 20.0
    assert abs(len(t) / 20.0 - 50.0) < 5.0
