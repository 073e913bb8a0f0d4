"""Seeded synthetic image pairs shaped like the paper's optical-flow workloads.

The paper evaluates on the Middlebury, Ettlinger-Tor, Rheinhafen and Yosemite sequences
(Sec. 4), which are not available here; these generators stand in for them.  Every image is
rendered analytically: a closed-form texture f is evaluated at I0(x) = f(x) and at
I1(y) = f(y - D(y)) for a known motion D, so the ground truth carries no interpolation error.
Noise is added to each frame independently and the result is clipped to [0, 1] and stored in
float32.  This module holds input generation only, none of the solver's arithmetic; the CUDA
library and the oracle both take their inputs from here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Pair:
    I0: np.ndarray          # float32 H x W, values in [0, 1]
    I1: np.ndarray          # float32 H x W
    u_true: np.ndarray      # float32 H x W, horizontal motion of frame-0 pixels
    v_true: np.ndarray      # float32 H x W, vertical motion


# ------------------------------------------------------------------ analytic textures
class Sinusoids:
    """Sum of `n` plane waves with periods in [pmin, pmax] px, random orientation and phase."""

    def __init__(self, rng, n=16, pmin=4.0, pmax=24.0):
        self.k = []
        for _ in range(n):
            period = rng.uniform(pmin, pmax)
            th = rng.uniform(0.0, math.pi)
            self.k.append((2 * math.pi / period * math.cos(th), 2 * math.pi / period * math.sin(th),
                           rng.uniform(0.0, 2 * math.pi)))

    def __call__(self, x, y):
        out = np.zeros(np.broadcast(x, y).shape, np.float64)
        for kx, ky, ph in self.k:
            out += np.sin(kx * x + ky * y + ph)
        return out


class GradientNoise:
    """Perlin-style gradient noise: `octaves` octaves, base cell `cell` px, lacunarity 2,
    gain 0.5; lattice gradients are random unit vectors from a seeded table."""

    def __init__(self, rng, octaves=4, cell=48.0, table=256):
        self.octaves, self.cell, self.n = octaves, cell, table
        ang = rng.uniform(0.0, 2 * math.pi, size=table)
        self.g = np.stack([np.cos(ang), np.sin(ang)], axis=1)
        self.perm = rng.permutation(table)
        self.off = rng.uniform(0.0, 1000.0, size=(octaves, 2))

    def _hash(self, ix, iy):
        return self.perm[(self.perm[ix % self.n] + iy) % self.n]

    def _octave(self, x, y):
        x0, y0 = np.floor(x), np.floor(y)
        fx, fy = x - x0, y - y0
        ix, iy = x0.astype(np.int64), y0.astype(np.int64)

        def dot(cx, cy, dx, dy):
            g = self.g[self._hash(ix + cx, iy + cy)]
            return g[..., 0] * dx + g[..., 1] * dy

        fade = lambda t: t * t * t * (t * (t * 6 - 15) + 10)
        sx, sy = fade(fx), fade(fy)
        n00, n10 = dot(0, 0, fx, fy), dot(1, 0, fx - 1, fy)
        n01, n11 = dot(0, 1, fx, fy - 1), dot(1, 1, fx - 1, fy - 1)
        return (1 - sy) * ((1 - sx) * n00 + sx * n10) + sy * ((1 - sx) * n01 + sx * n11)

    def __call__(self, x, y):
        x, y = np.broadcast_arrays(np.asarray(x, np.float64), np.asarray(y, np.float64))
        out = np.zeros(x.shape, np.float64)
        amp, cell = 1.0, self.cell
        for o in range(self.octaves):
            out += amp * self._octave(x / cell + self.off[o, 0], y / cell + self.off[o, 1])
            amp *= 0.5
            cell *= 0.5
        return out


def _finish(rng, f0, f1, sigma):
    lo, hi = float(f0.min()), float(f0.max())
    scale = 1.0 / (hi - lo) if hi > lo else 1.0
    out = []
    for f in (f0, f1):
        g = (f - lo) * scale + rng.normal(0.0, sigma, size=f.shape)
        out.append(np.clip(g, 0.0, 1.0).astype(np.float32))
    return out


def _grid(H, W):
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    return x, y


# ------------------------------------------------------------------ workloads
def sinusoid_pair(H=48, W=64, seed=0, sigma=0.01, left=(1.5, -0.5), right=(-0.75, 1.0), render="analytic"):
    """64 x 48 case: 16 random sinusoids, piecewise-constant motion (left half / right half).

    render="analytic": both frames evaluate the closed-form texture (frame 1 at y - D(y)), each with
    its own noise.  render="bilinear": frame 1 is frame 0 itself (noise included) resampled
    bilinearly at y - D(y), positions clamped to the image (the workload's literal wording)."""
    rng = np.random.default_rng(seed)
    tex = Sinusoids(rng)
    x, y = _grid(H, W)
    half = x < W / 2.0
    ut = np.where(half, left[0], right[0])
    vt = np.where(half, left[1], right[1])
    f0 = tex(x, y)
    if render == "bilinear":
        lo, hi = float(f0.min()), float(f0.max())
        g0 = (f0 - lo) * (1.0 / (hi - lo) if hi > lo else 1.0) + rng.normal(0.0, sigma, size=f0.shape)
        I0 = np.clip(g0, 0.0, 1.0).astype(np.float32)
        I1 = _bilinear(I0.astype(np.float64), x - ut, y - vt).astype(np.float32)
        return Pair(I0, I1, ut.astype(np.float32), vt.astype(np.float32))
    if render != "analytic":
        raise ValueError("render must be 'analytic' or 'bilinear'")
    f1 = tex(x - ut, y - vt)    # frame 1 at y shows the frame-0 point y - D(y)
    I0, I1 = _finish(rng, f0, f1, sigma)
    return Pair(I0, I1, ut.astype(np.float32), vt.astype(np.float32))


def _bilinear(img, xs, ys):
    """Bilinear samples of img at (xs, ys), positions clamped to [0, W-1] x [0, H-1]."""
    H, W = img.shape
    xs, ys = np.clip(xs, 0.0, W - 1.0), np.clip(ys, 0.0, H - 1.0)
    x0, y0 = np.floor(xs).astype(np.int64), np.floor(ys).astype(np.int64)
    fx, fy = xs - x0, ys - y0
    x1, y1 = np.minimum(x0 + 1, W - 1), np.minimum(y0 + 1, H - 1)
    top = (1.0 - fx) * img[y0, x0] + fx * img[y0, x1]
    bot = (1.0 - fx) * img[y1, x0] + fx * img[y1, x1]
    return (1.0 - fy) * top + fy * bot


def _affine(W, H, rot_deg, zoom, tx, ty):
    cx, cy = (W - 1) / 2.0, (H - 1) / 2.0
    th = math.radians(rot_deg)
    A = zoom * np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    return cx, cy, A, np.array([tx, ty])


def affine_rect_pair(H=480, W=640, seed=1, sigma=0.01, rot_deg=2.0, zoom=1.03, shift=(3.0, -2.0),
                     rect=(120, 80), rect_motion=(6.0, 4.0), rect_pos=None, cell=48.0):
    """640 x 480 case: 4-octave gradient-noise background under an affine motion (rotation,
    zoom, translation about the image centre) and a textured rect[0] x rect[1] box moving by
    rect_motion and occluding the background."""
    rng = np.random.default_rng(seed)
    bg = GradientNoise(rng, octaves=4, cell=cell)
    fg = GradientNoise(rng, octaves=4, cell=cell / 3.0)
    x, y = _grid(H, W)
    cx, cy, A, t = _affine(W, H, rot_deg, zoom, *shift)
    # frame 0: background, box on top at rect_pos
    rw, rh = min(rect[0], W), min(rect[1], H)
    if rect_pos is None:
        rect_pos = (int(rng.integers(0, max(1, W - rw))), int(rng.integers(0, max(1, H - rh))))
    bx, by = rect_pos
    mx, my = rect_motion
    in0 = (x >= bx) & (x < bx + rw) & (y >= by) & (y < by + rh)
    # the box texture is evaluated on the box's pixels only (the textures are pointwise, so the
    # values are those of a whole-image evaluation)
    f0 = bg(x, y)
    f0[in0] = 1.5 * fg(x[in0] - bx, y[in0] - by)
    # frame 1: inverse affine for the background; the box moved by (mx, my)
    Ai = np.linalg.inv(A)
    px, py = x - cx - t[0], y - cy - t[1]
    sx, sy = Ai[0, 0] * px + Ai[0, 1] * py + cx, Ai[1, 0] * px + Ai[1, 1] * py + cy
    in1 = (x >= bx + mx) & (x < bx + mx + rw) & (y >= by + my) & (y < by + my + rh)
    f1 = bg(sx, sy)
    f1[in1] = 1.5 * fg(x[in1] - bx - mx, y[in1] - by - my)
    # ground truth of frame-0 pixels
    ax = A[0, 0] * (x - cx) + A[0, 1] * (y - cy) + cx + t[0] - x
    ay = A[1, 0] * (x - cx) + A[1, 1] * (y - cy) + cy + t[1] - y
    ut = np.where(in0, mx, ax)
    vt = np.where(in0, my, ay)
    I0, I1 = _finish(rng, f0, f1, sigma)
    return Pair(I0, I1, ut.astype(np.float32), vt.astype(np.float32))


def layered_pair(H=436, W=1024, seed=2, sigma=0.02, n_layers=6, max_shift=20.0, rot_deg=1.0):
    """1024 x 436 case: textured ellipses over a textured background; each ellipse translates
    independently by up to max_shift px, the background rotates mildly about the centre."""
    rng = np.random.default_rng(seed)
    bg = GradientNoise(rng, octaves=4, cell=56.0)
    x, y = _grid(H, W)
    cx, cy, A, t = _affine(W, H, rot_deg, 1.0, 0.0, 0.0)
    Ai = np.linalg.inv(A)
    px, py = x - cx, y - cy
    sx, sy = Ai[0, 0] * px + Ai[0, 1] * py + cx, Ai[1, 0] * px + Ai[1, 1] * py + cy
    f0 = bg(x, y)
    f1 = bg(sx, sy)
    ut = A[0, 0] * (x - cx) + A[0, 1] * (y - cy) + cx - x
    vt = A[1, 0] * (x - cx) + A[1, 1] * (y - cy) + cy - y
    for _ in range(n_layers):
        tex = GradientNoise(rng, octaves=3, cell=float(rng.uniform(10.0, 24.0)))
        ex, ey = rng.uniform(0.1 * W, 0.9 * W), rng.uniform(0.1 * H, 0.9 * H)
        ra, rb = rng.uniform(0.05, 0.15) * W, rng.uniform(0.1, 0.3) * H
        ang = rng.uniform(0.0, 2 * math.pi)
        mag = rng.uniform(0.3, 1.0) * max_shift
        mx, my = mag * math.cos(ang), mag * math.sin(ang)
        inside0 = ((x - ex) / ra) ** 2 + ((y - ey) / rb) ** 2 <= 1.0
        inside1 = ((x - ex - mx) / ra) ** 2 + ((y - ey - my) / rb) ** 2 <= 1.0
        f0 = np.where(inside0, 1.3 * tex(x - ex, y - ey) + 0.4, f0)
        f1 = np.where(inside1, 1.3 * tex(x - ex - mx, y - ey - my) + 0.4, f1)
        ut = np.where(inside0, mx, ut)
        vt = np.where(inside0, my, vt)
    I0, I1 = _finish(rng, f0, f1, sigma)
    return Pair(I0, I1, ut.astype(np.float32), vt.astype(np.float32))


BATCH_SIZES = ((64, 96), (240, 320), (480, 640), (436, 1024), (375, 1242))   # (H, W)


def batch_specs(n=256, seed=3):
    """(H, W, pair seed) of each pair of the uneven-size batch, sizes drawn uniformly from
    BATCH_SIZES.  The first k specs of a batch of n are those of a batch of k."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        H, W = BATCH_SIZES[int(rng.integers(0, len(BATCH_SIZES)))]
        out.append((H, W, int(rng.integers(0, 2**31 - 1))))
    return out


def _spec_pair(spec, max_motion):
    H, W, s = spec
    return random_affine_rect_pair(H, W, s, max_motion)


def batch_pairs(n=256, seed=3, max_motion=15.0, workers=1):
    """Uneven-size batch: one affine+box pair (random_affine_rect_pair) with its own seed per
    spec of batch_specs.  workers > 1 renders the pairs in that many spawned processes (the
    pairs are the same)."""
    specs = batch_specs(n, seed)
    if workers <= 1 or n <= 1:
        return [_spec_pair(sp, max_motion) for sp in specs]
    import concurrent.futures as cf
    import multiprocessing as mp
    try:
        with cf.ProcessPoolExecutor(max_workers=min(workers, n), mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(_spec_pair, specs, [max_motion] * n, chunksize=4))
    except (OSError, cf.process.BrokenProcessPool):
        # no process pool on this host (e.g. no POSIX semaphores): threads give the same pairs
        with cf.ThreadPoolExecutor(max_workers=min(workers, n)) as ex:
            return list(ex.map(_spec_pair, specs, [max_motion] * n))


def random_affine_rect_pair(H, W, seed, max_motion=15.0, sigma=0.01):
    """Affine+box pair with random parameters: translation up to max_motion / 2 px, rotation up
    to 2 degrees and zoom 0.98 .. 1.03 about the image centre, and a box of up to 120 x 80 px
    (a quarter of the image at most) moving by 0.3 .. 1 x max_motion px.  The box motion and the
    translation stay within max_motion; rotation and zoom add up to about 0.05 px per px of
    distance from the centre, so the corners of the largest images move up to about 1.5 x
    max_motion."""
    rng = np.random.default_rng(seed)
    rot = float(rng.uniform(-2.0, 2.0))
    zoom = float(rng.uniform(0.98, 1.03))
    ang = rng.uniform(0.0, 2 * math.pi)
    mag = rng.uniform(0.0, 0.5) * max_motion
    ang2 = rng.uniform(0.0, 2 * math.pi)
    mag2 = rng.uniform(0.3, 1.0) * max_motion
    rect = (max(4, min(120, W // 4)), max(4, min(80, H // 4)))
    return affine_rect_pair(H, W, seed=int(rng.integers(0, 2**31 - 1)), sigma=sigma, rot_deg=rot,
                            zoom=zoom, shift=(mag * math.cos(ang), mag * math.sin(ang)), rect=rect,
                            rect_motion=(mag2 * math.cos(ang2), mag2 * math.sin(ang2)))


SERVE_MIX = (((240, 320), 0.40), ((480, 640), 0.30), ((436, 1024), 0.20), ((1080, 1920), 0.08),
             ((2160, 3840), 0.02))


def serve_sizes(n, seed=4):
    rng = np.random.default_rng(seed)
    p = np.array([w for _, w in SERVE_MIX])
    idx = rng.choice(len(SERVE_MIX), size=n, p=p / p.sum())
    return [SERVE_MIX[i][0] for i in idx]


def poisson_arrivals(rate_hz, duration_s, seed=5):
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            return out
        out.append(t)
