"""Flow evaluation in the form of Sec. 4's Tables 1-2: ground truth in the Middlebury ``.flo``
format, the average angular error (AAE, degrees) and the average end-point error (EPE, pixels).

The paper reports both measures without defining them; these are the standard definitions of the
Middlebury benchmark (Barron, Fleet and Beauchemin for the angular error):
  AAE = mean over valid pixels of arccos(((u, v, 1) . (u_gt, v_gt, 1)) / (|(u, v, 1)| |(u_gt, v_gt, 1)|))
  EPE = mean over valid pixels of |(u - u_gt, v - v_gt)|
and a ground-truth pixel is unknown (excluded) when |u_gt| or |v_gt| exceeds 1e9.

``.flo`` layout (little endian): float32 tag 202021.25, int32 width, int32 height, then height rows
of width (u, v) float32 pairs.  The data sets the paper evaluates on are not shipped here; this
module reads them when a user supplies them, and ``solve_and_evaluate`` runs the library on a pair
and scores it.  Host-side numpy only: evaluation is not part of the solver's hot path.
"""
from __future__ import annotations

import numpy as np

FLO_TAG = 202021.25
UNKNOWN_FLOW = 1e9


def write_flo(path, u, v) -> None:
    u = np.asarray(u, np.float32)
    v = np.asarray(v, np.float32)
    if u.shape != v.shape or u.ndim != 2:
        raise ValueError("u and v must be 2-D arrays of one shape")
    H, W = u.shape
    uv = np.empty((H, W, 2), "<f4")
    uv[..., 0] = u
    uv[..., 1] = v
    with open(path, "wb") as f:
        f.write(np.array([FLO_TAG], "<f4").tobytes())
        f.write(np.array([W, H], "<i4").tobytes())
        f.write(uv.tobytes())


def read_flo(path):
    """Returns (u, v) as float32 H x W arrays."""
    with open(path, "rb") as f:
        data = f.read()
    if len(data) < 12:
        raise ValueError("not a .flo file: too short")
    tag = np.frombuffer(data, "<f4", 1, 0)[0]
    if tag != np.float32(FLO_TAG):
        raise ValueError("not a .flo file: tag %r" % float(tag))
    W, H = (int(x) for x in np.frombuffer(data, "<i4", 2, 4))
    if W < 1 or H < 1 or len(data) != 12 + 8 * W * H:
        raise ValueError("bad .flo size: %d x %d for %d bytes" % (W, H, len(data)))
    uv = np.frombuffer(data, "<f4", 2 * W * H, 12).reshape(H, W, 2)
    return uv[..., 0].astype(np.float32), uv[..., 1].astype(np.float32)


def valid_mask(u_gt, v_gt):
    u_gt = np.asarray(u_gt, np.float64)
    v_gt = np.asarray(v_gt, np.float64)
    return (np.abs(u_gt) <= UNKNOWN_FLOW) & (np.abs(v_gt) <= UNKNOWN_FLOW) & np.isfinite(u_gt) & np.isfinite(v_gt)


def angular_error_deg(u, v, u_gt, v_gt):
    """Per-pixel angle between the space-time vectors (u, v, 1) and (u_gt, v_gt, 1), in degrees."""
    u, v, ug, vg = (np.asarray(x, np.float64) for x in (u, v, u_gt, v_gt))
    num = u * ug + v * vg + 1.0
    den = np.sqrt(u * u + v * v + 1.0) * np.sqrt(ug * ug + vg * vg + 1.0)
    return np.degrees(np.arccos(np.clip(num / den, -1.0, 1.0)))


def endpoint_error(u, v, u_gt, v_gt):
    u, v, ug, vg = (np.asarray(x, np.float64) for x in (u, v, u_gt, v_gt))
    return np.hypot(u - ug, v - vg)


def evaluate(u, v, u_gt, v_gt) -> dict:
    """AAE (degrees) and EPE (pixels) over the pixels with known ground truth."""
    m = valid_mask(u_gt, v_gt)
    n = int(m.sum())
    if n == 0:
        return {"aae_deg": float("nan"), "epe_px": float("nan"), "valid_px": 0}
    ug = np.where(m, u_gt, 0.0)
    vg = np.where(m, v_gt, 0.0)
    return {"aae_deg": float(angular_error_deg(u, v, ug, vg)[m].mean()),
            "epe_px": float(endpoint_error(u, v, ug, vg)[m].mean()), "valid_px": n}


def solve_and_evaluate(ctx, I0, I1, gt, params) -> dict:
    """Solves the pair (float32 H x W host arrays, intensities in [0, 1]) with the library and
    scores it against ground truth given as a ``.flo`` path or a (u_gt, v_gt) tuple."""
    from . import flow

    u_gt, v_gt = read_flo(gt) if isinstance(gt, (str, bytes)) or hasattr(gt, "__fspath__") else gt
    I0 = np.ascontiguousarray(I0, np.float32)
    I1 = np.ascontiguousarray(I1, np.float32)
    if I0.shape != I1.shape or I0.shape != np.shape(u_gt):
        raise ValueError("frames and ground truth must have one shape")
    u, v, st = flow.of_solve_host(ctx, I0, I1, params)
    out = evaluate(u, v, u_gt, v_gt)
    out.update(iters_run=st["iters_run"], energy=st["energy"])
    return out
