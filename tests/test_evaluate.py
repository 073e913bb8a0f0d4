"""Evaluation harness (AAE / EPE against Middlebury .flo ground truth, the measures of Sec. 4's
Tables 1-2): file format round trip and rejection of malformed files, closed-form values of the two
error measures, unknown-flow masking, and one GPU solve scored end to end."""
import math

import numpy as np
import pytest

from paper_2011_10979_gb300 import evaluate as ev


def test_flo_round_trip_and_layout(tmp_path):
    rng = np.random.default_rng(0)
    u = rng.normal(size=(5, 7)).astype(np.float32)
    v = rng.normal(size=(5, 7)).astype(np.float32)
    p = tmp_path / "a.flo"
    ev.write_flo(p, u, v)
    raw = p.read_bytes()
    assert len(raw) == 12 + 8 * 35
    assert np.frombuffer(raw[:4], "<f4")[0] == np.float32(202021.25)
    assert raw[:4] == b"PIEH"  # the tag's bytes spell the format's sanity check
    assert tuple(np.frombuffer(raw[4:12], "<i4")) == (7, 5)
    # row-major (u, v) pairs: element (i, j) at 12 + 8 (i W + j)
    i, j = 3, 4
    assert np.frombuffer(raw[12 + 8 * (i * 7 + j):12 + 8 * (i * 7 + j) + 8], "<f4").tolist() == [u[i, j], v[i, j]]
    ru, rv = ev.read_flo(p)
    assert np.array_equal(ru, u) and np.array_equal(rv, v)


def test_flo_rejects_malformed(tmp_path):
    p = tmp_path / "b.flo"
    p.write_bytes(b"xx")
    with pytest.raises(ValueError):
        ev.read_flo(p)
    p.write_bytes(np.array([1.0], "<f4").tobytes() + np.array([2, 2], "<i4").tobytes() + bytes(32))
    with pytest.raises(ValueError):
        ev.read_flo(p)
    p.write_bytes(np.array([202021.25], "<f4").tobytes() + np.array([2, 2], "<i4").tobytes() + bytes(31))
    with pytest.raises(ValueError):
        ev.read_flo(p)


def test_error_measures_closed_forms():
    z = np.zeros((1, 1))
    # (1, 0, 1) against (0, 0, 1): 45 degrees, end point error 1
    assert ev.angular_error_deg(z + 1, z, z, z)[0, 0] == pytest.approx(45.0, abs=1e-12)
    assert ev.endpoint_error(z + 1, z, z, z)[0, 0] == pytest.approx(1.0)
    # (u, v) = (3, 4) against (0, 0): EPE 5, angle arccos(1 / sqrt(26))
    assert ev.endpoint_error(z + 3, z + 4, z, z)[0, 0] == pytest.approx(5.0)
    assert ev.angular_error_deg(z + 3, z + 4, z, z)[0, 0] == pytest.approx(math.degrees(math.acos(1 / math.sqrt(26))))
    # identical flows: both zero (no NaN from rounding above 1 inside arccos)
    rng = np.random.default_rng(1)
    a, b = rng.normal(size=(20, 20)) * 50, rng.normal(size=(20, 20)) * 50
    assert np.all(ev.angular_error_deg(a, b, a, b) < 1e-5)
    assert np.all(ev.endpoint_error(a, b, a, b) == 0.0)
    # symmetric in its two arguments, invariant under rotating both flows
    c, d = rng.normal(size=(20, 20)), rng.normal(size=(20, 20))
    assert np.allclose(ev.angular_error_deg(a, b, c, d), ev.angular_error_deg(c, d, a, b))
    th = 0.7
    rot = lambda x, y: (math.cos(th) * x - math.sin(th) * y, math.sin(th) * x + math.cos(th) * y)
    assert np.allclose(ev.angular_error_deg(*rot(a, b), *rot(c, d)), ev.angular_error_deg(a, b, c, d))


def test_unknown_ground_truth_is_excluded():
    u = np.array([[1.0, 0.0, 5.0]])
    v = np.zeros((1, 3))
    ug = np.array([[0.0, 0.0, 1e10]])
    vg = np.array([[0.0, 0.0, 0.0]])
    r = ev.evaluate(u, v, ug, vg)
    assert r["valid_px"] == 2
    assert r["epe_px"] == pytest.approx(0.5)
    assert r["aae_deg"] == pytest.approx(22.5)
    r = ev.evaluate(u, v, ug * 0 + 2e9, vg)
    assert r["valid_px"] == 0 and math.isnan(r["epe_px"])


@pytest.mark.gpu
def test_solve_and_evaluate_known_motion(tmp_path):
    import torch
    from paper_2011_10979_gb300 import flow, synth
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pr = synth.sinusoid_pair()
    gt = tmp_path / "gt.flo"
    ev.write_flo(gt, pr.u_true, pr.v_true)
    ctx = flow.Context(0)
    try:
        r = ev.solve_and_evaluate(ctx, pr.I0, pr.I1, str(gt), flow.default_params(lam=5.0))
    finally:
        ctx.close()
    assert r["valid_px"] == pr.I0.size
    assert r["epe_px"] < 0.1 and r["aae_deg"] < 5.0, r
