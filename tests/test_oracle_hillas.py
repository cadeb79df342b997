"""Pins of the oracle's Hillas moments (direction reconstruction input, Sec. 4.1).

Closed forms: a noiseless Gaussian ellipse sampled on a fine camera returns its
generated centroid, length, width and angle; two pixels have width 0 and a
known length.  Library cross-check: numpy's weighted covariance and symmetric
eigensolver.  Invariants: translation, rotation, charge scaling.  The time
gradient of a linear ramp along the axis is its slope.
"""
import numpy as np
import pytest

import oracle

Hf = oracle.H


def grid(pitch, half):
    n = int(round(2 * half / pitch)) + 1
    a = (np.arange(n) - (n - 1) / 2) * pitch
    X, Y = np.meshgrid(a, a)
    return np.stack([X.ravel(), Y.ravel()], 1).astype(np.float32)


def ellipse_density(xy, cx, cy, L, W, psi):
    dx, dy = xy[:, 0].astype(np.float64) - cx, xy[:, 1].astype(np.float64) - cy
    l = dx * np.cos(psi) + dy * np.sin(psi)
    w = -dx * np.sin(psi) + dy * np.cos(psi)
    return np.exp(-0.5 * (l ** 2 / L ** 2 + w ** 2 / W ** 2)) / (2 * np.pi * L * W)


def angle_diff_mod_pi(a, b):
    d = (a - b) % np.pi
    return min(d, np.pi - d)


@pytest.mark.parametrize("cx,cy,L,W,psi", [(0.3, -0.2, 0.3, 0.05, 0.7), (-0.1, 0.25, 0.2, 0.08, -1.2),
                                           (0.0, 0.0, 0.15, 0.06, 1.5707), (0.2, 0.1, 0.35, 0.03, 0.0)])
def test_gaussian_ellipse_recovers_generated_parameters(cx, cy, L, W, psi):
    xy = grid(0.0075, 2.0)
    q = ellipse_density(xy, cx, cy, L, W, psi).astype(np.float32)
    mask = np.ones(len(q), np.uint8)
    h = oracle.hillas(xy, q, None, mask)
    assert h[Hf["x"]] == pytest.approx(cx, abs=1e-3 * 0.1)
    assert h[Hf["y"]] == pytest.approx(cy, abs=1e-3 * 0.1)
    assert h[Hf["length"]] == pytest.approx(L, rel=1e-3)
    assert h[Hf["width"]] == pytest.approx(W, rel=1e-3)
    assert angle_diff_mod_pi(h[Hf["psi"]], psi) < 1e-3
    assert -np.pi / 2 < h[Hf["psi"]] <= np.pi / 2
    assert h[Hf["r"]] == pytest.approx(np.hypot(cx, cy), abs=1e-4)
    if np.hypot(cx, cy) > 0:
        assert h[Hf["phi"]] == pytest.approx(np.arctan2(cy, cx), abs=1e-3)


def test_matches_numpy_weighted_covariance_and_eigh():
    rng = np.random.default_rng(11)
    for _ in range(50):
        n = rng.integers(3, 400)
        xy = rng.uniform(-2, 2, (n, 2)).astype(np.float32)
        q = rng.exponential(20, n).astype(np.float32)
        mask = (rng.uniform(size=n) < 0.7).astype(np.uint8)
        mask[:3] = 1
        h = oracle.hillas(xy, q, None, mask)
        sel = mask == 1
        C = np.cov(xy[sel].T.astype(np.float64), aweights=q[sel].astype(np.float64), bias=True)
        lam, vec = np.linalg.eigh(C)
        assert h[Hf["size"]] == pytest.approx(q[sel].astype(np.float64).sum(), rel=1e-12)
        assert h[Hf["length"]] == pytest.approx(np.sqrt(lam[1]), rel=1e-9)
        assert h[Hf["width"]] == pytest.approx(np.sqrt(max(lam[0], 0)), rel=1e-6, abs=1e-9)
        major = vec[:, 1]
        assert angle_diff_mod_pi(h[Hf["psi"]], np.arctan2(major[1], major[0])) < 1e-9
        mean = np.average(xy[sel].astype(np.float64), axis=0, weights=q[sel])
        assert h[Hf["x"]] == pytest.approx(mean[0], abs=1e-12)
        assert h[Hf["y"]] == pytest.approx(mean[1], abs=1e-12)
        assert h[Hf["n_pix"]] == sel.sum()
        # lambda1 + lambda2 = trace
        assert h[Hf["length"]] ** 2 + h[Hf["width"]] ** 2 == pytest.approx(np.trace(C), rel=1e-9)


def test_translation_rotation_scaling_invariants():
    rng = np.random.default_rng(12)
    n = 300
    ij = rng.integers(-64, 64, (n, 2))
    xy = (ij * 2.0 ** -6).astype(np.float32)           # exact binary fractions
    q = rng.exponential(10, n).astype(np.float32)
    mask = np.ones(n, np.uint8)
    h0 = oracle.hillas(xy, q, None, mask)
    # translation by an exactly representable offset
    h1 = oracle.hillas((xy + np.float32(0.5)).astype(np.float32), q, None, mask)
    assert h1[Hf["x"]] == pytest.approx(h0[Hf["x"]] + 0.5, abs=1e-12)
    for k in ["length", "width", "psi", "size"]:
        assert h1[Hf[k]] == pytest.approx(h0[Hf[k]], rel=1e-9, abs=1e-12)
    # rotation by 90 degrees is exact on the lattice: psi -> psi + pi/2 (mod pi)
    rot = np.stack([-xy[:, 1], xy[:, 0]], 1).astype(np.float32)
    h2 = oracle.hillas(rot, q, None, mask)
    assert angle_diff_mod_pi(h2[Hf["psi"]], h0[Hf["psi"]] + np.pi / 2) < 1e-9
    for k in ["length", "width", "size"]:
        assert h2[Hf[k]] == pytest.approx(h0[Hf[k]], rel=1e-9)
    # general rotation (positions rounded to fp32)
    th = 0.37
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    h3 = oracle.hillas((xy.astype(np.float64) @ R.T).astype(np.float32), q, None, mask)
    assert angle_diff_mod_pi(h3[Hf["psi"]], h0[Hf["psi"]] + th) < 1e-5
    assert h3[Hf["length"]] == pytest.approx(h0[Hf["length"]], rel=1e-6)
    # scaling the charges by 4 (exact in fp32)
    h4 = oracle.hillas(xy, (q * 4).astype(np.float32), None, mask)
    assert h4[Hf["size"]] == pytest.approx(4 * h0[Hf["size"]], rel=1e-12)
    for k in ["x", "y", "length", "width", "psi"]:
        assert h4[Hf[k]] == pytest.approx(h0[Hf[k]], rel=1e-12, abs=1e-14)


def test_two_pixels_closed_form():
    xy = np.array([[0.1, 0.2], [0.4, 0.6]], np.float32)
    q = np.array([3.0, 1.0], np.float32)
    h = oracle.hillas(xy, q, None, np.ones(2, np.uint8))
    d = np.hypot(*(xy[1].astype(np.float64) - xy[0]))
    assert h[Hf["width"]] == 0.0 or h[Hf["width"]] < 1e-7
    assert h[Hf["length"]] == pytest.approx(d * np.sqrt(3.0 * 1.0) / 4.0, rel=1e-7)
    assert angle_diff_mod_pi(h[Hf["psi"]], np.arctan2(0.4, 0.3)) < 1e-6


def test_time_gradient_of_linear_ramp():
    xy = grid(0.02, 1.0)
    psi_true = 0.6
    q = ellipse_density(xy, 0.1, -0.1, 0.3, 0.06, psi_true).astype(np.float32)
    mask = (q > 1e-3 * q.max()).astype(np.uint8)
    l_true = (xy[:, 0] - 0.1) * np.cos(psi_true) + (xy[:, 1] + 0.1) * np.sin(psi_true)
    t = 6.0 + 2.0 * l_true
    h = oracle.hillas(xy, q, t, mask)
    sign = np.sign(np.cos(h[Hf["psi"]] - psi_true))
    assert h[Hf["time_grad"]] * sign == pytest.approx(2.0, rel=1e-3)
    t2 = 6.0 + 0 * l_true
    assert oracle.hillas(xy, q, t2, mask)[Hf["time_grad"]] == pytest.approx(0.0, abs=1e-12)


def test_degenerate_images():
    xy = np.array([[0.0, 0.0], [0.1, 0.0]], np.float32)
    q = np.array([5.0, 7.0], np.float32)
    h = oracle.hillas(xy, q, np.array([1.0, 2.0]), np.zeros(2, np.uint8))
    assert h[Hf["flags"]] == oracle.FLAG_EMPTY | oracle.FLAG_NO_TIME and h[Hf["size"]] == 0
    h = oracle.hillas(xy, q, np.array([1.0, 2.0]), np.array([0, 1], np.uint8))
    assert h[Hf["n_pix"]] == 1 and h[Hf["length"]] == 0 and h[Hf["width"]] == 0
    assert int(h[Hf["flags"]]) & oracle.FLAG_NO_TIME
    assert h[Hf["x"]] == pytest.approx(0.1)
