"""Pins of the oracle's stereo Hillas intersection (direction + core, Sec. 4.1).

Lines that all pass through one point intersect there for any weights, so a
noiseless array (axes through the source in the camera and through the core
on the ground) is recovered exactly.  Two images reduce to a 2x2 linear solve.
Turning an axis by pi leaves the line unchanged; a round image (width =
length) carries no weight.
"""
import numpy as np
import pytest

import oracle

Hf = oracle.H
Sf = oracle.S


def make_rows(rng, src, core, tel, sizes=None, widths=None, lengths=None):
    m = len(tel)
    rows = np.zeros((m, 12))
    for i in range(m):
        d = tel[i] - core
        psi = np.arctan2(d[1], d[0])
        off = rng.uniform(0.1, 2.0)
        c = src + off * d / np.linalg.norm(d)
        rows[i, Hf["x"]], rows[i, Hf["y"]] = c
        rows[i, Hf["psi"]] = psi
        rows[i, Hf["size"]] = rng.uniform(50, 5000) if sizes is None else sizes[i]
        rows[i, Hf["length"]] = rng.uniform(0.1, 0.4) if lengths is None else lengths[i]
        rows[i, Hf["width"]] = rng.uniform(0.01, 0.09) if widths is None else widths[i]
        rows[i, Hf["n_pix"]] = 10
    return rows


@pytest.mark.parametrize("m", [2, 3, 5, 17, 40])
def test_noiseless_array_recovers_source_and_core(m):
    rng = np.random.default_rng(100 + m)
    for _ in range(20):
        src = rng.uniform(-2, 2, 2)
        core = rng.uniform(-500, 500, 2)
        tel = rng.uniform(-600, 600, (m, 2))
        rows = make_rows(rng, src, core, tel)
        out = oracle.stereo(rows, tel)
        assert out[Sf["flags"]] == 0
        assert out[Sf["dir_x"]] == pytest.approx(src[0], abs=1e-9)
        assert out[Sf["dir_y"]] == pytest.approx(src[1], abs=1e-9)
        assert out[Sf["core_x"]] == pytest.approx(core[0], abs=1e-7)
        assert out[Sf["core_y"]] == pytest.approx(core[1], abs=1e-7)
        assert out[Sf["n_valid"]] == m


def test_two_images_equal_linear_solve():
    rng = np.random.default_rng(7)
    for _ in range(100):
        rows = np.zeros((2, 12))
        rows[:, Hf["x"]] = rng.uniform(-2, 2, 2)
        rows[:, Hf["y"]] = rng.uniform(-2, 2, 2)
        rows[:, Hf["psi"]] = rng.uniform(-np.pi / 2, np.pi / 2, 2)
        rows[:, Hf["size"]] = rng.uniform(50, 500, 2)
        rows[:, Hf["length"]] = 0.3
        rows[:, Hf["width"]] = 0.05
        rows[:, Hf["n_pix"]] = 5
        tel = rng.uniform(-300, 300, (2, 2))
        out = oracle.stereo(rows, tel)
        u = np.stack([np.cos(rows[:, Hf["psi"]]), np.sin(rows[:, Hf["psi"]])], 1)
        A = np.stack([u[0], -u[1]], 1)
        if abs(np.linalg.det(A)) < 1e-3:
            continue
        s = np.linalg.solve(A, rows[1, [Hf["x"], Hf["y"]]] - rows[0, [Hf["x"], Hf["y"]]])
        p = rows[0, [Hf["x"], Hf["y"]]] + s[0] * u[0]
        g = tel[0] + np.linalg.solve(A, tel[1] - tel[0])[0] * u[0]
        np.testing.assert_allclose(out[:2], p, rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(out[2:4], g, rtol=1e-9, atol=1e-6)


def test_axis_flip_and_permutation_invariance():
    rng = np.random.default_rng(8)
    rows = np.zeros((6, 12))
    rows[:, Hf["x"]] = rng.uniform(-2, 2, 6)
    rows[:, Hf["y"]] = rng.uniform(-2, 2, 6)
    rows[:, Hf["psi"]] = rng.uniform(-1.5, 1.5, 6)
    rows[:, Hf["size"]] = rng.uniform(50, 500, 6)
    rows[:, Hf["length"]] = rng.uniform(0.1, 0.4, 6)
    rows[:, Hf["width"]] = rng.uniform(0.01, 0.09, 6)
    rows[:, Hf["n_pix"]] = 8
    tel = rng.uniform(-300, 300, (6, 2))
    a = oracle.stereo(rows, tel)
    flipped = rows.copy()
    flipped[::2, Hf["psi"]] += np.pi
    np.testing.assert_allclose(oracle.stereo(flipped, tel), a, rtol=1e-9, atol=1e-9)
    perm = rng.permutation(6)
    np.testing.assert_allclose(oracle.stereo(rows[perm], tel[perm]), a, rtol=1e-9, atol=1e-9)


def test_round_or_small_images_carry_no_weight():
    rng = np.random.default_rng(9)
    rows = np.zeros((3, 12))
    rows[:, Hf["x"]] = rng.uniform(-2, 2, 3)
    rows[:, Hf["y"]] = rng.uniform(-2, 2, 3)
    rows[:, Hf["psi"]] = [0.1, 1.0, -0.8]
    rows[:, Hf["size"]] = 100
    rows[:, Hf["length"]] = 0.3
    rows[:, Hf["width"]] = [0.05, 0.05, 0.3]      # image 2 is round
    rows[:, Hf["n_pix"]] = 10
    tel = rng.uniform(-300, 300, (3, 2))
    full = oracle.stereo(rows, tel)
    pair = oracle.stereo(rows[:2], tel[:2])
    np.testing.assert_allclose(full, np.r_[pair[:4], 3, 0], rtol=1e-12, atol=1e-12)
    rows[2, Hf["n_pix"]] = 2                       # fewer than 3 pixels: not used
    rows[2, Hf["width"]] = 0.05
    out = oracle.stereo(rows, tel)
    np.testing.assert_allclose(out[:4], pair[:4], rtol=1e-12)
    assert out[Sf["n_valid"]] == 2


def test_result_inside_hull_of_pairwise_intersections():
    rng = np.random.default_rng(10)
    rows = np.zeros((3, 12))
    rows[:, Hf["x"]] = rng.uniform(-1, 1, 3)
    rows[:, Hf["y"]] = rng.uniform(-1, 1, 3)
    rows[:, Hf["psi"]] = [0.2, 1.1, -0.9]
    rows[:, Hf["size"]] = [100, 300, 50]
    rows[:, Hf["length"]] = 0.3
    rows[:, Hf["width"]] = 0.05
    rows[:, Hf["n_pix"]] = 10
    tel = rng.uniform(-300, 300, (3, 2))
    out = oracle.stereo(rows, tel)
    pts = []
    for i, j in [(0, 1), (0, 2), (1, 2)]:
        pts.append(oracle.stereo(rows[[i, j]], tel[[i, j]])[:2])
    pts = np.array(pts)
    # barycentric coordinates of the result are all non-negative
    T = np.stack([pts[1] - pts[0], pts[2] - pts[0]], 1)
    lam = np.linalg.solve(T, out[:2] - pts[0])
    assert lam.min() >= -1e-9 and lam.sum() <= 1 + 1e-9


def test_degenerate_events():
    rows = np.zeros((2, 12))
    rows[:, Hf["psi"]] = [0.3, 0.3]
    rows[:, Hf["x"]] = [0.0, 1.0]
    rows[:, Hf["size"]] = 100
    rows[:, Hf["length"]] = 0.3
    rows[:, Hf["width"]] = 0.05
    rows[:, Hf["n_pix"]] = 10
    out = oracle.stereo(rows, np.zeros((2, 2)))
    assert out[Sf["flags"]] == oracle.FLAG_STEREO_INVALID       # parallel axes
    out = oracle.stereo(rows[:1], np.zeros((1, 2)))
    assert out[Sf["flags"]] == oracle.FLAG_STEREO_INVALID       # one image
