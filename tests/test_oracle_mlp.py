"""Pins of the oracle's deep-sets surrogate: gradients by central finite
differences, Adam against hand-computed steps, deep-sets invariances, the loss
at known points, the baseline geometry and bfloat16 rounding."""
import numpy as np
import pytest

from oracle import mlp


def small_params(rng, F=12, H=6, G=5):
    return {"W1": rng.normal(0, 0.5, (F, H)), "b1": rng.normal(0, 0.2, H), "W2": rng.normal(0, 0.5, (H, H)),
            "b2": rng.normal(0, 0.2, H), "V1": rng.normal(0, 0.5, (2 * H, G)), "c1": rng.normal(0, 0.2, G),
            "V2": rng.normal(0, 0.5, (G, 4)), "c2": rng.normal(0, 0.2, 4)}


def batch(rng, n_evt=7, F=12):
    m = rng.integers(1, 6, n_evt)
    evt_off = np.concatenate([[0], np.cumsum(m)])
    X = rng.normal(0, 1, (evt_off[-1], F))
    used = rng.uniform(size=evt_off[-1]) < 0.8
    logE = rng.normal(0, 1, n_evt)
    ddir = rng.normal(0, 0.2, (n_evt, 2))
    gam = rng.uniform(size=n_evt) < 0.5
    return X, used, evt_off, logE, ddir, gam


def total_loss(p, X, used, evt_off, logE, ddir, gam):
    y, _ = mlp.forward(p, X, used, evt_off)
    return mlp.loss(y, logE, ddir, gam)[0]


def test_backward_matches_central_finite_differences_everywhere():
    rng = np.random.default_rng(0)
    p = small_params(rng)
    args = batch(rng)
    y, cache = mlp.forward(p, *args[:3])
    L, dy = mlp.loss(y, *args[3:])
    g = mlp.backward(p, cache, dy)
    h = 1e-6
    for name, arr in p.items():
        fd = np.zeros_like(arr)
        for idx in np.ndindex(arr.shape):
            old = arr[idx]
            arr[idx] = old + h
            lp = total_loss(p, *args)
            arr[idx] = old - h
            lm = total_loss(p, *args)
            arr[idx] = old
            fd[idx] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(g[name], fd, rtol=1e-5, atol=1e-8, err_msg=name)


def test_backward_full_size_sampled_parameters():
    rng = np.random.default_rng(1)
    p = mlp.init_params(3)
    X, used, evt_off, logE, ddir, gam = batch(rng, n_evt=5)
    y, cache = mlp.forward(p, X, used, evt_off)
    L, dy = mlp.loss(y, logE, ddir, gam)
    g = mlp.backward(p, cache, dy)
    h = 1e-6
    for name, arr in p.items():
        for _ in range(12):
            idx = tuple(rng.integers(0, s) for s in arr.shape)
            old = arr[idx]
            arr[idx] = old + h
            lp = total_loss(p, X, used, evt_off, logE, ddir, gam)
            arr[idx] = old - h
            lm = total_loss(p, X, used, evt_off, logE, ddir, gam)
            arr[idx] = old
            assert g[name][idx] == pytest.approx((lp - lm) / (2 * h), rel=1e-4, abs=1e-8), (name, idx)


def test_adam_hand_computed_steps():
    # t = 1 from zero moments: m = 0.05, v = 0.00025, corrected 0.5 and 0.25 -> step lr * 0.5 / 0.5
    p, m, v = mlp.adam_step(np.array([1.0]), np.array([0.5]), np.zeros(1), np.zeros(1), 1, 0.1)
    assert m[0] == pytest.approx(0.05) and v[0] == pytest.approx(0.00025)
    assert p[0] == pytest.approx(1.0 - 0.1 * 0.5 / (0.5 + 1e-8), abs=1e-15)
    # t = 3, m = 0.2, v = 0.01, g = -1: m = 0.08, v = 0.01099; corrections 1 - 0.9^3, 1 - 0.999^3
    p, m, v = mlp.adam_step(np.array([2.0]), np.array([-1.0]), np.array([0.2]), np.array([0.01]), 3, 0.01)
    assert m[0] == pytest.approx(0.08) and v[0] == pytest.approx(0.01099)
    mh, vh = 0.08 / 0.271, 0.01099 / (1 - 0.999 ** 3)
    assert p[0] == pytest.approx(2.0 - 0.01 * mh / (np.sqrt(vh) + 1e-8), rel=1e-12)


def test_deep_sets_invariances():
    rng = np.random.default_rng(4)
    p = mlp.init_params(5)
    X = rng.normal(0, 1, (5, 12))
    used = np.array([True, True, False, True, True])
    y, _ = mlp.forward(p, X, used, np.array([0, 5]))
    perm = np.array([3, 0, 4, 2, 1])
    y2, _ = mlp.forward(p, X[perm], used[perm], np.array([0, 5]))
    np.testing.assert_allclose(y2, y, rtol=1e-12)                     # order of images is irrelevant
    X3 = X.copy()
    X3[2] = rng.normal(0, 5, 12)
    y3, _ = mlp.forward(p, X3, used, np.array([0, 5]))
    np.testing.assert_allclose(y3, y, rtol=1e-12)                     # an unused image is ignored
    # duplicating every used image doubles the sum half of the pool and keeps the mean half
    Xd = np.concatenate([X[used], X[used]])
    _, c1 = mlp.forward(p, X[used], np.ones(4, bool), np.array([0, 4]))
    _, c2 = mlp.forward(p, Xd, np.ones(8, bool), np.array([0, 8]))
    H = 128
    np.testing.assert_allclose(c2["pool"][0, :H], 2 * c1["pool"][0, :H], rtol=1e-12)
    np.testing.assert_allclose(c2["pool"][0, H:], c1["pool"][0, H:], rtol=1e-12)


def test_loss_known_points():
    y = np.zeros((2, 4))
    L, dy = mlp.loss(y, np.zeros(2), np.zeros((2, 2)), np.array([True, False]))
    assert L == pytest.approx(np.log(2.0))                           # BCE at logit 0, no regression error
    assert dy[:, 3] == pytest.approx([(0.5 - 1) / 2, 0.5 / 2])
    y = np.array([[1.0, 0.1, -0.2, 0.0]])
    L, _ = mlp.loss(y, np.array([0.5]), np.array([[0.0, 0.0]]), np.array([True]))
    assert L == pytest.approx(0.25 + (0.01 + 0.04) / 0.01 + np.log(2.0))


def test_baseline_geometry():
    # two bright images whose axes cross at (0.3, -0.2); a faint third one is ignored
    src = np.array([0.3, -0.2])
    rows = np.zeros((3, 12))
    for i, (ang, off, size) in enumerate([(0.4, 0.5, 900.0), (1.9, 0.8, 700.0), (-1.0, 0.3, 50.0)]):
        u = np.array([np.cos(ang), np.sin(ang)])
        rows[i, [1, 2]] = src + off * u
        rows[i, 5] = ang if ang <= np.pi / 2 else ang - np.pi
        rows[i, 0] = size
        rows[i, 10] = 10
    b = mlp.baseline(rows, mlp.used_images(rows))
    np.testing.assert_allclose(b, src, atol=1e-12)
    # nearly parallel brightest pair: size-weighted mean centroid
    rows[1, 5] = rows[0, 5] + 0.01
    b = mlp.baseline(rows, mlp.used_images(rows))
    w = rows[:, 0]
    np.testing.assert_allclose(b, (w[:, None] * rows[:, [1, 2]]).sum(0) / w.sum(), atol=1e-12)
    rows[:, 10] = 2                                                  # nothing used
    np.testing.assert_allclose(mlp.baseline(rows, mlp.used_images(rows)), [0, 0])


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -7, -2.5, 3.0e38], np.float32)
    r = mlp.bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0                              # tie to even
    assert r[2] == 1.0 + 2 ** -6                                     # tie to even upwards
    assert r[3] == 1.0 + 2 ** -7 and r[4] == -2.5
    assert abs(r[5] / 3.0e38 - 1) < 2 ** -8


def test_feature_rows_written_out_by_hand():
    """Every one of the 12 feature columns, for hand-built events, against values
    worked out on paper from the feature definition (log10 size, centroid minus
    baseline, length, width, cos 2psi, sin 2psi, time gradient / 10, distance to
    the baseline, camera code, telescope x and y in km). A slip such as cos psi
    for cos 2psi, a missing /10, x instead of x - b_x, or the brightest pair taken
    over unused images changes at least one entry."""
    PI = np.pi
    tel_xy = np.array([[100.0, -200.0], [250.0, 1000.0]])
    tel_code = np.array([0.5, -0.25])

    def row(size, x, y, L, W, psi, tg, npix, flags=0):
        r = np.zeros(12)
        r[[0, 1, 2, 3, 4, 5, 8, 10, 11]] = [size, x, y, L, W, psi, tg, npix, flags]
        return r

    rows = np.array([
        # event 0: brightest used A (psi 0) and B (psi pi/4); C is brighter than B but has 2 pixels.
        # A's axis y = 0.25 meets B's axis (-0.5 + t, 0.75 + t) at t = -0.5: b = (-1.0, 0.25)
        row(1000.0, 0.5, 0.25, 0.25, 0.125, 0.0, 2.5, 10),
        row(100.0, -0.5, 0.75, 0.5, 0.0625, PI / 4, -5.0, 7, flags=2),   # NO_TIME does not exclude
        row(500.0, 2.0, 2.0, 0.1, 0.1, PI / 4, 0.0, 2),
        # event 1: one used image (the other is flagged BAD_INPUT): b = its centroid
        row(10.0, 0.125, -0.375, 0.2, 0.05, -PI / 4, 1.0, 5),
        row(4000.0, 1.0, 1.0, 0.3, 0.1, 0.0, 0.0, 40, flags=4),
        # event 2: the brightest pair is parallel (|sin| = 0 < 0.1): size-weighted mean of the
        # used images, b = ((300 - 100) / 400, (0 + 40) / 400) = (0.5, 0.1)
        row(300.0, 1.0, 0.0, 0.2, 0.1, 0.0, 0.0, 9),
        row(100.0, -1.0, 0.4, 0.2, 0.1, 0.0, 0.0, 9),
        # event 3: three equal sizes; ties go to the lower index, so the pair is images 0 and 1
        # of the event (parallel, psi = 0): the mean of all three, b = (0, 0.5); the pair
        # (0, 2) would have crossed at (0.5, 0)
        row(200.0, 0.0, 0.0, 0.2, 0.1, 0.0, 0.0, 9),
        row(200.0, -1.5, 0.5, 0.2, 0.1, 0.0, 0.0, 9),
        row(200.0, 1.5, 1.0, 0.2, 0.1, PI / 4, 0.0, 9),
        # event 4: an empty image only: b = (0, 0), log10 of the 1e-3 floor
        row(0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0, flags=1),
    ])
    evt_off = np.array([0, 3, 5, 7, 10, 11])
    img_tel = np.array([0, 1, 0, 1, 0, 0, 1, 1, 0, 1, 0])
    X, used, base, n_used = mlp.features(rows, evt_off, img_tel, tel_xy, tel_code)
    T0 = [0.5, 0.1, -0.2]          # code, x / km, y / km of telescope 0
    T1 = [-0.25, 0.25, 1.0]
    r2 = np.sqrt(0.5)
    expect = np.array([
        [3.0, 1.5, 0.0, 0.25, 0.125, 1.0, 0.0, 0.25, 1.5] + T0,
        [2.0, 0.5, 0.5, 0.5, 0.0625, 0.0, 1.0, -0.5, r2] + T1,
        [np.log10(500.0), 3.0, 1.75, 0.1, 0.1, 0.0, 1.0, 0.0, np.hypot(3.0, 1.75)] + T0,
        [1.0, 0.0, 0.0, 0.2, 0.05, 0.0, -1.0, 0.1, 0.0] + T1,
        [np.log10(4000.0), 0.875, 1.375, 0.3, 0.1, 1.0, 0.0, 0.0, np.hypot(0.875, 1.375)] + T0,
        [np.log10(300.0), 0.5, -0.1, 0.2, 0.1, 1.0, 0.0, 0.0, np.hypot(0.5, 0.1)] + T0,
        [2.0, -1.5, 0.3, 0.2, 0.1, 1.0, 0.0, 0.0, np.hypot(1.5, 0.3)] + T1,
        [np.log10(200.0), 0.0, -0.5, 0.2, 0.1, 1.0, 0.0, 0.0, 0.5] + T1,
        [np.log10(200.0), -1.5, 0.0, 0.2, 0.1, 1.0, 0.0, 0.0, 1.5] + T0,
        [np.log10(200.0), 1.5, 0.5, 0.2, 0.1, 0.0, 1.0, 0.0, np.hypot(1.5, 0.5)] + T1,
        [-3.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0] + T0,
    ])
    np.testing.assert_allclose(X, expect, rtol=0, atol=1e-12)
    np.testing.assert_allclose(base, [[-1.0, 0.25], [0.125, -0.375], [0.5, 0.1], [0.0, 0.5], [0.0, 0.0]],
                               rtol=0, atol=1e-12)
    np.testing.assert_array_equal(used, [1, 1, 0, 1, 0, 1, 1, 1, 1, 1, 0])
    np.testing.assert_array_equal(n_used, [2, 1, 2, 3, 0])
