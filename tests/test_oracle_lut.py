"""The lookup-table oracle (energy and scaled width/length from per-cell gamma
statistics, the "calibration matrices" of Sec. 4.1) pinned to what its
definition fixes: bin edges by brute force, the impact distance against an FP64
hypot, cell statistics of hand-placed images in closed form, planted per-cell
distributions recovered, the zero-mean unit-variance identity of scaled
training images, event combinations in closed form, and a separation of gamma
rays from protons on generated showers."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import lut

H = oracle.H
SIZE_EDGES = np.float32(10.0) ** np.linspace(1.0, 5.0, 17, dtype=np.float32)
DIST_EDGES = np.linspace(0.0, 800.0, 17, dtype=np.float32)


def hrow(size, width, length, n_pix=10):
    r = np.zeros(12)
    r[H["size"]], r[H["width"]], r[H["length"]], r[H["n_pix"]] = size, width, length, n_pix
    return r


def srow(core_x, core_y, invalid=False):
    r = np.zeros(6)
    r[oracle.S["core_x"]], r[oracle.S["core_y"]] = core_x, core_y
    r[oracle.S["flags"]] = oracle.FLAG_STEREO_INVALID if invalid else 0
    return r


def test_bin_index_matches_a_linear_scan():
    rng = np.random.default_rng(1)
    e = np.float32([1.0, 2.5, 2.75, 10.0, 1e4])
    vals = np.concatenate([rng.uniform(0, 2e4, 300), e, np.nextafter(e, np.float32(0)), np.nextafter(e, np.float32(1e9)),
                           [np.nan, -1.0, np.inf]]).astype(np.float32)
    for v in vals:
        want = -1
        for i in range(len(e) - 1):
            if e[i] <= v < e[i + 1]:
                want = i
        assert lut.bin_index(v, e) == want, v
    assert lut.bin_index(np.float32(2.5), e) == 1          # an edge belongs to the bin above it
    assert lut.bin_index(np.float32(1e4), e) == -1         # the last edge closes the grid


def test_impact_distance_is_the_fp32_rounded_ground_distance():
    rng = np.random.default_rng(2)
    for _ in range(500):
        c = rng.uniform(-1500, 1500, 2).astype(np.float32)
        t = rng.uniform(-1500, 1500, 2).astype(np.float32)
        r = lut.impact_distance(c[0], c[1], t[0], t[1])
        exact = math.hypot(float(c[0]) - float(t[0]), float(c[1]) - float(t[1]))
        assert r.dtype == np.float32
        assert abs(float(r) - exact) <= 3 * np.spacing(np.float32(exact)) + 1e-30
    assert lut.impact_distance(100.0, 250.0, 100.0, 0.0) == np.float32(250.0)
    assert lut.impact_distance(3.0, 4.0, 0.0, 0.0) == np.float32(5.0)


def _one_telescope_array():
    tel_cam = np.array([2, 0], np.int32)
    tel_xy = np.float32([[100.0, 0.0], [-50.0, 30.0]])
    return tel_cam, tel_xy


def test_cell_statistics_of_hand_placed_images():
    """Four images of telescope 0 (camera 2) in one cell: widths 1, 2, 3, 4 give
    mean 2.5 and population deviation sqrt(1.25); a second cell with fewer
    images than min_count keeps only its count."""
    tel_cam, tel_xy = _one_telescope_array()
    se = np.float32([10.0, 100.0, 1000.0])
    de = np.float32([0.0, 200.0, 400.0])
    rows = [hrow(150.0, w, 2 * w + 1) for w in (1.0, 2.0, 3.0, 4.0)]     # size bin 1
    rows.append(hrow(50.0, 0.3, 0.5))                                     # size bin 0, alone in its cell
    rows.append(hrow(50.0, 0.3, 0.5, n_pix=2))                            # too few pixels: ignored
    rows.append(hrow(5000.0, 0.3, 0.5))                                   # above the size grid: ignored
    hrows = np.array(rows)
    img_tel = np.zeros(len(rows), np.int32)
    evt_off = np.arange(len(rows) + 1, dtype=np.int32)
    core = np.float32([[100.0, 250.0]] * len(rows))                       # 250 m from the telescope: bin 1
    loge = np.float32([0.5, 0.5, 1.5, 1.5, 0.0, 0.0, 0.0])
    cells, n = lut.lut_build(hrows, img_tel, evt_off, tel_cam, tel_xy, loge, core, None, se, de, min_count=2)
    c1 = (2 * 2 + 1) * 2 + 1
    c0 = (2 * 2 + 0) * 2 + 1
    assert n.sum() == 5 and n[c1] == 4 and n[c0] == 1
    assert cells[c1, 1] == np.float32(2.5) and cells[c1, 2] == np.float32(math.sqrt(1.25))
    assert cells[c1, 3] == np.float32(6.0) and cells[c1, 4] == np.float32(2 * math.sqrt(1.25))
    assert cells[c1, 5] == np.float32(1.0) and cells[c1, 6] == np.float32(0.5)
    assert cells[c0, 0] == 1 and not cells[c0, 1:].any()
    # the use mask drops events
    use = np.array([1, 1, 0, 0, 1, 1, 1], np.uint8)
    cells, n = lut.lut_build(hrows, img_tel, evt_off, tel_cam, tel_xy, loge, core, use, se, de, min_count=2)
    assert n[c1] == 2 and cells[c1, 1] == np.float32(1.5) and cells[c1, 6] == 0.0


def test_planted_cell_distributions_are_recovered():
    """Images drawn from per-cell normal distributions whose means depend
    differently on camera, size bin and distance bin: the built cells find
    those means and deviations (a swapped axis or camera index would not)."""
    rng = np.random.default_rng(3)
    tel_cam = np.array([0, 1, 0, 1], np.int32)
    tel_xy = np.float32([[0, 0], [200, 0], [0, 200], [200, 200]])
    se = np.float32([10.0, 100.0, 1000.0, 10000.0])
    de = np.float32([0.0, 150.0, 300.0])
    mu = lambda cam, iu, ir: (0.05 + 0.02 * cam + 0.03 * iu + 0.011 * ir, 0.1 + 0.05 * iu + 0.02 * ir,
                              -0.5 + 0.9 * iu + 0.13 * ir + 0.07 * cam)
    sd = lambda cam, iu, ir: (0.01 + 0.003 * iu, 0.02 + 0.004 * ir, 0.1 + 0.02 * cam)
    n = 12000
    t = rng.integers(0, 4, n)
    iu = rng.integers(0, 3, n)
    ir = rng.integers(0, 2, n)
    size = np.float32(10.0) ** (iu + rng.uniform(1.05, 1.95, n))
    ang = rng.uniform(0, 2 * np.pi, n)
    r = (ir + rng.uniform(0.05, 0.95, n)) * 150.0
    core = np.stack([tel_xy[t, 0] + r * np.cos(ang), tel_xy[t, 1] + r * np.sin(ang)], 1).astype(np.float32)
    rows, loge = [], []
    for k in range(n):
        m, s = mu(tel_cam[t[k]], iu[k], ir[k]), sd(tel_cam[t[k]], iu[k], ir[k])
        v = [rng.normal(m[j], s[j]) for j in range(3)]
        rows.append(hrow(size[k], v[0], v[1]))
        loge.append(v[2])
    cells, cnt = lut.lut_build(np.array(rows), t.astype(np.int32), np.arange(n + 1, dtype=np.int32), tel_cam, tel_xy,
                               np.float32(loge), core, None, se, de, min_count=10)
    assert cnt.sum() == n
    for cam in (0, 1):
        for a in range(3):
            for b in range(2):
                c = (cam * 3 + a) * 2 + b
                m, s = mu(cam, a, b), sd(cam, a, b)
                k = cnt[c]
                assert k > 500
                for j in range(3):
                    assert abs(cells[c, 1 + 2 * j] - m[j]) < 5 * s[j] / math.sqrt(k), (cam, a, b, j)
                    assert abs(cells[c, 2 + 2 * j] / s[j] - 1) < 5 / math.sqrt(2 * k), (cam, a, b, j)


def _hand_table():
    """Camera 2, size bins [10, 100), [100, 1000); distance bins [0, 200), [200, 400)."""
    se = np.float32([10.0, 100.0, 1000.0])
    de = np.float32([0.0, 200.0, 400.0])
    cells = np.zeros((16 * 2 * 2, 8), np.float32)
    idx = lambda cam, a, b: (cam * 2 + a) * 2 + b
    cells[idx(2, 1, 1)] = [50, 0.25, 0.5, 1.0, 0.25, 1.25, 0.5, 0]
    cells[idx(2, 0, 1)] = [80, 0.125, 0.25, 0.5, 0.125, 0.75, 0.25, 0]
    cells[idx(2, 0, 0)] = [80, 0.125, 0.0, 0.5, 0.125, 0.75, 0.25, 0]      # sigma_w = 0: unused
    return cells, se, de


def test_event_combination_in_closed_form():
    tel_cam, tel_xy = _one_telescope_array()
    cells, se, de = _hand_table()
    cuts = (-1.0, 1.0, -2.0, 2.0)
    rows = [hrow(500.0, 0.75, 1.5), hrow(50.0, 0.0, 0.25),        # event 0: two used images
            hrow(50.0, 0.5, 0.5), hrow(500.0, 2.0, 1.0, n_pix=2),  # event 1: one used, one too small
            hrow(500.0, 0.25, 1.0),                                # event 2: stereo invalid
            hrow(50.0, 0.3, 0.3),                                  # event 3: its cell has sigma 0
            hrow(5.0, 0.3, 0.3),                                   # event 4: below the size grid
            hrow(500.0, 0.25, 1.0)]                                # event 5: malformed range
    hrows = np.array(rows)
    img_tel = np.zeros(len(rows), np.int32)
    evt_off = np.array([0, 2, 4, 5, 6, 7, 9], np.int32)
    st = np.array([srow(100.0, 250.0), srow(100.0, 250.0), srow(0.0, 0.0, invalid=True), srow(100.0, 50.0),
                   srow(100.0, 250.0), srow(100.0, 250.0)])
    out = lut.lut_reconstruct(hrows, img_tel, evt_off, len(rows), tel_cam, tel_xy, st, cells, se, de, cuts)
    # event 0: scaled widths (0.75-0.25)/0.5 = 1 and (0-0.125)/0.25 = -0.5; lengths (1.5-1)/0.25 = 2 and
    # (0.25-0.5)/0.125 = -2; energies 1.25 (sigma 0.5, weight 4) and 0.75 (sigma 0.25, weight 16)
    assert out[0, 2] == 0.25 and out[0, 3] == 0.0 and out[0, 4] == 2
    assert out[0, 0] == (1.25 * 4 + 0.75 * 16) / 20 and out[0, 1] == math.sqrt(1 / 20)
    assert out[0, 5] == oracle.lut.LF_GAMMA
    # event 1: one image, (0.5-0.125)/0.25 = 1.5 > 1: outside the box
    assert list(out[1]) == [0.75, 0.25, 1.5, 0.0, 1, 0]
    assert out[2, 5] == lut.LF_NO_CORE and out[2, 4] == 0
    assert out[3, 5] == lut.LF_NO_IMAGE and out[4, 5] == lut.LF_NO_IMAGE
    assert out[5, 5] == lut.LF_MALFORMED and out[5, 4] == -1
    # the box is inclusive
    out = lut.lut_reconstruct(hrows, img_tel, evt_off, len(rows), tel_cam, tel_xy, st, cells, se, de,
                              (-1.0, 1.5, 0.0, 0.0))
    assert out[1, 5] == lut.LF_GAMMA and out[0, 5] == lut.LF_GAMMA
    out = lut.lut_reconstruct(hrows, img_tel, evt_off, len(rows), tel_cam, tel_xy, st, cells, se, de,
                              (0.3, 1.5, 0.0, 0.0))
    assert out[1, 5] == lut.LF_GAMMA and out[0, 5] == 0


def test_training_images_scale_to_zero_mean_and_unit_variance():
    """Reconstructing the training images themselves (one image per event, the
    true core as the stereo core) gives, in every cell, scaled widths and
    lengths of mean 0 and population variance 1, and energy residuals of mean 0:
    the build and the lookup agree on sign, scale and cell."""
    rng = np.random.default_rng(4)
    tel_cam, tel_xy = np.array([0, 3], np.int32), np.float32([[0, 0], [120, -40]])
    n = 3000
    t = rng.integers(0, 2, n).astype(np.int32)
    size = (10.0 ** rng.uniform(1.2, 4.8, n)).astype(np.float32)
    core = (tel_xy[t] + rng.uniform(-500, 500, (n, 2))).astype(np.float32)
    rows = [hrow(size[k], rng.gamma(4, 0.02), rng.gamma(6, 0.03)) for k in range(n)]
    loge = rng.normal(0, 0.5, n).astype(np.float32)
    hrows = np.array(rows)
    evt_off = np.arange(n + 1, dtype=np.int32)
    cells, cnt = lut.lut_build(hrows, t, evt_off, tel_cam, tel_xy, loge, core, None, SIZE_EDGES, DIST_EDGES, 2)
    st = np.array([srow(c[0], c[1]) for c in core])
    out = lut.lut_reconstruct(hrows, t, evt_off, n, tel_cam, tel_xy, st, cells, SIZE_EDGES, DIST_EDGES,
                              (-1, 1, -1, 1))
    used = out[:, 4] == 1
    assert used.sum() > 0.9 * n
    cell_of = []
    for k in range(n):
        a = lut.bin_index(size[k], SIZE_EDGES)
        b = lut.bin_index(lut.impact_distance(core[k, 0], core[k, 1], tel_xy[t[k], 0], tel_xy[t[k], 1]), DIST_EDGES)
        cell_of.append((tel_cam[t[k]] * 16 + a) * 16 + b)
    cell_of = np.array(cell_of)
    for c in np.unique(cell_of[used]):
        sel = used & (cell_of == c)
        k = sel.sum()
        assert k == cnt[c]
        for col, j in ((2, 1), (3, 3)):
            # exact with FP64 cell statistics; the FP32 mean and deviation move
            # every scaled value by at most d = ulp(mean) / sigma
            v = out[sel, col]
            d = float(np.spacing(cells[c, j])) / float(cells[c, j + 1])
            assert abs(v.sum()) <= k * (d + 1e-9)
            assert abs((v * v).sum() - k) <= k * (4e-7 + 2 * d + d * d)
        assert np.float32(out[sel, 0][0]) == cells[c, 5]          # one image: its cell's energy
        assert abs((loge[sel] - out[sel, 0]).sum()) <= 1e-5 * k


def test_image_order_only_changes_rounding():
    rng = np.random.default_rng(5)
    tel_cam, tel_xy = _one_telescope_array()
    cells, se, de = _hand_table()
    n_evt, m = 50, 6
    rows = [hrow(rng.uniform(10, 999), rng.uniform(0, 1), rng.uniform(0, 2)) for _ in range(n_evt * m)]
    hrows = np.array(rows)
    img_tel = np.zeros(len(rows), np.int32)
    evt_off = np.arange(0, n_evt * m + 1, m, dtype=np.int32)
    st = np.array([srow(100.0 + rng.uniform(-150, 150), rng.uniform(-150, 150)) for _ in range(n_evt)])
    a = lut.lut_reconstruct(hrows, img_tel, evt_off, len(rows), tel_cam, tel_xy, st, cells, se, de, (-1, 1, -1, 1))
    perm = np.concatenate([e * m + rng.permutation(m) for e in range(n_evt)])
    b = lut.lut_reconstruct(hrows[perm], img_tel, evt_off, len(rows), tel_cam, tel_xy, st, cells, se, de,
                            (-1, 1, -1, 1))
    np.testing.assert_allclose(a[:, :4], b[:, :4], rtol=1e-13, atol=1e-13)
    assert (a[:, 4:] == b[:, 4:]).all()


@pytest.fixture(scope="module")
def showers():
    """Generated gamma and proton showers through the oracle's image and stereo steps."""
    tr = synth.make_workload(3, 2400, seed=71)
    te = synth.make_workload(3, 1200, seed=72, calib_seed=tr.seed)
    return [(w, oracle.reconstruct(w)) for w in (tr, te)]


def test_tables_from_generated_gammas_separate_gammas_and_estimate_energy(showers):
    (tr, rt), (te, re) = showers
    gam = tr.truth[:, 5] == 0
    cells, cnt = lut.lut_build(rt["hillas"], tr.img_tel, tr.evt_off, tr.tel_cam, tr.tel_xy,
                               np.log10(tr.truth[:, 0]).astype(np.float32), tr.truth[:, 3:5].astype(np.float32),
                               gam, SIZE_EDGES, DIST_EDGES, min_count=5)
    assert (cnt >= 5).sum() > 20
    out = lut.lut_reconstruct(re["hillas"], te.img_tel, te.evt_off, te.n_img, te.tel_cam, te.tel_xy, re["stereo"],
                              cells, SIZE_EDGES, DIST_EDGES, (-2.0, 2.0, -2.0, 2.0))
    g = te.truth[:, 5] == 0
    ok = (out[:, 5].astype(int) & (lut.LF_NO_CORE | lut.LF_NO_IMAGE | lut.LF_MALFORMED)) == 0
    assert (ok & g).sum() > 200 and (ok & ~g).sum() > 50
    # scaled widths of gammas sit near 0 with spread near 1 / sqrt(images); protons are wider
    assert abs(np.median(out[ok & g, 2])) < 0.5
    assert np.median(out[ok & ~g, 2]) > np.median(out[ok & g, 2]) + 1.0
    eff_g = np.mean(out[ok & g, 5].astype(int) & lut.LF_GAMMA)
    eff_p = np.mean(out[ok & ~g, 5].astype(int) & lut.LF_GAMMA)
    assert eff_g > 0.8 and eff_p < 0.5 * eff_g
    de = out[ok & g, 0] - np.log10(te.truth[ok & g, 0])
    assert abs(np.median(de)) < 0.1 and np.std(de) < 0.35


def test_unknown_telescopes_flagged_images_and_malformed_events_are_left_out():
    tel_cam, tel_xy = _one_telescope_array()
    cells, se, de = _hand_table()
    good = hrow(500.0, 0.75, 1.5)
    bad_flag = hrow(500.0, 0.75, 1.5)
    bad_flag[H["flags"]] = 4
    hrows = np.array([good, good, bad_flag, good])
    img_tel = np.array([0, 7, 0, -1], np.int32)
    evt_off = np.array([0, 4], np.int32)
    out = lut.lut_reconstruct(hrows, img_tel, evt_off, 4, tel_cam, tel_xy, np.array([srow(100.0, 250.0)]), cells, se,
                              de, (-9, 9, -9, 9))
    assert out[0, 4] == 1 and out[0, 2] == 1.0
    # the build skips them too, and events whose range leaves [0, n_img]
    core = np.float32([[100.0, 250.0]] * 3)
    cl, n = lut.lut_build(hrows, img_tel, np.array([0, 4, 2, 9], np.int32), tel_cam, tel_xy, np.float32([1, 1, 1]),
                          core, None, se, de, 1)
    assert n.sum() == 1
