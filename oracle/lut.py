"""Lookup-table reconstruction oracle -- TEST INFRASTRUCTURE ONLY (imported by
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg).

The real-time reconstruction gets energy and gamma/hadron separation from
"calibration matrices" (Sec. 4.1). The paper does not define them. Here they
are the classic lookup tables of imaging Cherenkov arrays: for each camera
type, a grid over (image size, impact distance) whose cells hold the mean and
the standard deviation of the image width, the image length and log10 of the
true energy of simulated gamma-ray images. An event's images are scaled by
their cells (mean scaled width and length) and its energy is the
inverse-variance weighted mean of the cells' energies.

Decisions that floating point takes (the bin of a size, the impact distance
that picks a distance bin) are made in FP32 with one rounding per operation,
the precision the event rows are stored in. Everything after the lookup is
FP64, summed in image order; each operation is a single IEEE rounding.

Cell layout (one row of 8 per cell, index ((cam * n_size) + i_size) * n_dist
+ i_dist): n, mean_w, sigma_w, mean_l, sigma_l, mean_e, sigma_e, 0.
Event row (6 values): log_energy, sigma_log_energy, mscw, mscl, n_used, flags.
"""
from __future__ import annotations

import math

import numpy as np

N_CAMS = 16
MIN_PIX = 3                 # images the stereo step uses: at least 3 cleaned pixels
SKIP_FLAGS = 1 | 4          # ... and neither empty nor skipped as bad input
CELL_FIELDS = ["n", "mean_w", "sigma_w", "mean_l", "sigma_l", "mean_e", "sigma_e"]
EVENT_FIELDS = ["log_energy", "sigma_log_energy", "mscw", "mscl", "n_used", "flags"]
LF_GAMMA = 1                # the event passed the scaled-width and scaled-length box
LF_NO_CORE = 2              # no stereo reconstruction: no impact distances
LF_NO_IMAGE = 4             # no image fell into a filled cell
LF_MALFORMED = 8            # the event's image range is not inside [0, n_img]


def bin_index(v, edges):
    """i with edges[i] <= v < edges[i + 1] (FP32 comparisons), -1 outside or NaN."""
    v = np.float32(v)
    if not (v >= edges[0]) or not (v < edges[-1]):
        return -1
    i = int(np.searchsorted(edges, v, side="right")) - 1
    return i


def impact_distance(core_x, core_y, tel_x, tel_y):
    """Ground distance from a telescope to the shower core, FP32 with one
    rounding per operation: sqrt(dx*dx + dy*dy)."""
    f = np.float32
    dx = f(f(core_x) - f(tel_x))
    dy = f(f(core_y) - f(tel_y))
    return f(np.sqrt(f(f(dx * dx) + f(dy * dy))))


def _check_edges(edges):
    e = np.ascontiguousarray(edges, np.float32)
    if e.ndim != 1 or len(e) < 2 or not np.all(np.diff(e) > 0):
        raise ValueError("edges must be at least two strictly increasing values")
    return e


def lut_build(hrows, img_tel, evt_off, tel_cam, tel_xy, log_energy, core_xy, use, size_edges, dist_edges,
              min_count):
    """The cells from training events with known truth. hrows: Hillas rows
    (n_img, 12) as the oracle lays them out; log_energy (n_evt,) and core_xy
    (n_evt, 2) the events' true log10 E and impact point; use: events to take
    (gamma showers), None = all; events whose image range is not inside
    [0, n_img] are skipped. An image (the rule of _image_ok) enters cell
    (camera type, size bin, true-impact-distance bin) when both bins exist.
    Mean and population standard deviation per quantity; cells with fewer
    than min_count images keep n and get zeros elsewhere (unused).
    Returns (cells (N_CAMS * n_size * n_dist, 8) float32, n as int64)."""
    from . import H
    se, de = _check_edges(size_edges), _check_edges(dist_edges)
    n_size, n_dist = len(se) - 1, len(de) - 1
    n_cells = N_CAMS * n_size * n_dist
    hrows = np.asarray(hrows, np.float64)
    tel_xy = np.asarray(tel_xy, np.float32).reshape(-1, 2)
    cnt = np.zeros(n_cells, np.int64)
    s = np.zeros((n_cells, 3))          # sums of width, length, log E
    s2 = np.zeros((n_cells, 3))         # sums of squares
    n_img, n_tel = len(hrows), len(tel_cam)
    for e in range(len(evt_off) - 1):
        a, b = int(evt_off[e]), int(evt_off[e + 1])
        if (use is not None and not use[e]) or a < 0 or b < a or b > n_img:
            continue
        for i in range(a, b):
            h = hrows[i]
            t = int(img_tel[i])
            if not _image_ok(h, t, n_tel, H):
                continue
            cam = int(tel_cam[t])
            iu = bin_index(h[H["size"]], se)
            r = impact_distance(core_xy[e][0], core_xy[e][1], tel_xy[t, 0], tel_xy[t, 1])
            ir = bin_index(r, de)
            if iu < 0 or ir < 0:
                continue
            c = (cam * n_size + iu) * n_dist + ir
            v = np.array([np.float32(h[H["width"]]), np.float32(h[H["length"]]), np.float32(log_energy[e])],
                         np.float64)
            cnt[c] += 1
            s[c] += v
            s2[c] += v * v
    cells = np.zeros((n_cells, 8), np.float32)
    cells[:, 0] = cnt.astype(np.float32)
    full = cnt >= max(int(min_count), 1)
    n = cnt[full].astype(np.float64)[:, None]
    mean = s[full] / n
    var = np.maximum(s2[full] / n - mean * mean, 0.0)
    sd = np.sqrt(var)
    for k in range(3):
        cells[full, 1 + 2 * k] = mean[:, k].astype(np.float32)
        cells[full, 2 + 2 * k] = sd[:, k].astype(np.float32)
    return cells, cnt


def _image_ok(h, t, n_tel, H):
    """An image counts when its telescope id exists, it kept at least MIN_PIX
    pixels and is neither empty nor skipped as bad input (the stereo rule)."""
    return 0 <= t < n_tel and h[H["n_pix"]] >= MIN_PIX and not (int(h[H["flags"]]) & SKIP_FLAGS)


def _cell_ok(cell):
    return cell[0] >= 1 and cell[2] > 0 and cell[4] > 0 and cell[6] > 0


def lut_reconstruct(hrows, img_tel, evt_off, n_img, tel_cam, tel_xy, srows, cells, size_edges, dist_edges,
                    cuts):
    """Energy and scaled parameters of each event from the cells. srows: stereo
    rows (n_evt, 6) as the oracle lays them out, the core taken from there;
    cuts: (mscw_lo, mscw_hi, mscl_lo, mscl_hi), the gamma box (inclusive).
    Per used image (a known telescope, at least MIN_PIX pixels, neither empty
    nor bad input, both bins exist, the cell filled):
      scaled width   (w - mean_w) * (1 / sigma_w), likewise the length (the
                     reciprocal is a property of the cell, rounded once);
      weight         1 / sigma_e^2, estimate mean_e.
    mscw, mscl = the scaled values summed in image order over the images, / n;
    log_energy = sum(weight * estimate) / sum(weight); sigma = sqrt(1 / sum(weight)).
    Returns (n_evt, 6) float64 rows; the four values are what FP32 storage keeps."""
    from . import H, S, FLAG_STEREO_INVALID
    se, de = _check_edges(size_edges), _check_edges(dist_edges)
    n_size, n_dist = len(se) - 1, len(de) - 1
    cells = np.asarray(cells, np.float32).reshape(N_CAMS * n_size * n_dist, 8)
    tel_xy = np.asarray(tel_xy, np.float32).reshape(-1, 2)
    hrows = np.asarray(hrows, np.float64)
    srows = np.asarray(srows, np.float64)
    lo_w, hi_w, lo_l, hi_l = (float(np.float32(c)) for c in cuts)
    n_evt = len(evt_off) - 1
    out = np.zeros((n_evt, 6))
    for e in range(n_evt):
        a, b = int(evt_off[e]), int(evt_off[e + 1])
        if a < 0 or b < a or b > n_img:
            out[e, 4], out[e, 5] = -1, LF_MALFORMED
            continue
        if int(srows[e, S["flags"]]) & FLAG_STEREO_INVALID:
            out[e, 5] = LF_NO_CORE
            continue
        cx, cy = np.float32(srows[e, S["core_x"]]), np.float32(srows[e, S["core_y"]])
        sw = sl = num = den = 0.0
        n = 0
        for i in range(a, b):
            h = hrows[i]
            t = int(img_tel[i])
            if not _image_ok(h, t, len(tel_cam), H):
                continue
            iu = bin_index(h[H["size"]], se)
            ir = bin_index(impact_distance(cx, cy, tel_xy[t, 0], tel_xy[t, 1]), de)
            if iu < 0 or ir < 0:
                continue
            cell = cells[(int(tel_cam[t]) * n_size + iu) * n_dist + ir]
            if not _cell_ok(cell):
                continue
            w, ln = float(np.float32(h[H["width"]])), float(np.float32(h[H["length"]]))
            sw += (w - float(cell[1])) * (1.0 / float(cell[2]))
            sl += (ln - float(cell[3])) * (1.0 / float(cell[4]))
            se2 = float(cell[6]) * float(cell[6])
            wt = 1.0 / se2
            num += float(cell[5]) * wt
            den += wt
            n += 1
        if n == 0:
            out[e, 5] = LF_NO_IMAGE
            continue
        mscw, mscl = sw / n, sl / n
        flags = LF_GAMMA if (lo_w <= mscw <= hi_w and lo_l <= mscl <= hi_l) else 0
        out[e] = (num / den, math.sqrt(1.0 / den), mscw, mscl, n, flags)
    return out
