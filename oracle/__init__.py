"""CPU oracle of the reconstruction path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the ``librta`` CUDA library
and its binding) never loads it and shares no code with it.

``oracle.c`` holds the arithmetic (plain C, FP64 except the one deliberate FP32
calibration multiply); this module only marshals numpy arrays.  Row layouts:

  hillas row (12 doubles): size, x, y, length, width, psi, r, phi,
                           time_grad, time_mean, n_pix, flags
  stereo row (6 doubles):  dir_x, dir_y (deg), core_x, core_y (m), n_valid, flags

``mlp.py`` holds the FP64 deep-sets network, its backward pass and Adam.
The sky map (``skymap``) and the transient search on it (``li_ma``,
``disk_sum``, ``transient_maps``, ``transient_search``) are numpy here.
``lut.py`` holds the lookup-table ("calibration matrix") energy and scaled
width/length reconstruction; ``ingest.py`` the DL0 byte-stream decoder.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

H_FIELDS = ["size", "x", "y", "length", "width", "psi", "r", "phi", "time_grad", "time_mean", "n_pix", "flags"]
S_FIELDS = ["dir_x", "dir_y", "core_x", "core_y", "n_valid", "flags"]
H = {k: i for i, k in enumerate(H_FIELDS)}
S = {k: i for i, k in enumerate(S_FIELDS)}
FLAG_EMPTY = 1
FLAG_NO_TIME = 2
FLAG_STEREO_INVALID = 1


def build(force: bool = False) -> str:
    """Compile liboracle.so in-tree. -ffp-contract=off keeps the FP32 multiply un-fused."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, f32 = ctypes.c_int, ctypes.c_int64, ctypes.c_float
        lib.or_integrate.argtypes = [P, i32, i32, P, P, i32, i32, i32, P, P, P, P, P]
        lib.or_integrate_nbpeak.argtypes = [P, i32, i32, P, P, P, i32, i32, P, P, P]
        lib.or_clean.argtypes = [i32, P, P, i32, f32, f32, i32, P]
        lib.or_hillas.argtypes = [i32, P, P, P, P, P]
        lib.or_stereo.argtypes = [i32, P, P, P]
        lib.or_reconstruct.argtypes = [i64, P, P, P, P, P, P, P, P, P, P, i32, i32, i32, f32, f32, i32, P, P, P, P,
                                       P, i64, P, P, P, i32, P, i32]
        _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "array must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def integrate(wave, p16, scale, sliding: bool, start: int, W: int, weights=None):
    """wave (P, S) uint16 -> (q float32, t float64, window start int32, window sum int64).

    weights (W integers, optional): the digital-filter-style charge
    16 * sum_k c_k s[st + k] - (sum_k c_k) * p16, rounded to FP32 and multiplied by
    the scale, over the same window (st and the flat sum are unchanged)."""
    wave = np.ascontiguousarray(wave, np.uint16)
    P, Sn = wave.shape
    p16 = np.ascontiguousarray(p16, np.int32)
    scale = np.ascontiguousarray(scale, np.float32)
    q = np.zeros(P, np.float32)
    t = np.zeros(P, np.float64)
    ws = np.zeros(P, np.int32)
    wsum = np.zeros(P, np.int64)
    wts = None if weights is None else np.ascontiguousarray(weights, np.int32)
    if wts is not None and len(wts) != W:
        raise ValueError("weights must have W entries")
    if _L().or_integrate(_p(wave), P, Sn, _p(p16), _p(scale), int(sliding), int(start), int(W), _p(wts), _p(q),
                         _p(t), _p(ws), _p(wsum)) != 0:
        raise ValueError("or_integrate: bad arguments")
    return q, t, ws, wsum


def integrate_nbpeak(wave, p16, scale, nb, W: int):
    """Neighbour-peak window: wave (P, S) uint16, nb (P, K) int16 neighbour ids
    (-1 = none) -> (q float32, t float64, chosen window start int32)."""
    wave = np.ascontiguousarray(wave, np.uint16)
    P, Sn = wave.shape
    nb = np.ascontiguousarray(nb, np.int16).reshape(P, -1)
    q = np.zeros(P, np.float32)
    t = np.zeros(P, np.float64)
    ws = np.zeros(P, np.int32)
    if _L().or_integrate_nbpeak(_p(wave), P, Sn, _p(np.ascontiguousarray(p16, np.int32)),
                                _p(np.ascontiguousarray(scale, np.float32)), _p(nb), nb.shape[1], int(W), _p(q),
                                _p(t), _p(ws)) != 0:
        raise ValueError("or_integrate_nbpeak: bad arguments")
    return q, t, ws


def clean(q, nb, t_hi: float, t_lo: float, core_needs_neighbour: bool):
    q = np.ascontiguousarray(q, np.float32)
    nb = np.ascontiguousarray(nb, np.int16)
    mask = np.zeros(len(q), np.uint8)
    _L().or_clean(len(q), _p(q), _p(nb), nb.shape[1], float(t_hi), float(t_lo), int(core_needs_neighbour), _p(mask))
    return mask


def hillas(xy, q, t, mask):
    xy = np.ascontiguousarray(xy, np.float32)
    q = np.ascontiguousarray(q, np.float32)
    t = None if t is None else np.ascontiguousarray(t, np.float64)
    mask = np.ascontiguousarray(mask, np.uint8)
    out = np.zeros(len(H_FIELDS), np.float64)
    _L().or_hillas(len(q), _p(xy), _p(q), _p(t), _p(mask), _p(out))
    return out


def stereo(hrows, txy):
    hrows = np.ascontiguousarray(hrows, np.float64).reshape(-1, len(H_FIELDS))
    txy = np.ascontiguousarray(txy, np.float64).reshape(-1, 2)
    out = np.zeros(len(S_FIELDS), np.float64)
    _L().or_stereo(len(hrows), _p(hrows), _p(txy), _p(out))
    return out


SKY_N = 256
SKY_WINDOW_S = 30


def sky_bin(v):
    """Sky-map bin of a nominal-frame coordinate (deg): floor((v + 2.56) * 50) with
    both operations in FP32, round to nearest (the quantisation is decided in the
    precision of the device, as the reading of the binning states); -1 outside
    [0, 256) or for NaN."""
    v = np.asarray(v, np.float32)
    with np.errstate(invalid="ignore"):
        u = (v + np.float32(2.56)).astype(np.float32) * np.float32(50.0)
        u = u.astype(np.float32)
        ok = (u >= 0) & (u < SKY_N)
    return np.where(ok, np.floor(np.where(ok, u, 0)), -1).astype(np.int64)


def skymap(dir_x, dir_y, has_dir, arrival_s, now_s):
    """Counts of events with a direction whose arrival second lies in
    (now_s - 30, now_s], per bin [iy, ix]."""
    ix, iy = sky_bin(dir_x), sky_bin(dir_y)
    sec = np.asarray(arrival_s, np.int64)
    sel = np.asarray(has_dir, bool) & (ix >= 0) & (iy >= 0) & (sec > now_s - SKY_WINDOW_S) & (sec <= now_s)
    m = np.zeros((SKY_N, SKY_N), np.int64)
    np.add.at(m, (iy[sel], ix[sel]), 1)
    return m


def reconstruct(wl, threads: int | None = None, do_stereo: bool = True, per_pixel: bool = False, wave=None):
    """Whole chain over a synth.Workload.

    Returns dict(hillas=(n_img,12), stereo=(n_evt,6) or None, q/t/mask per pixel if asked)."""
    lib = _L()
    wave = wl.wave if wave is None else wave
    cam_info = np.zeros((16, 3), np.int32)
    cam_xy = (ctypes.c_void_p * 16)()
    cam_nb = (ctypes.c_void_p * 16)()
    keep = []
    for c, cam in wl.cams.items():
        cam_info[c] = (cam.n_pix, cam.n_samples, cam.K)
        xy = np.ascontiguousarray(cam.xy, np.float32)
        nb = np.ascontiguousarray(cam.nb, np.int16)
        keep += [xy, nb]
        cam_xy[c] = _p(xy).value
        cam_nb[c] = _p(nb).value
    n_img, n_evt = wl.n_img, wl.n_evt
    hil = np.zeros((n_img, len(H_FIELDS)), np.float64)
    ste = np.zeros((n_evt, len(S_FIELDS)), np.float64) if do_stereo else None
    npx = int(wl.pix_off[-1])
    q = np.zeros(npx, np.float32) if per_pixel else None
    t = np.zeros(npx, np.float64) if per_pixel else None
    mk = np.zeros(npx, np.uint8) if per_pixel else None
    pr = wl.proc
    threads = threads or os.cpu_count() or 1
    tel_xy = np.ascontiguousarray(wl.tel_xy, np.float32)
    wts = None if getattr(pr, "weights", None) is None else np.ascontiguousarray(pr.weights, np.int32)
    st = lib.or_reconstruct(n_img, _p(wave), _p(wl.wave_off), _p(wl.img_tel), _p(wl.tel_cam), _p(wl.tel_pix_off),
                            _p(wl.p16), _p(wl.scale), _p(cam_info), ctypes.cast(cam_xy, ctypes.c_void_p),
                            ctypes.cast(cam_nb, ctypes.c_void_p), int(pr.sliding), int(pr.start), int(pr.W),
                            float(pr.t_hi), float(pr.t_lo), int(pr.core_needs_neighbour), _p(hil),
                            _p(wl.pix_off) if per_pixel else None, _p(q), _p(t), _p(mk), n_evt if do_stereo else 0,
                            _p(wl.evt_off), _p(tel_xy), _p(ste), int(threads), _p(wts),
                            int(bool(getattr(pr, "nbpeak", False))))
    if st != 0:
        raise RuntimeError("or_reconstruct failed")
    return dict(hillas=hil, stereo=ste, q=q, t=t, mask=mk)


SKY_MIN_SLABS = 60


def li_ma(n_on, n_off, alpha):
    """Significance of an on/off count pair (Li & Ma 1983, ApJ 272, 317, Eq. 17),
    signed: negative when n_on < alpha * n_off. Terms with a zero count are 0
    (the limit of n ln n). FP64."""
    n_on = np.asarray(n_on, np.float64)
    n_off = np.asarray(n_off, np.float64)
    alpha = np.asarray(alpha, np.float64)
    tot = n_on + n_off
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = np.where(n_on > 0, n_on * np.log((1.0 + alpha) / alpha * (n_on / tot)), 0.0)
        t2 = np.where(n_off > 0, n_off * np.log((1.0 + alpha) * (n_off / tot)), 0.0)
    s = np.sqrt(np.maximum(2.0 * (t1 + t2), 0.0))
    s = np.where(tot > 0, s, 0.0)
    return np.where(n_on >= alpha * n_off, s, -s)


def disk_sum(m, radius):
    """Sum of m over the disk of bins (dx^2 + dy^2 <= radius^2) around every bin,
    bins outside the map counting 0."""
    m = np.asarray(m, np.int64)
    n = m.shape[0]
    out = np.zeros_like(m)
    for dy in range(-radius, radius + 1):
        for dx in range(-radius, radius + 1):
            if dx * dx + dy * dy > radius * radius:
                continue
            ys = slice(max(0, -dy), min(n, n - dy))
            yd = slice(max(0, dy), min(n, n + dy))
            xs = slice(max(0, -dx), min(n, n - dx))
            xd = slice(max(0, dx), min(n, n + dx))
            out[ys, xs] += m[yd, xd]
    return out


def _window_ok(on_s, off_s):
    if on_s < 1 or off_s < 1:
        return False
    if on_s + off_s <= SKY_WINDOW_S:
        return True
    return on_s % 60 == 0 and off_s % 60 == 0 and on_s + off_s <= 60 * SKY_MIN_SLABS


def transient_maps(dir_x, dir_y, has_dir, arrival_s, now_s, window, radius):
    """(significance, disk on counts, disk off counts, alpha) maps [iy, ix] of one
    window (on_s, off_s): on = arrival seconds in (now - on, now], off = the
    off_s seconds before that; seconds, or whole minutes (floor(s / 60)) when the
    window is longer than the one-second ring."""
    on_s, off_s = int(window[0]), int(window[1])
    if not _window_ok(on_s, off_s):
        raise ValueError("window outside the ring rules")
    ix, iy = sky_bin(dir_x), sky_bin(dir_y)
    sec = np.asarray(arrival_s, np.int64)
    ok = np.asarray(has_dir, bool) & (ix >= 0) & (iy >= 0)
    if on_s + off_s <= SKY_WINDOW_S:
        t, now, on, off = sec, int(now_s), on_s, off_s
    else:
        t, now, on, off = np.floor_divide(sec, 60), int(now_s) // 60, on_s // 60, off_s // 60
    sel_on = ok & (t > now - on) & (t <= now)
    sel_off = ok & (t > now - on - off) & (t <= now - on)
    m_on = np.zeros((SKY_N, SKY_N), np.int64)
    m_off = np.zeros((SKY_N, SKY_N), np.int64)
    np.add.at(m_on, (iy[sel_on], ix[sel_on]), 1)
    np.add.at(m_off, (iy[sel_off], ix[sel_off]), 1)
    d_on, d_off = disk_sum(m_on, radius), disk_sum(m_off, radius)
    alpha = on_s / off_s
    return li_ma(d_on, d_off, alpha), d_on, d_off, alpha


def transient_search(dir_x, dir_y, has_dir, arrival_s, now_s, windows, radius, s_min):
    """Alerts (window, ix, iy, n_on, n_off, alpha, significance) with significance
    >= s_min, sorted by (window, iy, ix)."""
    rows = []
    for w, win in enumerate(windows):
        sig, d_on, d_off, alpha = transient_maps(dir_x, dir_y, has_dir, arrival_s, now_s, win, radius)
        for y, x in zip(*np.nonzero(sig >= s_min)):
            rows.append((w, int(x), int(y), int(d_on[y, x]), int(d_off[y, x]), alpha, float(sig[y, x])))
    return rows


from .lut import bin_index, impact_distance, lut_build, lut_reconstruct  # noqa: E402
from . import ingest  # noqa: E402,F401
