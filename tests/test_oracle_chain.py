"""Whole-chain consistency of generator + oracle against the generated truth.

These are physics checks, not parity: a bright noiseless-ish ellipse must come
back near its generated centroid and axis, and noiseless stereo geometry of the
array preset must put the reconstructed direction near the true source.
"""
import numpy as np
import pytest

import oracle
import synth

Hf = oracle.H
Sf = oracle.S


def test_single_camera_images_recover_generated_ellipse():
    wl = synth.make_workload(0, 300)
    r = oracle.reconstruct(wl, do_stereo=False)
    h = r["hillas"]
    size_true = wl.ell[:, 0, 0]
    cx, cy, psi = wl.ell[:, 0, 1], wl.ell[:, 0, 2], wl.ell[:, 0, 5]
    inside = np.hypot(cx, cy) < 0.45
    bright = (size_true > 1500) & inside
    assert bright.sum() > 20
    assert np.median(np.abs(h[bright, Hf["x"]] - cx[bright])) < 0.02
    assert np.median(np.abs(h[bright, Hf["y"]] - cy[bright])) < 0.02
    d = (h[bright, Hf["psi"]] - psi[bright]) % np.pi
    d = np.minimum(d, np.pi - d)
    assert np.median(d) < 0.1
    ratio = h[bright, Hf["size"]] / size_true[bright]
    assert 0.8 < np.median(ratio) < 1.1


def test_noiseless_array_geometry_recovers_source():
    # electronic noise and NSB off: residual errors come from pixelisation and photon statistics
    wl = synth.make_workload(2, 150, flags=3)
    r = oracle.reconstruct(wl)
    s = r["stereo"]
    ok = s[:, Sf["flags"]] == 0
    assert ok.mean() > 0.5
    err = np.hypot(s[ok, Sf["dir_x"]] - wl.truth[ok, 1], s[ok, Sf["dir_y"]] - wl.truth[ok, 2])
    assert np.percentile(err, 68) < 0.4


def test_noisy_array_resolution_is_physical():
    wl = synth.make_workload(2, 300)
    r = oracle.reconstruct(wl)
    s = r["stereo"]
    ok = (s[:, Sf["flags"]] == 0) & (s[:, Sf["n_valid"]] >= 3)
    err = np.hypot(s[ok, Sf["dir_x"]] - wl.truth[ok, 1], s[ok, Sf["dir_y"]] - wl.truth[ok, 2])
    assert ok.sum() > 30
    assert np.percentile(err, 68) < 0.5
    core_err = np.hypot(s[ok, Sf["core_x"]] - wl.truth[ok, 3], s[ok, Sf["core_y"]] - wl.truth[ok, 4])
    assert np.percentile(core_err, 68) < 150


def test_threads_do_not_change_results():
    wl = synth.make_workload(2, 40)
    a = oracle.reconstruct(wl, threads=1, per_pixel=True)
    b = oracle.reconstruct(wl, threads=6, per_pixel=True)
    for k in ["hillas", "stereo", "q", "mask"]:
        np.testing.assert_array_equal(a[k], b[k])
