"""Edge cases of the CUDA path through the C ABI: empty and malformed inputs,
degenerate images, saturated samples, the generic (non-specialised) integration
paths at the maximum camera size, argument checks, and the full-size bundle on
sampled outputs."""
import time

import numpy as np
import pytest

import oracle
import synth
import paper_1307_6489_gb300 as rta

from gpu_helpers import (DIR_DEG, T_ABS, Dev, compare_hillas, core_ok, hillas_rows, hillas_rows_as_f32, make_ctx,
                         proc_args, stereo_rows, f32_rows_as_oracle)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def arr():
    wl = synth.make_workload(2, 40)
    ctx = make_ctx(wl)
    yield wl, ctx
    ctx.close()


def test_empty_bundle_is_a_no_op(arr):
    wl, ctx = arr
    dev = Dev(wl)
    out = torch.zeros(16, dtype=torch.float32, device="cuda")
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    rta.rta_image_chain(ctx.handle, dev.wave.data_ptr(), dev.wave.numel(), dev.wave_off.data_ptr(),
                        dev.img_tel.data_ptr(), 0, mode, start, W, t_hi, t_lo, core_nb, out.data_ptr(), 0)
    rta.rta_stereo(ctx.handle, 0, 0, 0, dev.evt_off.data_ptr(), 0, out.data_ptr(), 0)
    assert ctx.check() == 0
    assert float(out.abs().sum()) == 0.0


def test_malformed_images_are_flagged_not_read(arr):
    wl, ctx = arr
    dev = Dev(wl)
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    good = dev.hillas_buf()
    ctx.image_chain(dev.wave, dev.wave_off, dev.img_tel, mode, start, W, t_hi, t_lo, core_nb, good)
    ctx.check()
    off = dev.wave_off.clone()
    tel = dev.img_tel.clone()
    off[3] += 1                         # not a multiple of 8 samples
    tel[5] = 999                        # no such telescope
    off[7] = dev.wave.numel()           # past the end of the buffer
    off[9] = -8                         # negative
    out = dev.hillas_buf()
    ctx.image_chain(dev.wave, off, tel, mode, start, W, t_hi, t_lo, core_nb, out)
    with pytest.raises(rta.RtaError) as e:
        ctx.check()
    assert e.value.code == rta.RTA_E_DEVICE and e.value.bits & rta.RTA_DEV_BAD_IMAGE
    g = hillas_rows(out, wl.n_img)
    bad = [3, 5, 7, 9]
    for i in bad:
        assert g["flags"][i] & rta.RTA_HF_BAD_INPUT and g["n_pix"][i] == 0
    keep = np.setdiff1d(np.arange(wl.n_img), bad)
    a = out.cpu().numpy().reshape(-1, 16)[keep]
    b = good.cpu().numpy().reshape(-1, 16)[keep]
    np.testing.assert_array_equal(a.view(np.uint32), b.view(np.uint32))
    assert ctx.check() == 0             # the status word was cleared


def test_malformed_event_lists_are_flagged(arr):
    wl, ctx = arr
    dev = Dev(wl)
    h = dev.hillas_buf()
    evt = dev.evt_off.clone()
    evt[2] = wl.n_img + 5               # event 1 ends past n_img, event 2 starts there
    out = dev.stereo_buf()
    ctx.stereo(h, evt, dev.img_tel, out)
    with pytest.raises(rta.RtaError):
        ctx.check()
    s = stereo_rows(out, wl.n_evt)
    assert s["flags"][1] & rta.RTA_SF_INVALID and s["flags"][2] & rta.RTA_SF_INVALID


@pytest.mark.parametrize("level", ["pedestal", "saturated", "zero"])
def test_flat_waveforms(arr, level):
    wl0, ctx = arr
    wl = synth.subset(wl0, np.arange(10))
    wl.wave[:] = {"pedestal": 400, "saturated": 65535, "zero": 0}[level]
    ref = oracle.reconstruct(wl, per_pixel=True)
    dev = Dev(wl)
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    q = torch.zeros(dev.n_pix, dtype=torch.float32, device="cuda")
    t = torch.zeros(dev.n_pix, dtype=torch.float32, device="cuda")
    ctx.calibrate_integrate(dev.wave, dev.wave_off, dev.img_tel, dev.pix_off, mode, start, W, q, t)
    ctx.check()
    np.testing.assert_array_equal(q.cpu().numpy().view(np.uint32), ref["q"].view(np.uint32))
    assert np.max(np.abs(t.cpu().numpy() - ref["t"])) <= T_ABS
    h, s = dev.hillas_buf(), dev.stereo_buf()
    ctx.reconstruct(dev.wave, dev.wave_off, dev.img_tel, dev.evt_off, mode, start, W, t_hi, t_lo, core_nb, h, s)
    ctx.check()
    compare_hillas(hillas_rows(h, wl.n_img), ref["hillas"], level)
    st = stereo_rows(s, wl.n_evt)
    np.testing.assert_array_equal(st["flags"], ref["stereo"][:, oracle.S["flags"]].astype(np.uint32))


def random_waves(rng, n_img, P, S, xy):
    """Pedestal noise plus a bright Gaussian blob per image (arbitrary camera)."""
    ped = 400 + rng.normal(0, 3, P)
    w = ped[None, :, None] + rng.normal(0, 2, (n_img, P, S))
    for i in range(n_img):
        c = xy[rng.integers(P)]
        r2 = ((xy - c) ** 2).sum(1)
        amp = rng.uniform(50, 3000) * np.exp(-r2 / (2 * rng.uniform(0.01, 0.05)))
        t0 = rng.uniform(3, S - 4)
        k = np.arange(S)
        w[i] += amp[:, None] * np.exp(-((k[None, :] - t0) ** 2) / 4.5)
    return np.clip(np.floor(w + 0.5), 0, 65535).astype(np.uint16), ped


@pytest.mark.parametrize("kind,P,S,W,sliding", [("square", 4096, 128, 16, True), ("hex", 336, 27, 7, True),
                                                ("hex", 1000, 24, 3, False), ("grid", 64, 9, 9, True),
                                                ("square", 2048, 25, 6, True), ("hex", 1764, 30, 6, False)])
def test_generic_paths_and_largest_camera(kind, P, S, W, sliding):
    rng = np.random.default_rng(P + S)
    pitch = 0.1
    xy, nb = synth.lattice(kind, P, pitch)
    n_img = 12
    wave, ped = random_waves(rng, n_img, P, S, xy.astype(np.float64))
    gain = 8 * (1 + rng.normal(0, 0.05, P))
    p16 = np.round(16 * ped).astype(np.int32)
    scale = (1 / (16 * gain * 0.9)).astype(np.float32)
    ctx = rta.Context(0)
    ctx.register_camera(5, xy, nb, S)
    ctx.register_array(np.array([5], np.int32), np.zeros((1, 2), np.float32), p16, scale)
    start = 0 if sliding else S - W
    flat = wave.reshape(-1)
    d_wave = torch.from_numpy(flat.view(np.int16)).cuda()
    wave_off = torch.arange(n_img, dtype=torch.int64, device="cuda") * (P * S)
    img_tel = torch.zeros(n_img, dtype=torch.int32, device="cuda")
    pix_off = torch.arange(n_img, dtype=torch.int64, device="cuda") * P
    q = torch.zeros(n_img * P, dtype=torch.float32, device="cuda")
    t = torch.zeros(n_img * P, dtype=torch.float32, device="cuda")
    mode = rta.RTA_WINDOW_SLIDING if sliding else rta.RTA_WINDOW_FIXED
    ctx.calibrate_integrate(d_wave, wave_off, img_tel, pix_off, mode, start, W, q, t)
    out = torch.zeros(n_img * 16, dtype=torch.float32, device="cuda")
    ctx.image_chain(d_wave, wave_off, img_tel, mode, start, W, 10.0, 5.0, 1, out)
    ctx.check()
    qg, tg = q.cpu().numpy(), t.cpu().numpy()
    ref_rows = []
    for i in range(n_img):
        qr, tr, _, _ = oracle.integrate(wave[i], p16, scale, sliding, start, W)
        np.testing.assert_array_equal(qg[i * P:(i + 1) * P].view(np.uint32), qr.view(np.uint32))
        assert np.max(np.abs(tg[i * P:(i + 1) * P] - tr)) <= T_ABS
        m = oracle.clean(qr, nb, 10.0, 5.0, 1)
        ref_rows.append(oracle.hillas(xy, qr, tr, m))
    compare_hillas(hillas_rows(out, n_img), np.array(ref_rows), f"{kind}{P}x{S}")
    ctx.close()


def test_argument_checks(arr):
    wl, ctx = arr
    dev = Dev(wl)
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    out = dev.hillas_buf()
    with pytest.raises(rta.RtaError) as e:
        ctx.image_chain(dev.wave, dev.wave_off, dev.img_tel, mode, start, 26, t_hi, t_lo, core_nb, out)
    assert e.value.code == rta.RTA_E_INVALID            # W = 26 > 25 samples of the small camera
    with pytest.raises(rta.RtaError) as e:
        ctx.image_chain(dev.wave, dev.wave_off, dev.img_tel, mode, start, W, 8.0, 0.0, core_nb, out)
    assert e.value.code == rta.RTA_E_INVALID
    with pytest.raises(rta.RtaError) as e:
        rta.rta_image_chain(ctx.handle, dev.wave.data_ptr() + 2, dev.wave.numel() - 1, dev.wave_off.data_ptr(),
                            dev.img_tel.data_ptr(), wl.n_img, mode, start, W, t_hi, t_lo, core_nb, out.data_ptr(), 0)
    assert e.value.code == rta.RTA_E_ALIGN
    xy, nb = synth.lattice("hex", 7, 0.1)
    with pytest.raises(rta.RtaError) as e:
        ctx.register_camera(9, xy, nb, 5)               # 7 * 5 samples: not a multiple of 8
    assert e.value.code == rta.RTA_E_ALIGN
    with pytest.raises(rta.RtaError) as e:
        rta.rta_register_array(ctx.handle, 1, np.array([11], np.int32), np.zeros(2, np.float32),
                               np.zeros(7, np.int32), np.zeros(7, np.float32))
    assert e.value.code == rta.RTA_E_INVALID            # camera 11 not registered
    assert ctx.check() == 0


def test_stereo_degenerate_events(arr):
    """Single-image events, events whose images are all too small, and one event of 70 images (first 64 used)."""
    wl, ctx = arr
    ref = oracle.reconstruct(wl)
    rows32 = hillas_rows_as_f32(ref["hillas"])
    n = wl.n_img
    # events: [0,1) single image, [1,3) pair, then a big event of up to 70 images, rest as pairs
    big = min(70, n - 3)
    bounds = [0, 1, 3, 3 + big] + list(range(3 + big + 2, n + 1, 2))
    if bounds[-1] != n:
        bounds.append(n)
    evt = np.array(bounds, np.int32)
    rows32[1:3].view(np.int32)[:, 10] = 2                # both images of event 1 below 3 pixels
    h = torch.from_numpy(rows32.reshape(-1)).cuda()
    out = torch.zeros((len(evt) - 1) * 8, dtype=torch.float32, device="cuda")
    ctx.stereo(h, torch.from_numpy(evt).cuda(), torch.from_numpy(wl.img_tel).cuda(), out)
    ctx.check()
    g = stereo_rows(out, len(evt) - 1)
    same = f32_rows_as_oracle(rows32)
    S = oracle.S
    for e in range(len(evt) - 1):
        a, b = evt[e], evt[e + 1]
        b = min(b, a + 64)
        exp = oracle.stereo(same[a:b], wl.tel_xy[wl.img_tel[a:b]].astype(np.float64))
        assert g["flags"][e] == exp[S["flags"]] and g["n_valid"][e] == exp[S["n_valid"]]
        if exp[S["flags"]] == 0:
            assert np.hypot(g["dir_x"][e] - exp[S["dir_x"]], g["dir_y"][e] - exp[S["dir_y"]]) <= DIR_DEG
    assert g["flags"][0] == rta.RTA_SF_INVALID and g["flags"][1] == rta.RTA_SF_INVALID


def test_full_size_bundle_every_event():
    """The benchmark's workload (10,000 events, 46,292 images, ~5 GB) in the
    benchmark's launch configuration, against the oracle on every image and event:
    n_pix and flags exact and every Hillas row within tolerance (the lean kernel
    rta_reconstruct runs), every cleaning mask pixel by pixel (the same kernel
    compiled with the mask output, whose rows are identical bit for bit), every
    stereo row's flags and image count exact, the end-to-end direction within the
    end-to-end bars, and the stereo stage fed the oracle's FP32 rows within 1e-3 deg
    on every event."""
    wl = synth.make_workload(2, 10000)
    ctx = make_ctx(wl)
    dev = Dev(wl)
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    h, s = dev.hillas_buf(), dev.stereo_buf()
    ctx.reconstruct(dev.wave, dev.wave_off, dev.img_tel, dev.evt_off, mode, start, W, t_hi, t_lo, core_nb, h, s)
    ctx.check()
    mask = torch.full((dev.n_pix,), 7, dtype=torch.uint8, device="cuda")
    hm = torch.full_like(h, float("nan"))
    ctx.image_chain_masks(dev.wave, dev.wave_off, dev.img_tel, dev.pix_off, mode, start, W, t_hi, t_lo, core_nb, mask,
                          hm)
    ctx.check()
    np.testing.assert_array_equal(hm.cpu().numpy().view(np.uint32)[: wl.n_img * 16],
                                  h.cpu().numpy().view(np.uint32)[: wl.n_img * 16])
    ref = oracle.reconstruct(wl, per_pixel=True)
    del dev
    np.testing.assert_array_equal(mask.cpu().numpy(), ref["mask"])
    compare_hillas(hillas_rows(h, wl.n_img), ref["hillas"], "full-size bundle")
    st = stereo_rows(s, wl.n_evt)
    S = oracle.S
    np.testing.assert_array_equal(st["flags"], ref["stereo"][:, S["flags"]].astype(np.uint32))
    np.testing.assert_array_equal(st["n_valid"], ref["stereo"][:, S["n_valid"]].astype(np.int32))
    ok = ref["stereo"][:, S["flags"]] == 0
    assert ok.sum() > 0.4 * wl.n_evt
    d = np.hypot(st["dir_x"][ok] - ref["stereo"][ok, S["dir_x"]], st["dir_y"][ok] - ref["stereo"][ok, S["dir_y"]])
    assert np.percentile(d, 99) <= DIR_DEG and np.median(d) <= 1e-4
    # stage-isolated on every event: both sides get the same FP32 rows
    rows32 = hillas_rows_as_f32(ref["hillas"])
    s2 = torch.zeros(wl.n_evt * 8, dtype=torch.float32, device="cuda")
    ctx.stereo(torch.from_numpy(rows32.reshape(-1)).cuda(), torch.from_numpy(wl.evt_off).cuda(),
               torch.from_numpy(wl.img_tel).cuda(), s2)
    ctx.check()
    g = stereo_rows(s2, wl.n_evt)
    same = f32_rows_as_oracle(rows32)
    exp = np.zeros((wl.n_evt, 6))
    for e in range(wl.n_evt):
        a, b = wl.evt_off[e], wl.evt_off[e + 1]
        exp[e] = oracle.stereo(same[a:b], wl.tel_xy[wl.img_tel[a:b]].astype(np.float64))
    np.testing.assert_array_equal(g["flags"], exp[:, S["flags"]].astype(np.uint32))
    np.testing.assert_array_equal(g["n_valid"], exp[:, S["n_valid"]].astype(np.int32))
    ok = exp[:, S["flags"]] == 0
    assert np.max(np.hypot(g["dir_x"][ok] - exp[ok, S["dir_x"]], g["dir_y"][ok] - exp[ok, S["dir_y"]])) <= DIR_DEG
    assert core_ok(g["core_x"][ok], g["core_y"][ok], exp[ok, S["core_x"]], exp[ok, S["core_y"]]).all()
    ctx.close()


def test_bounded_device_wait_times_out_and_the_context_survives(arr):
    """Failure detection without a GPU fault: a wait that nothing completes gives
    up after its limit, reports RTA_DEV_TIMEOUT, and the next launch works."""
    wl, ctx = arr
    t0 = time.perf_counter()
    waited = rta.rta_selftest_wait_timeout(ctx.handle, 200)
    dt = time.perf_counter() - t0
    assert 0.2e9 <= waited < 2.0e9 and dt < 5.0
    with pytest.raises(rta.RtaError) as e:
        ctx.check()
    assert e.value.code == rta.RTA_E_DEVICE and e.value.bits == rta.RTA_DEV_TIMEOUT
    dev = Dev(wl)
    out = dev.hillas_buf()
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    ctx.image_chain(dev.wave, dev.wave_off, dev.img_tel, mode, start, W, t_hi, t_lo, core_nb, out)
    assert ctx.check() == 0
    assert (hillas_rows(out, wl.n_img)["n_pix"] > 0).any()
