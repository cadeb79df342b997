"""The neighbour-peak window (RTA_WINDOW_NEIGHBOUR) through the C ABI against
the oracle: charges and window choices bit for bit, cleaning (n_pix, flags)
exact and Hillas rows within the usual tolerances, for the generic search
(16-sample square camera), the 40-sample hexagonal camera and the three-camera
array; every tile shape and pipeline depth gives identical rows; and the full
10,000-event bundle in the benchmark's launch configuration."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
import paper_1307_6489_gb300 as rta

from gpu_helpers import (DIR_DEG, T_ABS, Dev, compare_hillas, hillas_rows, make_ctx, proc_args, stereo_rows)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WORKLOADS = {"square256": (0, 600, 5), "hex1855": (1, 200, 6), "array": (2, 200, 6)}


def nb_workload(preset, n, W):
    wl = synth.make_workload(preset, n)
    wl.proc = dataclasses.replace(wl.proc, sliding=True, W=W, nbpeak=True)
    return wl


@pytest.fixture(scope="module", params=list(WORKLOADS))
def nset(request):
    preset, n, W = WORKLOADS[request.param]
    wl = nb_workload(preset, n, W)
    ref = oracle.reconstruct(wl, per_pixel=True, do_stereo=preset == 2)
    ctx = make_ctx(wl)
    dev = Dev(wl)
    yield request.param, wl, ref, ctx, dev
    ctx.close()


def test_nbpeak_charges_and_times_match_the_oracle(nset):
    name, wl, ref, ctx, dev = nset
    mode, start, W, *_ = proc_args(wl)
    assert mode == rta.RTA_WINDOW_NEIGHBOUR
    q = torch.full((dev.n_pix,), np.nan, dtype=torch.float32, device="cuda")
    t = torch.full((dev.n_pix,), np.nan, dtype=torch.float32, device="cuda")
    ctx.calibrate_integrate(dev.wave, dev.wave_off, dev.img_tel, dev.pix_off, mode, start, W, q, t)
    assert ctx.check() == 0
    qg, tg = q.cpu().numpy(), t.cpu().numpy()
    np.testing.assert_array_equal(qg.view(np.uint32), ref["q"].view(np.uint32))
    assert np.max(np.abs(tg - ref["t"])) <= T_ABS
    # the neighbour-peak window differs from the sliding one somewhere (else the test is idle)
    flat = dataclasses.replace(wl.proc, nbpeak=False)
    q_sl = oracle.reconstruct(dataclasses.replace(wl, proc=flat), per_pixel=True, do_stereo=False)["q"]
    assert (q_sl != ref["q"]).mean() > 0.05


def test_nbpeak_chain_matches_the_oracle(nset):
    name, wl, ref, ctx, dev = nset
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    out = dev.hillas_buf()
    if ref["stereo"] is not None:
        s = dev.stereo_buf()
        ctx.reconstruct(dev.wave, dev.wave_off, dev.img_tel, dev.evt_off, mode, start, W, t_hi, t_lo, core_nb, out, s)
    else:
        ctx.image_chain(dev.wave, dev.wave_off, dev.img_tel, mode, start, W, t_hi, t_lo, core_nb, out)
    assert ctx.check() == 0
    g = hillas_rows(out, wl.n_img)
    compare_hillas(g, ref["hillas"], name)
    assert (g["n_pix"] > 0).mean() > 0.3
    if ref["stereo"] is not None:
        st = stereo_rows(s, wl.n_evt)
        S = oracle.S
        np.testing.assert_array_equal(st["flags"], ref["stereo"][:, S["flags"]].astype(np.uint32))
        ok = ref["stereo"][:, S["flags"]] == 0
        d = np.hypot(st["dir_x"][ok] - ref["stereo"][ok, S["dir_x"]], st["dir_y"][ok] - ref["stereo"][ok, S["dir_y"]])
        assert np.percentile(d, 99) <= DIR_DEG


def test_nbpeak_chain_masks_bit_exact(nset):
    """The neighbour-peak kernel's cleaning masks against the oracle's, pixel by
    pixel; its Hillas rows equal rta_image_chain's bit for bit."""
    name, wl, ref, ctx, dev = nset
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    base = dev.hillas_buf()
    ctx.image_chain(dev.wave, dev.wave_off, dev.img_tel, mode, start, W, t_hi, t_lo, core_nb, base)
    mask = torch.full((dev.n_pix,), 7, dtype=torch.uint8, device="cuda")
    out = torch.full_like(base, float("nan"))
    ctx.image_chain_masks(dev.wave, dev.wave_off, dev.img_tel, dev.pix_off, mode, start, W, t_hi, t_lo, core_nb, mask,
                          out)
    assert ctx.check() == 0
    np.testing.assert_array_equal(mask.cpu().numpy(), ref["mask"])
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), base.cpu().numpy().view(np.uint32))


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("n_stages,ctas", [(2, 1), (3, 0), (6, 1)])
def test_nbpeak_every_tile_and_pipeline_depth_is_identical(nset, variant, n_stages, ctas):
    name, wl, ref, ctx, dev = nset
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    default = ctx.chain_config()
    base = dev.hillas_buf()
    ctx.image_chain(dev.wave, dev.wave_off, dev.img_tel, mode, start, W, t_hi, t_lo, core_nb, base)
    out = dev.hillas_buf()
    try:
        try:
            ctx.set_chain_config(variant, n_stages, ctas)
            ctx.image_chain(dev.wave, dev.wave_off, dev.img_tel, mode, start, W, t_hi, t_lo, core_nb, out)
        except rta.RtaError as e:
            pytest.skip(f"configuration does not fit: {e}")
        assert ctx.check() == 0
    finally:
        ctx.set_chain_config(default["variant"], default["n_stages"], 0)
    assert torch.equal(out, base)


def test_nbpeak_full_size_bundle():
    """10,000 events (46,292 images): every image's n_pix and flags exact, Hillas
    rows of 300 sampled events within tolerance; many images per CTA, so the
    sweep barriers cycle through many phases."""
    wl = nb_workload(2, 10000, 6)
    ref = oracle.reconstruct(wl, do_stereo=False)
    ctx = make_ctx(wl)
    dev = Dev(wl)
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    out = dev.hillas_buf()
    ctx.image_chain(dev.wave, dev.wave_off, dev.img_tel, mode, start, W, t_hi, t_lo, core_nb, out)
    assert ctx.check() == 0
    g = hillas_rows(out, wl.n_img)
    H = oracle.H
    np.testing.assert_array_equal(g["n_pix"], ref["hillas"][:, H["n_pix"]].astype(np.int32))
    np.testing.assert_array_equal(g["flags"], ref["hillas"][:, H["flags"]].astype(np.uint32))
    rng = np.random.default_rng(7)
    ev = rng.choice(wl.n_evt, 300, replace=False)
    imgs = np.concatenate([np.arange(wl.evt_off[e], wl.evt_off[e + 1]) for e in ev])
    compare_hillas({k: v[imgs] for k, v in g.items()}, ref["hillas"][imgs], "nbpeak full bundle")
    ctx.close()


def test_calibration_scales_must_be_finite_and_positive():
    """The neighbour-peak shortcut (a pixel's charge in any window is at most
    its sliding-window charge) needs positive scales; registration refuses
    others."""
    wl = synth.make_workload(0, 4)
    ctx = rta.Context(0)
    for c, cam in wl.cams.items():
        ctx.register_camera(c, cam.xy, cam.nb, cam.n_samples)
    for bad in (0.0, -1.0, np.nan, np.inf):
        scale = wl.scale.copy()
        scale[3] = bad
        with pytest.raises(rta.RtaError) as e:
            ctx.register_array(wl.tel_cam, wl.tel_xy, wl.p16, scale)
        assert e.value.code == rta.RTA_E_INVALID
    ctx.register_array(wl.tel_cam, wl.tel_xy, wl.p16, wl.scale)
    ctx.close()


def test_a_cta_count_tuned_for_the_plain_kernel_does_not_block_the_neighbour_peak_window(nset):
    """The autotuner may pin 3 CTAs per SM for the plain kernel; the
    neighbour-peak kernel (more shared memory) runs with as many as fit."""
    name, wl, ref, ctx, dev = nset
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    default = ctx.chain_config()
    base = dev.hillas_buf()
    ctx.image_chain(dev.wave, dev.wave_off, dev.img_tel, mode, start, W, t_hi, t_lo, core_nb, base)
    out = dev.hillas_buf()
    try:
        ctx.set_chain_config(4, 2, 3)
        ctx.image_chain(dev.wave, dev.wave_off, dev.img_tel, mode, start, W, t_hi, t_lo, core_nb, out)
        assert ctx.check() == 0
    finally:
        ctx.set_chain_config(default["variant"], default["n_stages"], 0)
    assert torch.equal(out, base)
