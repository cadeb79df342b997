"""The digital-filter-style extractor (RTA_WINDOW_FILTER) through the C ABI
against the oracle: charges and cleaning masks bit for bit, Hillas rows and
stereo within the usual tolerances; unit weights equal the flat window."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
import paper_1307_6489_gb300 as rta

from gpu_helpers import (DIR_DEG, T_ABS, Dev, compare_hillas, hillas_rows, make_ctx, proc_args, stereo_rows)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WEIGHTS = (1, 4, 9, 8, 4, 2)      # a pulse-shaped filter over the 6-sample window


def filter_workload(weights=WEIGHTS, n=150):
    wl = synth.make_workload(2, n)
    wl.proc = dataclasses.replace(wl.proc, weights=tuple(weights))
    # normalise the filter in the calibration scale (flat response W, filter response sum(c))
    wl.scale = (wl.scale * np.float32(len(weights) / sum(weights))).astype(np.float32)
    return wl


@pytest.fixture(scope="module")
def fset():
    wl = filter_workload()
    ref = oracle.reconstruct(wl, per_pixel=True)
    ctx = make_ctx(wl)
    dev = Dev(wl)
    yield wl, ref, ctx, dev
    ctx.close()


def test_filter_charges_and_times_match_the_oracle(fset):
    wl, ref, ctx, dev = fset
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    assert mode == rta.RTA_WINDOW_FILTER
    q = torch.zeros(dev.n_pix, dtype=torch.float32, device="cuda")
    t = torch.zeros(dev.n_pix, dtype=torch.float32, device="cuda")
    ctx.calibrate_integrate(dev.wave, dev.wave_off, dev.img_tel, dev.pix_off, mode, start, W, q, t)
    assert ctx.check() == 0
    np.testing.assert_array_equal(q.cpu().numpy().view(np.uint32), ref["q"].view(np.uint32))
    assert np.max(np.abs(t.cpu().numpy() - ref["t"])) <= T_ABS


def test_filter_chain_and_stereo_match_the_oracle(fset):
    wl, ref, ctx, dev = fset
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    h, s = dev.hillas_buf(), dev.stereo_buf()
    ctx.reconstruct(dev.wave, dev.wave_off, dev.img_tel, dev.evt_off, mode, start, W, t_hi, t_lo, core_nb, h, s)
    assert ctx.check() == 0
    g = hillas_rows(h, wl.n_img)
    compare_hillas(g, ref["hillas"], "filter")
    assert (g["n_pix"] > 0).mean() > 0.3
    st = stereo_rows(s, wl.n_evt)
    S = oracle.S
    np.testing.assert_array_equal(st["flags"], ref["stereo"][:, S["flags"]].astype(np.uint32))
    ok = ref["stereo"][:, S["flags"]] == 0
    ddir = np.hypot(st["dir_x"][ok] - ref["stereo"][ok, S["dir_x"]], st["dir_y"][ok] - ref["stereo"][ok, S["dir_y"]])
    assert np.percentile(ddir, 99) <= DIR_DEG


def test_filter_chain_masks_bit_exact(fset):
    wl, ref, ctx, dev = fset
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


def test_unit_weights_equal_the_flat_window():
    wl = synth.make_workload(2, 40)
    ctx = make_ctx(wl)
    dev = Dev(wl)
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    flat = dev.hillas_buf()
    ctx.image_chain(dev.wave, dev.wave_off, dev.img_tel, mode, start, W, t_hi, t_lo, core_nb, flat)
    rta.rta_set_filter_weights(ctx.handle, [1] * W)
    filt = dev.hillas_buf()
    ctx.image_chain(dev.wave, dev.wave_off, dev.img_tel, rta.RTA_WINDOW_FILTER, start, W, t_hi, t_lo, core_nb, filt)
    assert ctx.check() == 0
    assert torch.equal(flat, filt)
    ctx.close()


def test_filter_arguments_are_checked(fset):
    wl, ref, ctx, dev = fset
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    out = dev.hillas_buf()
    with pytest.raises(rta.RtaError) as e:
        ctx.image_chain(dev.wave, dev.wave_off, dev.img_tel, mode, start, W - 1, t_hi, t_lo, core_nb, out)
    assert e.value.code == rta.RTA_E_INVALID                   # W differs from the weights' length
    for bad in [[0, 0, 0, 0, 0, 0], [5000, 1, 1, 1, 1, 1], [1] * 17]:
        with pytest.raises(rta.RtaError):
            rta.rta_set_filter_weights(ctx.handle, bad)
