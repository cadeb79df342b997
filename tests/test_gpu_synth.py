"""The GPU renderer of the input generator (bulk training and evaluation sets)
against the host renderer, statistically: the same planned showers rendered both
ways give waveforms and reconstructed images with the same distributions (the
two compute in FP32 and FP64 and are not equal bit for bit)."""
import numpy as np
import pytest

import synth
import paper_1307_6489_gb300 as rta

from gpu_helpers import Dev, hillas_rows, make_ctx, proc_args

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def both():
    wl = synth.make_workload(3, 400)
    d = torch.empty(wl.n_samples_total, dtype=torch.int16, device="cuda")
    keep = synth.render_waves_gpu(wl, d)
    torch.cuda.synchronize()
    g = d.cpu().numpy().view(np.uint16)
    del keep
    return wl, wl.wave.copy(), g


def test_sample_distributions_agree(both):
    wl, c, g = both
    assert g.shape == c.shape
    ped = np.concatenate([np.repeat(wl.ped[wl.tel_pix_off[t]:wl.tel_pix_off[t + 1]], wl.cams[int(wl.tel_cam[t])].n_samples)
                          for t in wl.img_tel])
    dc, dg = c.astype(np.float64) - ped, g.astype(np.float64) - ped
    # pedestal-dominated quantiles within a tenth of an ADC count, the signal tail within a few percent
    for qq in (1, 10, 50, 90, 99):
        assert abs(np.percentile(dc, qq) - np.percentile(dg, qq)) <= 0.6, qq
    assert abs(dc.std() - dg.std()) / dc.std() < 0.03
    hi_c, hi_g = np.sum(dc[dc > 50]), np.sum(dg[dg > 50])
    assert abs(hi_g / hi_c - 1) < 0.05


def test_reconstructed_images_agree(both):
    wl, c, g = both
    ctx = make_ctx(wl)
    dev = Dev(wl)
    proc = proc_args(wl)
    out = {}
    for name, w in (("host", c), ("gpu", g)):
        dev.wave = torch.from_numpy(w.view(np.int16)).cuda()
        h = dev.hillas_buf()
        ctx.image_chain(dev.wave, dev.wave_off, dev.img_tel, *proc, h)
        ctx.check()
        out[name] = hillas_rows(h, wl.n_img)
    a, b = out["host"], out["gpu"]
    used_a, used_b = a["n_pix"] >= 3, b["n_pix"] >= 3
    assert abs(used_a.mean() - used_b.mean()) < 0.02
    assert abs(b["size"].sum() / a["size"].sum() - 1) < 0.03
    assert abs(b["n_pix"].mean() / a["n_pix"].mean() - 1) < 0.03
    both_used = used_a & used_b
    # same showers: the axes agree image by image where both are elongated
    el = both_used & (a["length"] > 1.5 * a["width"]) & (a["n_pix"] >= 10)
    d = np.abs(a["psi"][el] - b["psi"][el]) % np.pi
    d = np.minimum(d, np.pi - d)
    assert el.sum() > 50 and np.median(d) < 0.05
    ctx.close()
