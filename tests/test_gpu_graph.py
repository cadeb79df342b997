"""The step captured as a CUDA graph at capacity, with device-resident counts."""
import numpy as np
import pytest

import synth
import paper_1307_6489_gb300 as rta

from gpu_helpers import Dev, make_ctx, proc_args

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_graph_at_capacity_matches_direct_launches_for_any_count():
    wl = synth.make_workload(2, 200)
    ctx = make_ctx(wl)
    dev = Dev(wl)
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    h_ref, s_ref = dev.hillas_buf(), dev.stereo_buf()
    ctx.reconstruct(dev.wave, dev.wave_off, dev.img_tel, dev.evt_off, mode, start, W, t_hi, t_lo, core_nb, h_ref, s_ref)
    ctx.check()
    n_img_d = torch.tensor([wl.n_img], dtype=torch.int64, device="cuda")
    n_evt_d = torch.tensor([wl.n_evt], dtype=torch.int64, device="cuda")
    h, s = dev.hillas_buf(), dev.stereo_buf()
    g = rta.rta_graph_create(ctx.handle, dev.wave.data_ptr(), dev.wave.numel(), dev.wave_off.data_ptr(),
                             dev.img_tel.data_ptr(), n_img_d.data_ptr(), wl.n_img, dev.evt_off.data_ptr(),
                             n_evt_d.data_ptr(), wl.n_evt, mode, start, W, t_hi, t_lo, core_nb, h.data_ptr(),
                             s.data_ptr())
    stream = torch.cuda.current_stream().cuda_stream
    try:
        rta.rta_graph_launch(g, stream)
        ctx.check(stream)
        assert torch.equal(h, h_ref) and torch.equal(s, s_ref)
        for n_ev in [57, 1, 200]:
            h.fill_(float("nan"))
            s.fill_(float("nan"))
            n_img = int(wl.evt_off[n_ev])
            n_img_d.fill_(n_img)
            n_evt_d.fill_(n_ev)
            rta.rta_graph_launch(g, stream)
            ctx.check(stream)
            assert torch.equal(h[: n_img * 16], h_ref[: n_img * 16])
            assert torch.equal(s[: n_ev * 8], s_ref[: n_ev * 8])
            assert bool(torch.isnan(h[n_img * 16:]).all()) and bool(torch.isnan(s[n_ev * 8:]).all())
    finally:
        rta.rta_graph_destroy(g)
    ctx.close()
