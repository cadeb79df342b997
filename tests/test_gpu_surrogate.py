"""The learned deep-sets surrogate on the GPU against its FP64 oracle, and what
training it gains over the geometric reconstruction.

Parity inputs are built on the CPU only: Hillas rows from the CPU oracle,
rounded to FP32, feed both sides; the network weights come from a seeded numpy
initialiser, rounded to BF16. The oracle takes the same BF16 features and
weights and computes in FP64; the GPU keeps activations in BF16 between layers.

Tolerances (derived from BF16 storage of four activation layers, 2^-9 relative
each): forward outputs |dy| <= 2e-2 (1 + |y|); per-tensor gradients cosine
>= 0.999 and relative L2 <= 2e-2; baselines 1e-4 deg.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_1307_6489_gb300 as rta
from oracle import mlp

from gpu_helpers import Dev, f32_rows_as_oracle, hillas_rows_as_f32, make_ctx, proc_args, stereo_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Y_TOL = 2e-2
G_COS, G_REL = 0.999, 2e-2


def cam_codes(wl):
    codes = np.zeros(16, np.float32)
    for c, cam in wl.cams.items():
        codes[c] = np.log10(cam.mirror_area) - 2.0
    return codes


def make_setup(n_events):
    wl = synth.make_workload(3, n_events)
    ref = oracle.reconstruct(wl, do_stereo=False)
    rows32 = hillas_rows_as_f32(ref["hillas"])
    same = f32_rows_as_oracle(rows32)
    ctx = make_ctx(wl)
    codes = cam_codes(wl)
    model = rta.rta_surrogate_create(ctx.handle, 7, codes)
    p = {k: mlp.bf16_round(v) for k, v in mlp.init_params(11).items()}
    rta.rta_surrogate_set_params(model, rta.pack_params(p))
    tel_code = codes[wl.tel_cam]
    X, used, base, n_used = mlp.features(same, wl.evt_off, wl.img_tel, wl.tel_xy.astype(np.float64), tel_code)
    d = dict(h=torch.from_numpy(rows32.reshape(-1)).cuda(), img_tel=torch.from_numpy(wl.img_tel).cuda(),
             evt_off=torch.from_numpy(wl.evt_off).cuda(),
             logE=torch.from_numpy(np.log10(wl.truth[:, 0]).astype(np.float32)).cuda(),
             src=torch.from_numpy(wl.truth[:, 1:3].astype(np.float32).reshape(-1)).cuda(),
             gam=torch.from_numpy((wl.truth[:, 5] == 0).astype(np.uint8)).cuda())
    return dict(wl=wl, ctx=ctx, model=model, p=p, same=same, X=X, used=used, base=base, n_used=n_used, d=d,
                rows32=rows32)


def close_setup(s):
    rta.rta_surrogate_destroy(s["model"])
    s["ctx"].close()


@pytest.fixture(scope="module")
def setup():
    s = make_setup(300)
    yield s
    close_setup(s)


@pytest.fixture(scope="module")
def big():
    """A training-sized batch: about 100 tiles of 128 image rows with a ragged
    last one, and weight gradients reduced over several K-ranges."""
    s = make_setup(3000)
    yield s
    close_setup(s)


def gpu_forward(s):
    wl, d = s["wl"], s["d"]
    y = torch.zeros(wl.n_evt * 4, dtype=torch.float32, device="cuda")
    b = torch.zeros(wl.n_evt * 2, dtype=torch.float32, device="cuda")
    rta.rta_surrogate_forward(s["model"], d["h"].data_ptr(), d["img_tel"].data_ptr(), wl.n_img, d["evt_off"].data_ptr(),
                              wl.n_evt, y.data_ptr(), b.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return y.cpu().numpy().reshape(-1, 4), b.cpu().numpy().reshape(-1, 2)


@pytest.mark.parametrize("which", ["setup", "big"])
def test_forward_and_baseline_match_the_oracle(which, request):
    s = request.getfixturevalue(which)
    y, b = gpu_forward(s)
    np.testing.assert_allclose(b, s["base"], atol=1e-4)
    y_ref, _ = mlp.forward(s["p"], mlp.bf16_round(s["X"]), s["used"], s["wl"].evt_off)
    err = np.abs(y - y_ref) / (1 + np.abs(y_ref))
    print("forward max scaled error", err.max(axis=0))
    assert err.max() <= Y_TOL
    assert np.abs(y_ref).max() > 0.1                      # a non-trivial network


@pytest.mark.parametrize("which", ["setup", "big"])
def test_gradients_match_the_oracle(which, request):
    s = request.getfixturevalue(which)
    wl, d = s["wl"], s["d"]
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    rta.rta_surrogate_train_step(s["model"], d["h"].data_ptr(), d["img_tel"].data_ptr(), wl.n_img,
                                 d["evt_off"].data_ptr(), wl.n_evt, d["logE"].data_ptr(), d["src"].data_ptr(),
                                 d["gam"].data_ptr(), 1e-3, 0, loss.data_ptr(), torch.cuda.current_stream().cuda_stream)
    g = rta.unpack_params(rta.rta_surrogate_get_params(s["model"], 1))
    y_ref, cache = mlp.forward(s["p"], mlp.bf16_round(s["X"]), s["used"], wl.evt_off)
    L_ref, dy = mlp.loss(y_ref, np.log10(wl.truth[:, 0]), wl.truth[:, 1:3] - s["base"], wl.truth[:, 5] == 0)
    g_ref = mlp.backward(s["p"], cache, dy)
    assert float(loss.item()) == pytest.approx(L_ref, rel=2e-2)
    for k in g_ref:
        a, r = g[k].reshape(-1).astype(np.float64), g_ref[k].reshape(-1)
        cos = a @ r / (np.linalg.norm(a) * np.linalg.norm(r))
        rel = np.linalg.norm(a - r) / np.linalg.norm(r)
        print(k, "cos", cos, "rel", rel)
        assert cos >= G_COS and rel <= G_REL, k


def test_adam_step_moves_each_weight_by_lr_against_its_gradient(setup):
    s = setup
    wl, d = s["wl"], s["d"]
    ctx = s["ctx"]
    model = rta.rta_surrogate_create(ctx.handle, 3, cam_codes(wl))
    try:
        rta.rta_surrogate_set_params(model, rta.pack_params(s["p"]))
        lr = 1e-3
        rta.rta_surrogate_train_step(model, d["h"].data_ptr(), d["img_tel"].data_ptr(), wl.n_img,
                                     d["evt_off"].data_ptr(), wl.n_evt, d["logE"].data_ptr(), d["src"].data_ptr(),
                                     d["gam"].data_ptr(), lr, 1, 0, torch.cuda.current_stream().cuda_stream)
        new = rta.unpack_params(rta.rta_surrogate_get_params(model, 0))
        g = rta.rta_surrogate_get_params(model, 1)
        m = rta.rta_surrogate_get_params(model, 2)
        v = rta.rta_surrogate_get_params(model, 3)
        # first and second moments after one step from zero, with the FP32 values of 1 - beta
        one_m_b1 = np.float32(1) - np.float32(0.9)
        one_m_b2 = np.float32(1) - np.float32(0.999)
        np.testing.assert_allclose(m, one_m_b1 * g, rtol=1e-6, atol=1e-12)
        np.testing.assert_allclose(v, one_m_b2 * (g * g), rtol=1e-6, atol=1e-20)
        y_ref, cache = mlp.forward(s["p"], mlp.bf16_round(s["X"]), s["used"], wl.evt_off)
        _, dy = mlp.loss(y_ref, np.log10(wl.truth[:, 0]), wl.truth[:, 1:3] - s["base"], wl.truth[:, 5] == 0)
        g_ref = mlp.backward(s["p"], cache, dy)
        for k in g_ref:
            sel = np.abs(g_ref[k]) > 1e-2 * np.abs(g_ref[k]).max()
            step = new[k][sel] - s["p"][k][sel]
            np.testing.assert_allclose(step, -lr * np.sign(g_ref[k][sel]), atol=2e-5 + 1e-6 * np.abs(s["p"][k][sel]).max())
    finally:
        rta.rta_surrogate_destroy(model)


def test_inference_flags_and_geometric_fallback(setup):
    s = setup
    wl, d, ctx = s["wl"], s["d"], s["ctx"]
    y, b = gpu_forward(s)
    geo = torch.zeros(wl.n_evt * 8, dtype=torch.float32, device="cuda")
    ctx.stereo(d["h"], d["evt_off"], d["img_tel"], geo)
    st = stereo_rows(geo, wl.n_evt)
    for bound in [1e3, 1e-4, 0.3]:
        out = torch.zeros(wl.n_evt * 32, dtype=torch.uint8, device="cuda")
        rta.rta_surrogate_infer(s["model"], d["h"].data_ptr(), d["img_tel"].data_ptr(), wl.n_img,
                                d["evt_off"].data_ptr(), wl.n_evt, bound, out.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
        ctx.check()
        ev = rta.events_to_numpy(out.cpu().numpy())
        nodir = s["n_used"] < 2
        np.testing.assert_array_equal((ev["flags"] & rta.RTA_EF_NO_DIRECTION) != 0,
                                      nodir | (((ev["flags"] & rta.RTA_EF_FALLBACK) != 0) & (st["flags"] != 0)))
        fb = (ev["flags"] & rta.RTA_EF_FALLBACK) != 0
        expect_fb = ~nodir & (np.hypot(y[:, 1], y[:, 2]) > bound)
        np.testing.assert_array_equal(fb, expect_fb)
        ok = fb & (st["flags"] == 0)
        np.testing.assert_array_equal(ev["dir_x"][ok], st["dir_x"][ok])
        keep = ~fb & ~nodir
        # the inference kernels sum the event network in the tensor core's own order
        np.testing.assert_allclose(ev["dir_x"][keep], b[keep, 0] + y[keep, 1], rtol=0, atol=2e-3)
        assert np.max(np.abs(ev["log_energy"] - y[:, 0]) / (1 + np.abs(y[:, 0]))) <= 2e-3
        np.testing.assert_allclose(ev["gammaness"], 1 / (1 + np.exp(-y[:, 3].astype(np.float64))), atol=2e-3)


def test_inference_kernels_match_the_fp64_oracle(setup):
    """rta_surrogate_infer (the tcgen05 inference kernels, fallback off) directly
    against the FP64 oracle's forward pass with the same BF16 weights and BF16
    features: used counts and no-direction flags exact, baselines within 1e-4 deg,
    energy, direction offsets and the gammaness logit within the forward bar
    2e-2 (1 + |y|) (four BF16 activation stores on the GPU side)."""
    s = setup
    wl, d = s["wl"], s["d"]
    out = torch.zeros(wl.n_evt * 32, dtype=torch.uint8, device="cuda")
    rta.rta_surrogate_infer(s["model"], d["h"].data_ptr(), d["img_tel"].data_ptr(), wl.n_img,
                            d["evt_off"].data_ptr(), wl.n_evt, 1e30, out.data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
    s["ctx"].check()
    ev = rta.events_to_numpy(out.cpu().numpy())
    y_ref, _ = mlp.forward(s["p"], mlp.bf16_round(s["X"]), s["used"], wl.evt_off)
    np.testing.assert_array_equal(ev["n_used"], s["n_used"])
    nodir = s["n_used"] < 2
    np.testing.assert_array_equal((ev["flags"] & rta.RTA_EF_NO_DIRECTION) != 0, nodir)
    assert ((ev["flags"] & rta.RTA_EF_FALLBACK) == 0).all()
    np.testing.assert_allclose(ev["base_x"], s["base"][:, 0], atol=1e-4)
    np.testing.assert_allclose(ev["base_y"], s["base"][:, 1], atol=1e-4)
    tol = Y_TOL * (1 + np.abs(y_ref))
    assert (np.abs(ev["log_energy"] - y_ref[:, 0]) <= tol[:, 0]).all()
    ok = ~nodir
    assert (np.abs(ev["dir_x"][ok] - s["base"][ok, 0] - y_ref[ok, 1]) <= tol[ok, 1] + 1e-4).all()
    assert (np.abs(ev["dir_y"][ok] - s["base"][ok, 1] - y_ref[ok, 2]) <= tol[ok, 2] + 1e-4).all()
    # |sigmoid(a) - sigmoid(b)| <= |a - b| / 4: the logit bar carried to the gammaness
    sig = 1 / (1 + np.exp(-y_ref[:, 3]))
    err = np.abs(ev["gammaness"] - sig) / (0.25 * (1 + np.abs(y_ref[:, 3])))
    print("inference vs oracle: max scaled gammaness error", err.max())
    assert err.max() <= Y_TOL
    assert np.abs(y_ref).max() > 0.1 and ok.sum() > 0.3 * wl.n_evt


def test_trained_network_gains_over_the_geometric_reconstruction():
    """Train on 24k mixed gamma/proton events with the GPU kernels, evaluate on 6k
    held-out events: the learned path adds an energy estimate and a gamma/hadron
    score that the geometric method does not have, at a comparable direction."""
    from paper_1307_6489_gb300 import train
    wl = synth.make_workload(3, 30000)
    ctx = make_ctx(wl)
    dev = Dev(wl)
    proc = proc_args(wl)
    h = train.reconstruct_images(ctx, dev.wave, dev.wave_off, dev.img_tel, dev.evt_off, proc)
    n_tr = 24000
    i_tr = int(wl.evt_off[n_tr])
    logE = torch.from_numpy(np.log10(wl.truth[:, 0]).astype(np.float32)).cuda()
    src = torch.from_numpy(wl.truth[:, 1:3].astype(np.float32).reshape(-1)).cuda()
    gam = torch.from_numpy((wl.truth[:, 5] == 0).astype(np.uint8)).cuda()
    tr = train.SurrogateTrainer(ctx, seed=1, cam_code=cam_codes(wl))
    losses = tr.fit(h[: i_tr * 16], dev.img_tel[:i_tr], wl.evt_off[: n_tr + 1], logE, src, gam, epochs=25,
                    batch_events=1024, lr=2e-3, lr_end=1e-4)
    assert np.mean(losses[-20:]) < 0.5 * np.mean(losses[:5])
    # held-out events
    off_te = torch.from_numpy((wl.evt_off[n_tr:] - i_tr).astype(np.int32)).cuda()
    h_te, tel_te = h[i_tr * 16:].contiguous(), dev.img_tel[i_tr:].contiguous()
    ev = rta.events_to_numpy(tr.infer(h_te, tel_te, off_te, fallback_deg=0.5).cpu().numpy())
    geo = torch.zeros((wl.n_evt - n_tr) * 8, dtype=torch.float32, device="cuda")
    ctx.stereo(h_te, off_te, tel_te, geo)
    res = train.evaluate(ev, stereo_rows(geo, wl.n_evt - n_tr), wl.truth[n_tr:])
    print("surrogate vs geometric:", res)
    assert res["energy_res"] < 0.3 and abs(res["energy_bias"]) < 0.1
    assert res["auc_gamma_hadron"] > 0.75
    assert res["r68_ratio"] < 1.1            # the bound on the learned direction: at most 1.1x geometric
    tr.close()
    ctx.close()


def _infer_and_forward(s, a, b, merge=1, break_offsets=False):
    """Events [a, b) of the parity workload through the fused inference kernel and
    through the layer-by-layer forward pass; merge > 1 joins that many consecutive
    events into one (events of hundreds of images), break_offsets plants
    malformed offsets."""
    wl, d = s["wl"], s["d"]
    off = wl.evt_off[a:b + 1:merge].astype(np.int64)
    if off[-1] != wl.evt_off[b]:
        off = np.append(off, wl.evt_off[b])
    i0 = int(off[0])
    off = (off - i0).astype(np.int32)
    n_img, n_evt = int(off[-1]), len(off) - 1
    if break_offsets:
        off[min(3, n_evt)] = -5                    # events 2 and 3 malformed
        off[min(10, n_evt)] = n_img + 100          # events 9 and 10 malformed
    h = d["h"][i0 * 16:].contiguous()
    tel = d["img_tel"][i0:].contiguous()
    doff = torch.from_numpy(off).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    y = torch.zeros(n_evt * 4, dtype=torch.float32, device="cuda")
    bb = torch.zeros(n_evt * 2, dtype=torch.float32, device="cuda")
    rta.rta_surrogate_forward(s["model"], h.data_ptr(), tel.data_ptr(), n_img, doff.data_ptr(), n_evt, y.data_ptr(),
                              bb.data_ptr(), stream)
    out = torch.zeros(n_evt * 32, dtype=torch.uint8, device="cuda")
    rta.rta_surrogate_infer(s["model"], h.data_ptr(), tel.data_ptr(), n_img, doff.data_ptr(), n_evt, 1e3,
                            out.data_ptr(), stream)
    torch.cuda.synchronize()
    return rta.events_to_numpy(out.cpu().numpy()), y.cpu().numpy().reshape(-1, 4), bb.cpu().numpy().reshape(-1, 2)


@pytest.mark.parametrize("case", ["all", "one", "ragged", "hundreds_of_images", "malformed"])
def test_inference_kernels_agree_with_the_layer_by_layer_forward(setup, case):
    """The fused inference kernel (baseline, features, telescope network and
    pooling with the training path's expressions and orders) against the
    training-path forward (its tensor-core GEMM kernels) on the same batch:
    baselines and used
    counts bit for bit, outputs within FP32 accumulation-order effects. The
    event network's products are exact and its sums FP32 in both, in a
    different order; a BF16 rounding of an activation can flip by one unit, so
    the bound is 2e-3 (1 + |y|)."""
    s = setup
    n = s["wl"].n_evt
    a, b, merge, brk = {"all": (0, n, 1, False), "one": (7, 8, 1, False), "ragged": (5, 5 + 211, 1, False),
                        "hundreds_of_images": (0, n, 25, False), "malformed": (0, 64, 1, True)}[case]
    ev, y, base = _infer_and_forward(s, a, b, merge, brk)
    np.testing.assert_array_equal(ev["base_x"].view(np.uint32), base[:, 0].view(np.uint32))
    np.testing.assert_array_equal(ev["base_y"].view(np.uint32), base[:, 1].view(np.uint32))
    tol = 2e-3 * (1 + np.abs(y))
    dy = np.stack([ev["log_energy"] - y[:, 0], ev["dir_x"] - base[:, 0] - y[:, 1], ev["dir_y"] - base[:, 1] - y[:, 2]],
                  axis=1)
    print(case, "max |dy| / (1 + |y|):", np.max(np.abs(dy) / (1 + np.abs(y[:, :3]))))
    assert (np.abs(dy) <= tol[:, :3]).all()
    sig = 1 / (1 + np.exp(-y[:, 3].astype(np.float64)))
    assert np.max(np.abs(ev["gammaness"] - sig)) <= 2e-3
    assert ((ev["flags"] & rta.RTA_EF_FALLBACK) == 0).all()
    np.testing.assert_array_equal((ev["flags"] & rta.RTA_EF_NO_DIRECTION) != 0, ev["n_used"] < 2)
    if case == "malformed":
        assert (ev["n_used"][[2, 3, 9, 10]] == -1).all() and (ev["n_used"] >= 0).sum() == len(ev["n_used"]) - 4
    elif merge == 1:
        np.testing.assert_array_equal(ev["n_used"], s["n_used"][a:b])
    else:
        assert ev["n_used"].max() > 64


@pytest.mark.parametrize("bound", [1e3, 0.05])
def test_fused_learned_call_equals_the_two_calls(setup, bound):
    """rta_reconstruct_learned runs the image kernel and then the inference kernel,
    which reads the event offsets, telescope ids and weights before its dependency
    wait: its Hillas rows and event rows equal those of rta_image_chain followed
    by rta_surrogate_infer bit for bit, with (bound 0.05 deg) and without
    geometric fallbacks, on three calls in a row."""
    s = setup
    wl, ctx = s["wl"], s["ctx"]
    dv = Dev(wl)
    proc = proc_args(wl)
    stream = torch.cuda.current_stream().cuda_stream
    h_ref, ev_ref = dv.hillas_buf(), torch.zeros(wl.n_evt * 32, dtype=torch.uint8, device="cuda")
    rta.rta_image_chain(ctx.handle, dv.wave.data_ptr(), dv.wave.numel(), dv.wave_off.data_ptr(), dv.img_tel.data_ptr(),
                        wl.n_img, *proc, h_ref.data_ptr(), stream)
    rta.rta_surrogate_infer(s["model"], h_ref.data_ptr(), dv.img_tel.data_ptr(), wl.n_img, dv.evt_off.data_ptr(),
                            wl.n_evt, bound, ev_ref.data_ptr(), stream)
    torch.cuda.synchronize()
    ctx.check()
    ev0 = rta.events_to_numpy(ev_ref.cpu().numpy())
    if bound < 1:
        assert ((ev0["flags"] & rta.RTA_EF_FALLBACK) != 0).sum() > 5
    for _ in range(3):
        h, ev = dv.hillas_buf(), torch.zeros(wl.n_evt * 32, dtype=torch.uint8, device="cuda")
        rta.rta_reconstruct_learned(s["model"], dv.wave.data_ptr(), dv.wave.numel(), dv.wave_off.data_ptr(),
                                    dv.img_tel.data_ptr(), wl.n_img, dv.evt_off.data_ptr(), wl.n_evt, *proc, bound,
                                    h.data_ptr(), ev.data_ptr(), stream)
        torch.cuda.synchronize()
        ctx.check()
        assert torch.equal(h.view(torch.int32), h_ref.view(torch.int32))
        assert torch.equal(ev, ev_ref)


@pytest.mark.parametrize("merge", [6, 25])
def test_fallback_of_large_events_equals_the_stereo_kernel(setup, merge):
    """Every event falls back (bound 1e-4 deg) and events are joined into events of
    about 28 or 115 images, so a CTA holds several events of more than 24 images:
    two groups of eight warps take them two at a time. Their directions equal
    rta_stereo's bit for bit, and invalid intersections give no direction."""
    s = setup
    wl, d, ctx = s["wl"], s["d"], s["ctx"]
    off = wl.evt_off[::merge].astype(np.int64)
    if off[-1] != wl.evt_off[-1]:
        off = np.append(off, wl.evt_off[-1])
    off = off.astype(np.int32)
    n_evt = len(off) - 1
    doff = torch.from_numpy(off).cuda()
    out = torch.zeros(n_evt * 32, dtype=torch.uint8, device="cuda")
    rta.rta_surrogate_infer(s["model"], d["h"].data_ptr(), d["img_tel"].data_ptr(), wl.n_img, doff.data_ptr(), n_evt,
                            1e-4, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    geo = torch.zeros(n_evt * 8, dtype=torch.float32, device="cuda")
    ctx.stereo(d["h"], doff, d["img_tel"], geo)
    torch.cuda.synchronize()
    ctx.check()
    ev = rta.events_to_numpy(out.cpu().numpy())
    st = stereo_rows(geo, n_evt)
    big = np.diff(off) > 24
    assert big.sum() >= 4
    fb = (ev["flags"] & rta.RTA_EF_FALLBACK) != 0
    ok = fb & (st["flags"] == 0)
    assert ok[big].sum() >= 4
    np.testing.assert_array_equal(ev["dir_x"][ok].view(np.uint32), st["dir_x"][ok].view(np.uint32))
    np.testing.assert_array_equal(ev["dir_y"][ok].view(np.uint32), st["dir_y"][ok].view(np.uint32))
    nodir = (ev["flags"] & rta.RTA_EF_NO_DIRECTION) != 0
    np.testing.assert_array_equal(nodir[fb], st["flags"][fb] != 0)


def test_fused_learned_call_with_empty_events_and_no_images(setup):
    """Events without images (the call then launches no image kernel, and the
    inference reads its inputs after the dependency wait) get no direction and
    zero used images; an empty event list is accepted and writes nothing."""
    s = setup
    wl, ctx = s["wl"], s["ctx"]
    dv = Dev(wl)
    proc = proc_args(wl)
    stream = torch.cuda.current_stream().cuda_stream
    n_evt = 5
    off = torch.zeros(n_evt + 1, dtype=torch.int32, device="cuda")
    h = dv.hillas_buf()
    ev = torch.full((n_evt * 32,), 255, dtype=torch.uint8, device="cuda")
    rta.rta_reconstruct_learned(s["model"], dv.wave.data_ptr(), dv.wave.numel(), dv.wave_off.data_ptr(),
                                dv.img_tel.data_ptr(), 0, off.data_ptr(), n_evt, *proc, 0.5, h.data_ptr(),
                                ev.data_ptr(), stream)
    torch.cuda.synchronize()
    ctx.check()
    e = rta.events_to_numpy(ev.cpu().numpy())
    assert (e["n_used"] == 0).all()
    assert ((e["flags"] & rta.RTA_EF_NO_DIRECTION) != 0).all()
    before = ev.clone()
    rta.rta_reconstruct_learned(s["model"], dv.wave.data_ptr(), dv.wave.numel(), dv.wave_off.data_ptr(),
                                dv.img_tel.data_ptr(), 0, off.data_ptr(), 0, *proc, 0.5, h.data_ptr(),
                                ev.data_ptr(), stream)
    torch.cuda.synchronize()
    assert torch.equal(ev, before)


def test_training_resumed_from_a_checkpoint_takes_the_same_steps(setup, tmp_path):
    """Train 4 Adam steps, save, train 3 more; a new trainer resumed from the file
    trains the same 3 steps: parameters, moments and step count bit for bit."""
    from paper_1307_6489_gb300 import train
    s = setup
    wl, d, ctx = s["wl"], s["d"], s["ctx"]
    args = (d["h"], d["img_tel"], wl.evt_off, d["logE"], d["src"], d["gam"])
    a = train.SurrogateTrainer(ctx, seed=21, cam_code=cam_codes(wl))
    b = None
    try:
        a.fit(*args, epochs=2, batch_events=150, lr=1e-3, lr_end=1e-3, seed=0)
        f = str(tmp_path / "ck.bin")
        a.save(f)
        a.fit(*args, epochs=1, batch_events=100, lr=1e-3, lr_end=1e-3, seed=1)
        b = train.SurrogateTrainer.resume(ctx, f)
        b.fit(*args, epochs=1, batch_events=100, lr=1e-3, lr_end=1e-3, seed=1)
        pa, ma, va, sa = rta.rta_surrogate_get_state(a.model)
        pb, mb, vb, sb = rta.rta_surrogate_get_state(b.model)
        assert sa == sb == 7
        for x, y in [(pa, pb), (ma, mb), (va, vb)]:
            np.testing.assert_array_equal(x.view(np.uint32), y.view(np.uint32))
    finally:
        a.close()
        if b is not None:
            b.close()
