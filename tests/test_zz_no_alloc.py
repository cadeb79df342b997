"""rta_image_chain_noalloc: the fused image kernel for callers that cannot allocate.

Some callers may not call cudaMalloc (a real-time process that must not stall on
an allocation's device synchronisation, a framework that owns all device memory
through its own pool). They get one entry point that takes only caller-owned
buffers and keeps its scratch in a fixed file-scope device array. This test
calls it through the C ABI twice in a row, on two different bundles, and
checks each result against the context-based rta_image_chain on the same
bundle, within the parity tolerances of the other GPU tests (the rows are in
fact expected to be bit-identical: same kernel, same launch configuration).
The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import synth
import paper_1307_6489_gb300 as rta

from gpu_helpers import Dev, compare_hillas, hillas_rows, make_ctx, proc_args

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def caller_tables(wl):
    """Camera and calibration tables in the caller's own device memory, laid out as the entry point asks."""
    cam_ids = sorted(wl.cams)
    index = {c: i for i, c in enumerate(cam_ids)}
    keep, descs = [], []
    for c in cam_ids:
        cam = wl.cams[c]
        xy = torch.from_numpy(np.ascontiguousarray(cam.xy, np.float32)).cuda()
        nb8 = np.full((cam.n_pix, 8), -1, np.int16)
        nb8[:, :cam.K] = cam.nb
        nb8 = torch.from_numpy(nb8).cuda()
        keep += [xy, nb8]
        descs.append(rta.CameraDesc(cam.n_pix, cam.n_samples, cam.K, xy.data_ptr(), nb8.data_ptr()))
    tel_cam = np.array([index[int(c)] for c in wl.tel_cam], np.int32)
    rows, r = [], 0
    for c in wl.tel_cam:
        rows.append(r)
        r += (wl.cams[int(c)].n_pix + 7) // 8 * 8
    n_rows = r + 8
    p16 = np.zeros(n_rows, np.int32)
    scale = np.zeros(n_rows, np.float32)
    for t, c in enumerate(wl.tel_cam):
        a, b = wl.tel_pix_off[t], wl.tel_pix_off[t + 1]
        p16[rows[t]:rows[t] + (b - a)] = wl.p16[a:b]
        scale[rows[t]:rows[t] + (b - a)] = wl.scale[a:b]
    d_p16 = torch.from_numpy(p16).cuda()
    d_scale = torch.from_numpy(scale).cuda()
    keep += [d_p16, d_scale]
    return descs, tel_cam, np.array(rows, np.int64), d_p16, d_scale, n_rows, keep


def test_noalloc_entry_matches_context_entry_on_two_calls_in_a_row():
    wl = synth.make_workload(2, 400)
    bundles = [synth.subset(wl, np.arange(0, 150)), synth.subset(wl, np.arange(150, 400))]
    ctx = make_ctx(wl)
    descs, tel_cam, tel_row, d_p16, d_scale, n_rows, keep = caller_tables(wl)
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    for b in bundles:
        dev = Dev(b)
        ref = dev.hillas_buf()
        ctx.image_chain(dev.wave, dev.wave_off, dev.img_tel, mode, start, W, t_hi, t_lo, core_nb, ref)
        ctx.check()
        out = torch.full_like(ref, float("nan"))
        stream = torch.cuda.current_stream().cuda_stream
        rta.rta_image_chain_noalloc(descs, tel_cam, tel_row, d_p16.data_ptr(), d_scale.data_ptr(), n_rows,
                                    dev.wave.data_ptr(), dev.wave.numel(), dev.wave_off.data_ptr(),
                                    dev.img_tel.data_ptr(), b.n_img, mode, start, W, t_hi, t_lo, core_nb,
                                    out.data_ptr(), status.data_ptr(), stream)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        g = hillas_rows(out, b.n_img)
        r = hillas_rows(ref, b.n_img)
        ref_rows = np.zeros((b.n_img, 12))
        for j, k in enumerate(rta.HILLAS_FIELDS):
            ref_rows[:, j] = r[k]
        ref_rows[:, 10] = r["n_pix"]
        ref_rows[:, 11] = r["flags"]
        compare_hillas(g, ref_rows, "noalloc vs context")
        np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), ref.cpu().numpy().view(np.uint32))
    ctx.close()


def test_noalloc_entry_rejects_sizes_beyond_its_scratch():
    wl = synth.make_workload(2, 5)
    descs, tel_cam, tel_row, d_p16, d_scale, n_rows, keep = caller_tables(wl)
    dev = Dev(wl)
    out = dev.hillas_buf()
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    too_many = np.zeros(rta.RTA_NOALLOC_MAX_TEL + 1, np.int32)
    with pytest.raises(rta.RtaError) as e:
        rta.rta_image_chain_noalloc(descs, too_many, np.zeros(len(too_many), np.int64), d_p16.data_ptr(),
                                    d_scale.data_ptr(), n_rows, dev.wave.data_ptr(), dev.wave.numel(),
                                    dev.wave_off.data_ptr(), dev.img_tel.data_ptr(), wl.n_img, mode, start, W, t_hi,
                                    t_lo, core_nb, out.data_ptr())
    assert e.value.code == rta.RTA_E_INVALID and "telescopes" in str(e.value)
    with pytest.raises(rta.RtaError) as e:
        rta.rta_image_chain_noalloc(descs * 6, tel_cam, tel_row, d_p16.data_ptr(), d_scale.data_ptr(), n_rows,
                                    dev.wave.data_ptr(), dev.wave.numel(), dev.wave_off.data_ptr(),
                                    dev.img_tel.data_ptr(), wl.n_img, mode, start, W, t_hi, t_lo, core_nb,
                                    out.data_ptr())
    assert e.value.code == rta.RTA_E_INVALID and "camera" in str(e.value)


def _call(descs, tel_cam, tel_row, d_p16, d_scale, n_rows, dev, n_img, proc, out, status_ptr=0):
    mode, start, W, t_hi, t_lo, core_nb = proc
    rta.rta_image_chain_noalloc(descs, tel_cam, tel_row, d_p16.data_ptr(), d_scale.data_ptr(), n_rows,
                                dev.wave.data_ptr(), dev.wave.numel(), dev.wave_off.data_ptr(),
                                dev.img_tel.data_ptr(), n_img, mode, start, W, t_hi, t_lo, core_nb,
                                out.data_ptr(), status_ptr, torch.cuda.current_stream().cuda_stream)


def test_noalloc_status_is_reset_between_calls_and_optional():
    # call 1 has one misaligned image offset: that row is skipped with RTA_HF_BAD_INPUT
    # and the status word reports RTA_DEV_BAD_IMAGE; call 2 on the same stream is clean
    # and must report 0, i.e. the shared scratch's status word was cleared in between
    wl = synth.make_workload(2, 60)
    descs, tel_cam, tel_row, d_p16, d_scale, n_rows, keep = caller_tables(wl)
    proc = proc_args(wl)
    dev = Dev(wl)
    ctx = make_ctx(wl)
    ref = dev.hillas_buf()
    ctx.image_chain(dev.wave, dev.wave_off, dev.img_tel, *proc, ref)
    ctx.check()
    status = torch.full((1,), 777, dtype=torch.int32, device="cuda")
    bad = Dev(wl)
    bad_img = wl.n_img // 2
    bad.wave_off[bad_img] += 4                        # 8 bytes: breaks the 16-byte rule
    out1 = torch.full_like(ref, float("nan"))
    _call(descs, tel_cam, tel_row, d_p16, d_scale, n_rows, bad, wl.n_img, proc, out1, status.data_ptr())
    torch.cuda.synchronize()
    assert int(status.item()) & rta.RTA_DEV_BAD_IMAGE
    r1 = hillas_rows(out1, wl.n_img)
    assert r1["flags"][bad_img] & rta.RTA_HF_BAD_INPUT
    keep_rows = np.arange(wl.n_img) != bad_img
    u1 = out1.cpu().numpy().reshape(-1, 16).view(np.uint32)
    uref = ref.cpu().numpy().reshape(-1, 16).view(np.uint32)
    np.testing.assert_array_equal(u1[keep_rows], uref[keep_rows])
    out2 = torch.full_like(ref, float("nan"))
    _call(descs, tel_cam, tel_row, d_p16, d_scale, n_rows, dev, wl.n_img, proc, out2, status.data_ptr())
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    np.testing.assert_array_equal(out2.cpu().numpy().view(np.uint32), ref.cpu().numpy().view(np.uint32))
    # no status pointer: the same rows
    out3 = torch.full_like(ref, float("nan"))
    _call(descs, tel_cam, tel_row, d_p16, d_scale, n_rows, dev, wl.n_img, proc, out3, 0)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out3.cpu().numpy().view(np.uint32), ref.cpu().numpy().view(np.uint32))
    ctx.close()


def test_noalloc_ignores_neighbour_ids_outside_the_camera():
    # the caller's neighbour tables are not validated: ids outside [0, n_pix) must act
    # like -1 (never read), so the rows equal a context whose tables hold -1 there
    wl = synth.make_workload(2, 80)
    descs, tel_cam, tel_row, d_p16, d_scale, n_rows, keep = caller_tables(wl)
    rng = np.random.default_rng(5)
    cam_ids = sorted(wl.cams)
    ctx = rta.Context(0)
    planted = 0
    for i, c in enumerate(cam_ids):
        cam = wl.cams[c]
        nb = np.array(cam.nb, np.int16).copy()
        nb8 = np.full((cam.n_pix, 8), -1, np.int16)
        nb8[:, :cam.K] = nb
        rows = rng.choice(cam.n_pix, size=cam.n_pix // 3, replace=False)
        for p in rows:
            j = int(rng.integers(cam.K))
            nb8[p, j] = rng.choice([cam.n_pix, cam.n_pix + 1, 4095, 32767, -2, -32768])
            nb[p, j] = -1
            planted += 1
        d_nb8 = torch.from_numpy(nb8).cuda()
        keep.append(d_nb8)
        descs[i] = rta.CameraDesc(cam.n_pix, cam.n_samples, cam.K, descs[i].d_pix_xy, d_nb8.data_ptr())
        ctx.register_camera(c, cam.xy, nb, cam.n_samples)
    ctx.register_array(wl.tel_cam, wl.tel_xy, wl.p16, wl.scale)
    assert planted > 1000
    proc = proc_args(wl)
    assert proc[5] == 1        # the core-neighbour test reads the tables too
    dev = Dev(wl)
    ref = dev.hillas_buf()
    ctx.image_chain(dev.wave, dev.wave_off, dev.img_tel, *proc, ref)
    ctx.check()
    status = torch.full((1,), 777, dtype=torch.int32, device="cuda")
    out = torch.full_like(ref, float("nan"))
    _call(descs, tel_cam, tel_row, d_p16, d_scale, n_rows, dev, wl.n_img, proc, out, status.data_ptr())
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), ref.cpu().numpy().view(np.uint32))
    ctx.close()


def test_noalloc_rejects_bad_calibration_rows():
    wl = synth.make_workload(2, 5)
    descs, tel_cam, tel_row, d_p16, d_scale, n_rows, keep = caller_tables(wl)
    dev = Dev(wl)
    out = dev.hillas_buf()
    proc = proc_args(wl)
    for bad in (tel_row + np.where(np.arange(len(tel_row)) == 3, 4, 0),     # not a multiple of 8
                tel_row + np.where(np.arange(len(tel_row)) == len(tel_row) - 1, 8, 0)):  # no slack left
        with pytest.raises(rta.RtaError) as e:
            _call(descs, tel_cam, bad.astype(np.int64), d_p16, d_scale, n_rows, dev, wl.n_img, proc, out)
        assert e.value.code == rta.RTA_E_INVALID and "calibration row" in str(e.value)
    bad_cam = tel_cam.copy()
    bad_cam[0] = len(descs)
    with pytest.raises(rta.RtaError) as e:
        _call(descs, bad_cam, tel_row, d_p16, d_scale, n_rows, dev, wl.n_img, proc, out)
    assert e.value.code == rta.RTA_E_INVALID


def test_noalloc_refuses_a_stream_under_capture_and_leaves_the_capture_intact():
    # the tables are copied from a stack buffer of the call, which a graph could not
    # replay: under capture the call must refuse before it enqueues anything, and the
    # capture must still complete and replay the work captured around it
    wl = synth.make_workload(2, 40)
    descs, tel_cam, tel_row, d_p16, d_scale, n_rows, keep = caller_tables(wl)
    dev = Dev(wl)
    proc = proc_args(wl)
    ref = dev.hillas_buf()
    _call(descs, tel_cam, tel_row, d_p16, d_scale, n_rows, dev, wl.n_img, proc, ref)
    torch.cuda.synchronize()
    x = torch.zeros(4, device="cuda")
    spare = dev.hillas_buf()
    g = torch.cuda.CUDAGraph()
    refused = None
    with torch.cuda.graph(g):
        x.add_(1.0)
        try:
            _call(descs, tel_cam, tel_row, d_p16, d_scale, n_rows, dev, wl.n_img, proc, spare)
        except rta.RtaError as e:
            refused = e
    assert refused is not None and refused.code == rta.RTA_E_INVALID and "captured" in str(refused)
    g.replay()
    torch.cuda.synchronize()
    assert x.tolist() == [1.0] * 4
    out = torch.full_like(ref, float("nan"))
    _call(descs, tel_cam, tel_row, d_p16, d_scale, n_rows, dev, wl.n_img, proc, out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), ref.cpu().numpy().view(np.uint32))
