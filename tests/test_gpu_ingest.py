"""DL0 byte-stream ingest on the GPU (rta_ingest) against the oracle decoder,
and the zero-copy reconstruction (rta_reconstruct_stream) against the
reconstruction of the same bundle in the contiguous layout. Directories and
fault reports are compared exactly; the reconstruction must be bit-identical."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
import paper_1307_6489_gb300 as rta
from oracle import ingest

from gpu_helpers import Dev, compare_hillas, hillas_rows, make_ctx, proc_args

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def cams_of(wl):
    return {c: (cam.n_pix, cam.n_samples) for c, cam in wl.cams.items()}


class GpuDir:
    """Device buffers of a directory with the given capacities."""

    def __init__(self, seg_cap, img_cap, evt_cap):
        self.seg_cap, self.img_cap, self.evt_cap = seg_cap, img_cap, evt_cap
        self.seg = torch.zeros(max(seg_cap, 1) * 2, dtype=torch.int64, device="cuda")
        self.img_seg = torch.zeros(img_cap + 1, dtype=torch.int32, device="cuda")
        self.img_tel = torch.zeros(max(img_cap, 1), dtype=torch.int32, device="cuda")
        self.evt_off = torch.zeros(evt_cap + 1, dtype=torch.int32, device="cuda")
        self.evt_number = torch.zeros(max(evt_cap, 1), dtype=torch.int64, device="cuda")
        self.evt_time = torch.zeros(max(evt_cap, 1), dtype=torch.int64, device="cuda")
        self.counts = torch.zeros(6, dtype=torch.int64, device="cuda")

    def ingest(self, ctx, d_stream, n_bytes, verify_crc=True):
        rta.rta_ingest(ctx.handle, d_stream.data_ptr(), n_bytes, verify_crc, self.seg.data_ptr(), self.seg_cap,
                       self.img_seg.data_ptr(), self.img_tel.data_ptr(), self.img_cap, self.evt_off.data_ptr(),
                       self.evt_number.data_ptr(), self.evt_time.data_ptr(), self.evt_cap, self.counts.data_ptr())
        torch.cuda.synchronize()
        bits = 0
        try:
            ctx.check()
        except rta.RtaError as e:
            bits = e.bits
        c = self.counts.cpu().numpy()
        n_seg, n_img, n_evt = int(c[0]), int(c[1]), int(c[2])
        seg = self.seg.cpu().numpy().view(np.uint8)[: n_seg * 16].view(rta.SEGMENT_DTYPE)
        return dict(seg=np.stack([seg["offset"], seg["first_pixel"], seg["n_pixels"]], 1).astype(np.int64),
                    img_seg=self.img_seg.cpu().numpy()[: n_img + 1] if not c[4] else np.zeros(0, np.int32),
                    img_tel=self.img_tel.cpu().numpy()[:n_img], evt_off=self.evt_off.cpu().numpy()[: n_evt + 1]
                    if not c[4] else np.zeros(0, np.int32),
                    evt_number=self.evt_number.cpu().numpy()[:n_evt].view(np.uint64),
                    evt_time_ns=self.evt_time.cpu().numpy()[:n_evt], n_samples=int(c[3]), error=int(c[4]),
                    error_offset=int(c[5]), bits=bits)


def dev_bytes(buf):
    """A 16-byte aligned device copy of a byte stream."""
    t = torch.zeros((len(buf) + 15) // 16 * 16 + 16, dtype=torch.uint8, device="cuda")
    t[: len(buf)] = torch.from_numpy(np.ascontiguousarray(buf))
    assert t.data_ptr() % 16 == 0
    return t


def compare_dirs(g, r):
    assert (g["error"], g["error_offset"]) == (r["error"], r["error_offset"])
    if r["error"]:
        assert g["bits"] & rta.RTA_DEV_BAD_STREAM
        return
    assert g["bits"] == 0
    np.testing.assert_array_equal(g["seg"], r["seg"])
    np.testing.assert_array_equal(g["img_seg"], r["img_seg"])
    np.testing.assert_array_equal(g["img_tel"], r["img_tel"])
    np.testing.assert_array_equal(g["evt_off"], r["evt_off"])
    np.testing.assert_array_equal(g["evt_number"], r["evt_number"])
    np.testing.assert_array_equal(g["evt_time_ns"], r["evt_time_ns"])
    assert g["n_samples"] == r["n_samples"]


@pytest.fixture(scope="module")
def sset():
    wl = synth.make_workload(2, 120)
    ctx = make_ctx(wl)
    yield wl, ctx
    ctx.close()


@pytest.mark.parametrize("seg", [None, {1: 200, 2: 256, 3: 520}])
@pytest.mark.parametrize("crc", [True, False])
def test_directory_matches_the_oracle(sset, seg, crc):
    wl, ctx = sset
    t = 1_700_000_000_000_000_000 + 987_654_321 * np.arange(wl.n_evt)
    buf, plan = synth.encode_stream(wl, times_ns=t, seg_pixels=seg)
    assert len(buf) > 8 << 20                              # several 1 MiB pieces
    r = ingest.decode_stream(buf, wl.tel_cam, cams_of(wl), verify_crc=crc)
    d = GpuDir(len(plan["img"]) + 5, wl.n_img + 3, wl.n_evt + 1)
    g = d.ingest(ctx, dev_bytes(buf), len(buf), crc)
    compare_dirs(g, r)
    assert g["error"] == 0 and len(g["img_tel"]) == wl.n_img


def test_every_planted_fault_is_reported_like_the_oracle(sset):
    from test_oracle_ingest import faults
    wl, ctx = sset
    buf, plan, cases = faults(wl, cams_of(wl))
    d = GpuDir(len(plan["img"]) + 5, wl.n_img + 3, wl.n_evt + 1)
    for name, b, code, k in cases:
        r = ingest.decode_stream(b, wl.tel_cam, cams_of(wl))
        assert r["error"] == code, name
        compare_dirs(d.ingest(ctx, dev_bytes(b), len(b)), r)
    # a clean stream afterwards decodes again
    compare_dirs(d.ingest(ctx, dev_bytes(buf), len(buf)), ingest.decode_stream(buf, wl.tel_cam, cams_of(wl)))


def test_short_packets_crc_like_the_oracle():
    """Segments of 8 pixels: packets of 18-43 16-byte words, so some warps have
    lanes without a word (fewer words than lanes) and some exactly one more than
    the lanes; the clean stream and a flipped bit in a short packet and in a
    long one are judged like the oracle."""
    wl = synth.make_workload(2, 6)
    ctx = make_ctx(wl)
    buf, plan = synth.encode_stream(wl, seg_pixels={1: 8, 2: 8, 3: 8})
    words = plan["size"] // 16
    assert words.min() < 32 and words.max() > 32 and (words == 33).any()
    d = GpuDir(len(plan["img"]) + 5, wl.n_img + 3, wl.n_evt + 1)
    r = ingest.decode_stream(buf, wl.tel_cam, cams_of(wl), verify_crc=True)
    assert r["error"] == 0
    compare_dirs(d.ingest(ctx, dev_bytes(buf), len(buf), True), r)
    for k in (int(np.argmin(words)), int(np.nonzero(words == 33)[0][0]), int(np.argmax(words))):
        b = buf.copy()
        b[plan["off"][k] + plan["size"][k] - 20] ^= 0x01          # a sample bit near the packet's end
        r = ingest.decode_stream(b, wl.tel_cam, cams_of(wl), verify_crc=True)
        assert (r["error"], r["error_offset"]) == (ingest.CRC, plan["off"][k])
        compare_dirs(d.ingest(ctx, dev_bytes(b), len(b), True), r)
    ctx.close()


def test_capacities_like_the_oracle(sset):
    wl, ctx = sset
    buf, plan = synth.encode_stream(wl)
    db = dev_bytes(buf)
    for caps in [(len(plan["img"]), wl.n_img, wl.n_evt), (5, wl.n_img, wl.n_evt), (len(plan["img"]), 10, wl.n_evt),
                 (len(plan["img"]), wl.n_img, 3), (0, 0, 0)]:
        r = ingest.decode_stream(buf, wl.tel_cam, cams_of(wl), seg_cap=caps[0], img_cap=caps[1], evt_cap=caps[2])
        compare_dirs(GpuDir(*caps).ingest(ctx, db, len(buf)), r)


def test_a_header_hidden_in_the_samples_is_not_taken_for_a_packet(sset):
    """Two plausible packet headers (valid fields, each the other's successor)
    planted in the samples right at a 1 MiB boundary, the carrying packet's CRC
    fixed up: the piece's scan takes them for packets, the walks do not join,
    and the decoder must still find the true chain."""
    wl, ctx = sset
    buf, plan = synth.encode_stream(wl)
    buf = buf.copy()
    off, size = plan["off"], plan["size"]
    # a 1 MiB boundary inside a packet's samples with room for both fakes after it
    for boundary in range(1 << 20, len(buf), 1 << 20):
        k = int(np.searchsorted(off, boundary, side="right") - 1)
        if off[k] + 32 < boundary and boundary + 2 * 448 + 48 < off[k] + size[k] - 16:
            break
    else:
        pytest.fail("no usable boundary")
    # a fake header for a camera of 25 samples: 8 pixels, 48 + 2*8*25 = 448 bytes
    cam25 = [c for c, cm in wl.cams.items() if cm.n_samples == 25][0]
    tel = int(np.nonzero(wl.tel_cam == cam25)[0][0])
    P = wl.cams[cam25].n_pix

    def fake(pos, first):
        h = bytearray(32)
        h[0:2] = ((1 << 11) | tel).to_bytes(2, "big")
        h[2:4] = ((0 << 14) | 5).to_bytes(2, "big")       # continuation segment
        h[4:6] = (448 - 7).to_bytes(2, "big")
        h[6:10] = bytes([0x10, 200, 1, 0])
        h[16:24] = (77).to_bytes(8, "big")
        h[24:26] = first.to_bytes(2, "big")
        h[26:28] = (8).to_bytes(2, "big")
        h[28:30] = P.to_bytes(2, "big")
        h[30:32] = (25).to_bytes(2, "big")
        buf[pos:pos + 32] = np.frombuffer(bytes(h), np.uint8)

    fake(boundary, 8)
    fake(boundary + 448, 16)
    L = size[k]
    buf[off[k] + L - 2: off[k] + L] = np.frombuffer(ingest.crc16(buf[off[k]:off[k] + L - 2]).to_bytes(2, "big"),
                                                     np.uint8)
    r = ingest.decode_stream(buf, wl.tel_cam, cams_of(wl))
    assert r["error"] == 0
    d = GpuDir(len(plan["img"]), wl.n_img, wl.n_evt)
    compare_dirs(d.ingest(ctx, dev_bytes(buf), len(buf)), r)


def reconstruct_both(wl, ctx, seg=None, nbpeak=False):
    if nbpeak:
        wl.proc = dataclasses.replace(wl.proc, nbpeak=True)
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    dev = Dev(wl)
    h0, s0 = dev.hillas_buf(), dev.stereo_buf()
    ctx.reconstruct(dev.wave, dev.wave_off, dev.img_tel, dev.evt_off, mode, start, W, t_hi, t_lo, core_nb, h0, s0)
    buf, plan = synth.encode_stream(wl, seg_pixels=seg)
    db = dev_bytes(buf)
    d = GpuDir(len(plan["img"]), wl.n_img, wl.n_evt)
    g = d.ingest(ctx, db, len(buf), True)
    assert g["error"] == 0
    h1 = torch.full_like(h0, np.nan)
    s1 = torch.full_like(s0, np.nan)
    rta.rta_reconstruct_stream(ctx.handle, db.data_ptr(), len(buf), d.seg.data_ptr(), d.seg_cap, d.img_seg.data_ptr(),
                               d.img_tel.data_ptr(), wl.n_img, d.evt_off.data_ptr(), wl.n_evt, d.counts.data_ptr(),
                               mode, start, W, t_hi, t_lo, core_nb, h1.data_ptr(), s1.data_ptr())
    torch.cuda.synchronize()
    assert ctx.check() == 0
    return h0, s0, h1, s1, buf, plan


@pytest.mark.parametrize("seg", [None, {1: 200, 2: 256, 3: 520}, {1: 40, 2: 48, 3: 64}])
def test_zero_copy_reconstruction_equals_the_contiguous_bundle(sset, seg):
    wl, ctx = sset
    h0, s0, h1, s1, _, _ = reconstruct_both(wl, ctx, seg)
    assert torch.equal(h0, h1) and torch.equal(s0, s1)
    ref = oracle.reconstruct(wl, do_stereo=False)
    compare_hillas(hillas_rows(h1, wl.n_img), ref["hillas"], "stream")


def test_zero_copy_neighbour_peak_equals_the_contiguous_bundle():
    wl = synth.make_workload(2, 60)
    ctx = make_ctx(wl)
    h0, s0, h1, s1, _, _ = reconstruct_both(wl, ctx, {1: 200, 2: 256, 3: 520}, nbpeak=True)
    assert torch.equal(h0, h1) and torch.equal(s0, s1)
    ctx.close()


def test_full_size_stream():
    """The 10,000-event bundle as a byte stream: directory as the oracle's
    (headers; CRCs checked on the GPU only), zero-copy rows equal to the
    contiguous bundle's."""
    wl = synth.make_workload(2, 10000)
    ctx = make_ctx(wl)
    h0, s0, h1, s1, buf, plan = reconstruct_both(wl, ctx)
    assert torch.equal(h0, h1) and torch.equal(s0, s1)
    r = ingest.decode_stream(buf, wl.tel_cam, cams_of(wl), verify_crc=False)
    d = GpuDir(len(plan["img"]), wl.n_img, wl.n_evt)
    compare_dirs(d.ingest(ctx, dev_bytes(buf), len(buf), True), r)
    ctx.close()


def test_stream_autotune_keeps_the_rows_and_tunes_only_the_stream_path():
    """rta_autotune_stream measures every configuration that fits on the stream,
    keeps one for the stream path alone (the contiguous bundle's stays), and the
    zero-copy rows under it are still those of the contiguous bundle; the
    neighbour-peak window is refused (it is tuned by rta_autotune)."""
    wl = synth.make_workload(2, 120)
    ctx = make_ctx(wl)
    plain = rta.rta_get_chain_config(ctx.handle)
    h0, s0, h1, s1, buf, plan = reconstruct_both(wl, ctx, {1: 200, 2: 256, 3: 520})
    assert torch.equal(h0, h1)
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    db = dev_bytes(buf)
    d = GpuDir(len(plan["img"]), wl.n_img, wl.n_evt)
    assert d.ingest(ctx, db, len(buf), False)["error"] == 0
    ht = torch.full_like(h0, np.nan)
    entries = rta.rta_autotune_stream(ctx.handle, db.data_ptr(), len(buf), d.seg.data_ptr(), d.seg_cap,
                                      d.img_seg.data_ptr(), d.img_tel.data_ptr(), wl.n_img, d.counts.data_ptr(), mode,
                                      start, W, t_hi, t_lo, core_nb, ht.data_ptr(), reps=1)
    torch.cuda.synchronize()
    assert ctx.check() == 0
    assert len(entries) >= 10 and all(e["ms"] > 0 for e in entries)
    assert len({(e["variant"], e["n_stages"], e["ctas_per_sm"]) for e in entries}) == len(entries)
    assert torch.equal(ht, h0)
    assert rta.rta_get_chain_config(ctx.handle) == plain
    # the stream path under the tuned configuration: the same rows and stereo results
    h2 = torch.full_like(h0, np.nan)
    s2 = torch.full_like(s0, np.nan)
    rta.rta_reconstruct_stream(ctx.handle, db.data_ptr(), len(buf), d.seg.data_ptr(), d.seg_cap, d.img_seg.data_ptr(),
                               d.img_tel.data_ptr(), wl.n_img, d.evt_off.data_ptr(), wl.n_evt, d.counts.data_ptr(),
                               mode, start, W, t_hi, t_lo, core_nb, h2.data_ptr(), s2.data_ptr())
    torch.cuda.synchronize()
    assert ctx.check() == 0
    assert torch.equal(h2, h0) and torch.equal(s2, s0)
    with pytest.raises(rta.RtaError) as e:
        rta.rta_autotune_stream(ctx.handle, db.data_ptr(), len(buf), d.seg.data_ptr(), d.seg_cap,
                                d.img_seg.data_ptr(), d.img_tel.data_ptr(), wl.n_img, d.counts.data_ptr(),
                                rta.RTA_WINDOW_NEIGHBOUR, start, W, t_hi, t_lo, core_nb, ht.data_ptr(), reps=1)
    assert e.value.code == rta.RTA_E_INVALID
    ctx.close()
