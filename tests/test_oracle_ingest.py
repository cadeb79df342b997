"""The DL0 byte-stream decoder oracle pinned to what the format fixes: the CRC
against its published check values and its linearity, a packet written out byte
by byte from the format table, the round trip of generated bundles (also with
many segments per image), and one planted fault of each kind reported at the
packet that holds it."""
import numpy as np
import pytest

import oracle
import synth
from oracle import ingest


def test_crc_check_values_and_linearity():
    assert ingest.crc16(b"123456789") == 0x29B1        # the published check value of CRC-16/CCITT-FALSE
    assert ingest.crc16(b"") == 0xFFFF
    assert ingest.crc16(b"A") == 0xB915
    rng = np.random.default_rng(1)
    for n in (1, 7, 64, 1000):
        x, y, z = (rng.integers(0, 256, n, dtype=np.uint8) for _ in range(3))
        # with the preset register, an XOR of an odd number of equal-length messages
        # has the XOR of their CRCs
        assert ingest.crc16(x ^ y ^ z) == ingest.crc16(x) ^ ingest.crc16(y) ^ ingest.crc16(z)
    m = rng.integers(0, 256, 50, dtype=np.uint8)
    c = ingest.crc16(m)
    for bit in range(0, 400, 7):                        # every single-bit error is detected
        e = m.copy()
        e[bit // 8] ^= np.uint8(1 << (bit % 8))
        assert ingest.crc16(e) != c


def hand_packet(apid, flags, count, event, sec, fine, first, n, P, S, samples):
    """One packet written from the format table, byte by byte."""
    L = 48 + 2 * n * S
    b = bytearray()
    b += bytes([(1 << 3) | (apid >> 8), apid & 0xFF])                  # version 0, TM, sec hdr, APID
    b += bytes([(flags << 6) | (count >> 8), count & 0xFF])
    b += (L - 7).to_bytes(2, "big")
    b += bytes([0x10, 200, 1, 0])
    b += sec.to_bytes(4, "big") + fine.to_bytes(2, "big")
    b += event.to_bytes(8, "big")
    b += first.to_bytes(2, "big") + n.to_bytes(2, "big") + P.to_bytes(2, "big") + S.to_bytes(2, "big")
    b += np.asarray(samples, "<u2").tobytes()
    b += bytes(14)
    b += ingest.crc16(bytes(b)).to_bytes(2, "big")
    assert len(b) == L
    return bytes(b)


def test_a_packet_written_from_the_table():
    # telescope 5 has camera 2 of 16 pixels x 4 samples, sent in two segments of 8 pixels
    tel_cam = np.array([0, 0, 0, 0, 0, 2], np.int32)
    cams = {2: (16, 4), 0: (8, 8)}
    s = np.arange(64, dtype=np.uint16) * 1000 + 7
    p1 = hand_packet(5, 1, 7, 0x0102030405060708, 1_700_000_000, 32768, 0, 8, 16, 4, s[:32])
    p2 = hand_packet(5, 2, 8, 0x0102030405060708, 1_700_000_000, 32768, 8, 8, 16, 4, s[32:])
    assert p1[:6] == bytes([0x08, 0x05, 0x40, 0x07, 0x00, 0x69])   # length 112 - 7 = 105
    f = ingest.parse_header(np.frombuffer(p1, np.uint8), 0)
    assert (f["apid"], f["seq_flags"], f["seq_count"], f["length"], f["event"]) == (5, 1, 7, 112, 0x0102030405060708)
    buf = np.frombuffer(p1 + p2, np.uint8)
    d = ingest.decode_stream(buf, tel_cam, cams)
    assert d["error"] == ingest.OK
    assert d["seg"].tolist() == [[32, 0, 8], [112 + 32, 8, 8]]
    assert d["img_seg"].tolist() == [0, 2] and d["img_tel"].tolist() == [5] and d["evt_off"].tolist() == [0, 1]
    assert d["evt_number"].tolist() == [0x0102030405060708]
    assert d["evt_time_ns"].tolist() == [1_700_000_000 * 10 ** 9 + 500_000_000]
    wave, off = ingest.gather(buf, d, [(16, 4)])
    np.testing.assert_array_equal(wave, s)


@pytest.fixture(scope="module")
def bundle():
    wl = synth.make_workload(2, 24)
    cams = {c: (cam.n_pix, cam.n_samples) for c, cam in wl.cams.items()}
    return wl, cams


@pytest.mark.parametrize("seg", [None, {1: 200, 2: 256, 3: 520}])
def test_round_trip_of_a_generated_bundle(bundle, seg):
    wl, cams = bundle
    t = 1_700_000_000_000_000_000 + 123_456_789 * np.arange(wl.n_evt)
    buf, plan = synth.encode_stream(wl, times_ns=t, seg_pixels=seg)
    if seg:
        assert len(plan["img"]) > 3 * wl.n_img
    d = ingest.decode_stream(buf, wl.tel_cam, cams)
    assert d["error"] == ingest.OK
    np.testing.assert_array_equal(d["img_tel"], wl.img_tel)
    np.testing.assert_array_equal(d["evt_off"], wl.evt_off)
    np.testing.assert_array_equal(d["evt_number"], 1000 + np.arange(wl.n_evt))
    # CUC fine time: 1/65536 s, floored when written and when read
    fine = ((t % 10 ** 9) * 65536) // 10 ** 9
    np.testing.assert_array_equal(d["evt_time_ns"], (t // 10 ** 9) * 10 ** 9 + (fine * 10 ** 9) // 65536)
    assert np.all(np.abs(d["evt_time_ns"] - t) < 15_259)
    wave, off = ingest.gather(buf, d, [cams[int(wl.tel_cam[x])] for x in d["img_tel"]])
    np.testing.assert_array_equal(wave, wl.wave)
    np.testing.assert_array_equal(off, wl.wave_off)
    assert d["n_samples"] == wl.wave.size


def test_equal_event_numbers_in_a_row_are_one_event(bundle):
    wl, cams = bundle
    ev = 1000 + np.arange(wl.n_evt)
    ev[5] = ev[4]
    buf, _ = synth.encode_stream(wl, event_numbers=ev)
    d = ingest.decode_stream(buf, wl.tel_cam, cams)
    assert len(d["evt_off"]) - 1 == wl.n_evt - 1
    assert d["evt_off"][5] == wl.evt_off[6]


def faults(wl, cams):
    """(name, stream, expected code, packet index) for one planted fault each."""
    buf, plan = synth.encode_stream(wl, seg_pixels={1: 400, 2: 512, 3: 520})
    off, size = plan["off"], plan["size"]
    k = 7                                  # a packet in the middle
    out = []
    b = buf.copy()
    b[off[k] + 40] ^= 0x20                 # a sample bit
    out.append(("crc", b, ingest.CRC, k))
    b = buf.copy()
    b[off[k] + 7] = 201                    # service type
    out.append(("service", b, ingest.HEADER, k))
    b = buf.copy()
    b[off[k]] = (b[off[k]] & 0xF8) | 0x07  # APID high bits: telescope 1792+
    out.append(("telescope", b, ingest.CAMERA, k))
    b = buf[: off[k] + size[k] // 2].copy()
    out.append(("truncated", b, ingest.FRAMING, k))
    b = buf.copy()
    b[off[k] + 5] = (int(b[off[k] + 5]) + 16) & 0xFF   # length 16 bytes longer
    out.append(("length", b, ingest.HEADER, k))
    # the image's segments swapped: the second one arrives first
    i = plan["img"][k]
    ks = np.nonzero(plan["img"] == i)[0]
    assert len(ks) >= 2
    a, c = ks[0], ks[1]
    b = np.concatenate([buf[:off[a]], buf[off[c]:off[c] + size[c]], buf[off[a]:off[a] + size[a]],
                        buf[off[c] + size[c]:]])
    out.append(("order", b, ingest.SEGMENT, a))
    # a middle segment dropped: the next one does not continue the image
    b = np.concatenate([buf[:off[c]], buf[off[c] + size[c]:]])
    out.append(("dropped", b, ingest.SEGMENT, c))
    # the stream ends inside an image
    b = buf[: off[c]].copy()
    out.append(("unfinished", b, ingest.SEGMENT, a))
    return buf, plan, out


def test_each_planted_fault_is_reported_at_its_packet(bundle):
    wl, cams = bundle
    buf, plan, cases = faults(wl, cams)
    assert ingest.decode_stream(buf, wl.tel_cam, cams)["error"] == ingest.OK
    for name, b, code, k in cases:
        d = ingest.decode_stream(b, wl.tel_cam, cams)
        assert (d["error"], d["error_offset"]) == (code, plan["off"][k]), name
        assert len(d["seg"]) == 0 and len(d["img_tel"]) == 0
    # without the CRC check the flipped bit passes and lands in the samples
    d = ingest.decode_stream(cases[0][1], wl.tel_cam, cams, verify_crc=False)
    assert d["error"] == ingest.OK


def test_capacities(bundle):
    wl, cams = bundle
    buf, plan = synth.encode_stream(wl)
    first_of = {int(i): int(np.nonzero(plan["img"] == i)[0][0]) for i in np.unique(plan["img"])}
    d = ingest.decode_stream(buf, wl.tel_cam, cams, img_cap=10)
    assert (d["error"], d["error_offset"]) == (ingest.CAPACITY, plan["off"][first_of[10]])
    d = ingest.decode_stream(buf, wl.tel_cam, cams, seg_cap=5)
    assert (d["error"], d["error_offset"]) == (ingest.CAPACITY, plan["off"][5])
    d = ingest.decode_stream(buf, wl.tel_cam, cams, evt_cap=3)
    assert (d["error"], d["error_offset"]) == (ingest.CAPACITY, plan["off"][first_of[int(wl.evt_off[3])]])
    d = ingest.decode_stream(buf, wl.tel_cam, cams, seg_cap=len(plan["img"]), img_cap=wl.n_img, evt_cap=wl.n_evt)
    assert d["error"] == ingest.OK
