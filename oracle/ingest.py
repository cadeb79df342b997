"""DL0 byte-stream decoder oracle -- TEST INFRASTRUCTURE ONLY (imported by
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg).

Sec. 5 has the telescope data travel as a byte stream formatted like satellite
telemetry (CCSDS space packets with a PUS secondary header) and names no packet
contents. The layout read here is the one the library documents: a 32-byte
header (big-endian fields), the samples of a pixel range of one image, 14 bytes
of padding and a CRC-16-CCITT. This decoder walks the stream one packet at a
time from byte 0, checks every packet in a fixed order and stops at the first
packet with a problem:

  framing   fewer than 48 bytes left, or a length that is not a multiple of 16,
            below 48, above 65536 or past the end
  header    a fixed field (version, type, secondary-header flag, PUS version,
            service, subservice) is wrong; the length disagrees with 48 + 2 n S;
            n = 0, n S not a multiple of 8, first + n past the image; the
            sequence flags disagree with the segment's place in the image
  camera    unknown telescope, or pixels/samples differ from its camera
  segment   a packet does not continue the previous packet's unfinished image
            (same telescope and event number, next pixel), or starts an image
            at a pixel other than 0, or the stream ends inside an image
  crc       the packet error control field differs from the CRC (if asked)
  capacity  more segments, images or events than the capacities
"""
from __future__ import annotations

import ctypes

import numpy as np

OK, FRAMING, HEADER, CAMERA, SEGMENT, CRC, CAPACITY = range(7)


def crc16(data) -> int:
    """CRC-16-CCITT of a byte string by its bit-serial definition (oracle.c)."""
    from . import _L, _p
    a = np.ascontiguousarray(np.frombuffer(bytes(data), np.uint8) if not isinstance(data, np.ndarray) else data,
                             np.uint8)
    lib = _L()
    lib.or_crc16.restype = ctypes.c_uint32
    lib.or_crc16.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    return int(lib.or_crc16(_p(a), a.size))


def _be(b, i, n):
    v = 0
    for k in range(n):
        v = (v << 8) | int(b[i + k])
    return v


def parse_header(buf, pos):
    """The fields of the packet header at byte pos (no checks)."""
    h = buf[pos:pos + 32]
    w0, w1 = _be(h, 0, 2), _be(h, 2, 2)
    return dict(version=w0 >> 13, type=(w0 >> 12) & 1, sec_hdr=(w0 >> 11) & 1, apid=w0 & 0x7FF,
                seq_flags=w1 >> 14, seq_count=w1 & 0x3FFF, length=_be(h, 4, 2) + 7, pus=int(h[6]),
                service=int(h[7]), subservice=int(h[8]), dest=int(h[9]), sec=_be(h, 10, 4), fine=_be(h, 14, 2),
                event=_be(h, 16, 8), first=_be(h, 24, 2), n=_be(h, 26, 2), P=_be(h, 28, 2), S=_be(h, 30, 2))


def _check_packet(buf, pos, n_bytes, tel_cam, cams):
    """The first failing check of the packet at pos among framing, header and
    camera, and its fields."""
    if n_bytes - pos < 48:
        return FRAMING, None
    f = parse_header(buf, pos)
    if f["version"] != 0 or f["type"] != 0 or f["sec_hdr"] != 1 or f["pus"] != 0x10 or f["service"] != 200 \
            or f["subservice"] != 1:
        return HEADER, f
    L = f["length"]
    if L % 16 or L < 48 or L > 65536 or pos + L > n_bytes:
        return FRAMING, f
    n, S, P, first = f["n"], f["S"], f["P"], f["first"]
    if 48 + 2 * n * S != L or n == 0 or (n * S) % 8 or first + n > P:
        return HEADER, f
    whole, starts, ends = first == 0 and first + n == P, first == 0, first + n == P
    want = 3 if whole else (1 if starts else (2 if ends else 0))
    if f["seq_flags"] != want:
        return HEADER, f
    t = f["apid"]
    if t >= len(tel_cam) or int(tel_cam[t]) not in cams or cams[int(tel_cam[t])] != (P, S):
        return CAMERA, f
    return OK, f


def decode_stream(buf, tel_cam, cams, verify_crc=True, seg_cap=1 << 62, img_cap=1 << 62, evt_cap=1 << 62):
    """Directory of a byte stream. cams: {camera id: (pixels, samples)}.
    Returns dict(seg=(n, 3) int64 [offset of the first sample, first pixel,
    pixels], img_seg, img_tel, evt_off, evt_number, evt_time_ns, n_samples,
    error, error_offset); on an error the directory is empty."""
    buf = np.ascontiguousarray(buf, np.uint8)
    n_bytes = buf.size
    seg, img_seg, img_tel, evt_off, evnum, evtime = [], [], [], [], [], []
    n_samples = 0
    prev = None
    pos = 0

    def fail(code, at):
        return dict(seg=np.zeros((0, 3), np.int64), img_seg=np.zeros(0, np.int32), img_tel=np.zeros(0, np.int32),
                    evt_off=np.zeros(0, np.int32), evt_number=np.zeros(0, np.uint64),
                    evt_time_ns=np.zeros(0, np.int64), n_samples=0, error=code, error_offset=at)

    while pos < n_bytes:
        code, f = _check_packet(buf, pos, n_bytes, tel_cam, cams)
        if code != OK:
            return fail(code, pos)
        open_image = prev is not None and prev["first"] + prev["n"] < prev["P"]
        if open_image:
            if f["apid"] != prev["apid"] or f["event"] != prev["event"] or f["first"] != prev["first"] + prev["n"]:
                return fail(SEGMENT, pos)
        elif f["first"] != 0:
            return fail(SEGMENT, pos)
        L = f["length"]
        if verify_crc and crc16(buf[pos:pos + L - 2]) != _be(buf, pos + L - 2, 2):
            return fail(CRC, pos)
        new_image = f["first"] == 0
        new_event = new_image and (prev is None or f["event"] != prev["event"])
        n_img_next = len(img_tel) + (1 if new_image else 0)
        n_evt_next = len(evnum) + (1 if new_event else 0)
        if len(seg) + 1 > seg_cap or n_img_next > img_cap or n_evt_next > evt_cap:
            return fail(CAPACITY, pos)
        if new_event:
            evt_off.append(len(img_tel))
            evnum.append(f["event"])
            evtime.append(f["sec"] * 1_000_000_000 + (f["fine"] * 1_000_000_000) // 65536)
        if new_image:
            img_seg.append(len(seg))
            img_tel.append(f["apid"])
            n_samples += f["P"] * f["S"]
        seg.append((pos + 32, f["first"], f["n"]))
        prev = f
        pos += L
    if prev is not None and prev["first"] + prev["n"] < prev["P"]:
        return fail(SEGMENT, pos - prev["length"])
    img_seg.append(len(seg))
    evt_off.append(len(img_tel))
    return dict(seg=np.array(seg, np.int64).reshape(-1, 3), img_seg=np.array(img_seg, np.int32),
                img_tel=np.array(img_tel, np.int32), evt_off=np.array(evt_off, np.int32),
                evt_number=np.array(evnum, np.uint64), evt_time_ns=np.array(evtime, np.int64),
                n_samples=n_samples, error=OK, error_offset=-1)


def gather(buf, directory, cams_of_img):
    """The contiguous bundle (uint16 samples, wave_off) the directory describes.
    cams_of_img[i] = (pixels, samples) of image i."""
    buf = np.ascontiguousarray(buf, np.uint8)
    sizes = np.array([P * S for P, S in cams_of_img], np.int64)
    wave_off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    wave = np.zeros(int(sizes.sum()), np.uint16)
    seg, img_seg = directory["seg"], directory["img_seg"]
    for i in range(len(sizes)):
        S = cams_of_img[i][1]
        for k in range(img_seg[i], img_seg[i + 1]):
            off, first, n = (int(v) for v in seg[k])
            w = buf[off:off + 2 * n * S].view("<u2")
            wave[wave_off[i] + first * S: wave_off[i] + (first + n) * S] = w
    return wave, wave_off
