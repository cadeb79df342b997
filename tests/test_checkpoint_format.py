"""The surrogate's checkpoint file (host side): a round trip keeps every value
and the step count; files of another kind, another version or a wrong length
are refused."""
import numpy as np
import pytest

from paper_1307_6489_gb300 import train


def test_round_trip_keeps_every_value(tmp_path):
    rng = np.random.default_rng(3)
    p, m, v = (rng.standard_normal(1001).astype(np.float32) for _ in range(3))
    codes = np.array([0.0, 0.57, -1.1], np.float32)
    f = tmp_path / "c.bin"
    train.write_checkpoint(str(f), p, m, v, 12345, codes)
    p2, m2, v2, step, codes2 = train.read_checkpoint(str(f))
    assert step == 12345
    for a, b in [(p, p2), (m, m2), (v, v2)]:
        np.testing.assert_array_equal(a.view(np.uint32), b.view(np.uint32))
    np.testing.assert_array_equal(codes2[:3], codes)
    assert (codes2[3:] == 0).all() and len(codes2) == 16
    assert f.stat().st_size == 8 + 8 + 8 + 64 + 3 * 4 * 1001


@pytest.mark.parametrize("damage", ["magic", "version", "truncated", "padded"])
def test_damaged_files_are_refused(tmp_path, damage):
    f = tmp_path / "c.bin"
    train.write_checkpoint(str(f), np.ones(10), np.ones(10), np.ones(10), 1, [0])
    raw = bytearray(f.read_bytes())
    if damage == "magic":
        raw[0:8] = b"NOTACKPT"
    elif damage == "version":
        raw[8:12] = np.array([2], "<u4").tobytes()
    elif damage == "truncated":
        raw = raw[:-4]
    else:
        raw += b"\0\0\0\0"
    f.write_bytes(bytes(raw))
    with pytest.raises(ValueError):
        train.read_checkpoint(str(f))
