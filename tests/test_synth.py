"""The seeded input generator: counter-based RNG, determinism, distributions."""
import numpy as np
import pytest

import synth


def test_philox_known_answers():
    """Known-answer vectors of Philox-4x32-10 (Salmon et al. 2011, Random123 KAT)."""
    cases = [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ]
    lib = synth._L()
    for ctr, key, want in cases:
        c = np.array(ctr, np.uint32)
        k = np.array(key, np.uint32)
        o = np.zeros(4, np.uint32)
        lib.synth_philox_block(synth._p(c), synth._p(k), synth._p(o))
        assert [int(x) for x in o] == want


def test_uniform_normal_poisson_moments():
    lib = synth._L()
    n = 200000
    u = np.zeros(n)
    lib.synth_test_uniforms(1, n, synth._p(u))
    assert 0 < u.min() and u.max() < 1
    assert u.mean() == pytest.approx(0.5, abs=0.005) and u.var() == pytest.approx(1 / 12, rel=0.02)
    z = np.zeros(n)
    lib.synth_test_normals(2, n, synth._p(z))
    assert z.mean() == pytest.approx(0, abs=0.01) and z.std() == pytest.approx(1, rel=0.01)
    for mu in [0.3, 4.0, 9.99, 10.0, 37.5, 2000.0]:
        k = np.zeros(n, np.int64)
        lib.synth_test_poisson(3, mu, n, synth._p(k))
        assert k.min() >= 0
        assert k.mean() == pytest.approx(mu, rel=0.02, abs=0.01)
        assert k.var() == pytest.approx(mu, rel=0.03, abs=0.01)


def test_render_is_deterministic_and_thread_independent():
    a = synth.make_workload(2, 30, threads=1)
    b = synth.make_workload(2, 30, threads=5)
    np.testing.assert_array_equal(a.wave, b.wave)
    np.testing.assert_array_equal(a.evt_off, b.evt_off)
    c = synth.make_workload(2, 30, seed=a.seed + 100)
    assert not np.array_equal(a.evt_off, c.evt_off) or not np.array_equal(a.wave[:1000], c.wave[:1000])


def test_layout_and_offsets():
    wl = synth.make_workload(2, 200)
    m = np.diff(wl.evt_off)
    assert m.min() >= 2 and m.max() <= 40
    assert (wl.wave_off * 2 % 16 == 0).all()                 # every image starts 16-byte aligned
    tel_cam, tel_xy = synth.array_layout()
    assert len(tel_cam) == 69 and np.bincount(tel_cam).tolist() == [0, 4, 15, 50]
    for e in range(wl.n_evt):                                # telescopes ascending within an event
        t = wl.img_tel[wl.evt_off[e]:wl.evt_off[e + 1]]
        assert (np.diff(t) > 0).all()
    assert wl.wave.size == wl.n_samples_total
    E = wl.truth[:, 0]
    assert 0.03 <= E.min() and E.max() <= 100


def test_pedestal_only_pixels_statistics():
    wl = synth.make_workload(0, 400)
    w = wl.wave.reshape(400, 256, 16).astype(np.float64)
    ped = wl.ped.reshape(256)
    # pixels far from the ellipse: residual = NSB (0.3 pe * 8 ADC spread over 16 samples) + N(0, 2) noise
    d = np.hypot(wl.cams[0].xy[None, :, 0] - wl.ell[:, 0, 1][:, None],
                 wl.cams[0].xy[None, :, 1] - wl.ell[:, 0, 2][:, None])
    res = (w - ped[None, :, None])[d > 1.2]
    assert 0.0 < res.mean() < 0.3
    assert 2.0 < res.std() < 3.0
    assert (wl.p16 == np.round(16 * wl.ped)).all()
    f = synth.window_fraction(False, 4, 5)
    np.testing.assert_array_equal(wl.scale, (1.0 / (16 * wl.gain * f)).astype(np.float32))


def test_sub_array_workload():
    sub = [0, 1, 2, 3, 4, 5, 6, 20, 21, 22]
    wl = synth.make_workload(2, 50, telescopes=sub)
    assert set(np.unique(wl.img_tel)) <= set(sub)
    assert len(wl.tel_cam) == 69 and np.diff(wl.evt_off).min() >= 2
