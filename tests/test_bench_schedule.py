"""The serving benchmark's arrival schedule (host logic of bench.py, no GPU):
Poisson arrivals scaled to offer exactly the nominal rate, at least eight of
them however low the rate, and the burst."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

POOL = [849_000_000, 1_441_000_000, 921_000_000, 842_000_000, 3_118_000_000, 2_068_000_000]


@pytest.mark.parametrize("rate", [0.5, 2.0, 8.0])
def test_schedule_offers_exactly_the_nominal_rate(rate):
    s = bench.arrival_schedule(POOL, rate, 5.0, np.random.default_rng(3))
    t = np.array([dt for dt, _ in s], np.float64)
    total = sum(POOL[i] for _, i in s)
    assert np.all(np.diff(t) >= 0) and t[0] > 0
    assert total / (t[-1] / 1e9) / 1e9 == pytest.approx(rate, rel=1e-9)
    assert len(s) >= 8
    assert t[-1] / 1e9 >= 5.0 * 0.5            # about the requested span (the last gap is random)


def test_low_rates_still_get_eight_arrivals():
    s = bench.arrival_schedule(POOL, 0.1, 1.0, np.random.default_rng(4))
    assert len(s) >= 8


def test_gaps_are_exponential_in_shape():
    # many arrivals of one bundle size: the scaled gaps have mean bytes/rate and the
    # exponential's coefficient of variation of 1
    s = bench.arrival_schedule([10**9], 1.0, 2000.0, np.random.default_rng(5))
    t = np.array([dt for dt, _ in s], np.float64) / 1e9
    g = np.diff(np.concatenate([[0.0], t]))
    assert g.mean() == pytest.approx(1.0, rel=1e-6)
    assert g.std() / g.mean() == pytest.approx(1.0, abs=0.1)


def test_burst():
    s = bench.arrival_schedule(POOL, float("inf"), 5.0, np.random.default_rng(6))
    assert len(s) == 24 and all(dt == 0 for dt, _ in s)
    assert all(0 <= i < len(POOL) for _, i in s)


def test_rates_must_be_positive():
    for bad in (0.0, -1.0, float("nan")):
        with pytest.raises(ValueError):
            bench.arrival_schedule(POOL, bad, 5.0, np.random.default_rng(7))


def test_feed_bundles_are_contiguous_event_ranges_of_the_feed():
    """A serving bundle cut from the feed carries exactly its events' images and
    waveforms: tables rebased to its first sample and image, samples equal to the
    segments' own renderings."""
    import synth
    rng = np.random.default_rng(11)
    plans = [synth.make_workload(2, 12, seed=100 + k, telescopes=rng.choice(69, 25 + 10 * k, replace=False))
             for k in range(3)]
    feed = bench.feed_layout(plans)
    wave = np.concatenate([p.wave for p in plans])
    assert wave.size == feed["n_samples"]
    feed["wave"] = wave
    imgs = [(p, i) for p in plans for i in range(p.n_img)]
    evts = [(p, e) for p in plans for e in range(p.n_evt)]
    for b in bench.feed_bundles(feed, 20, rng, lo=3, hi=30):
        assert 3 <= b["n_evt"] <= 30 and b["evt"][0] == 0 and b["evt"][-1] == b["n_img"]
        w0 = (b["ptr"] - wave.ctypes.data) // 2
        e0 = int(np.searchsorted(feed["evt_off"], feed["wave_off"].searchsorted(w0), side="left"))
        i0 = int(feed["evt_off"][e0])
        assert b["off"][0] == 0 and b["n_wave"] == sum(
            imgs[i0 + k][0].image_wave(imgs[i0 + k][1]).size for k in range(b["n_img"]))
        for k in range(b["n_img"]):
            p, i = imgs[i0 + k]
            assert b["tel"][k] == p.img_tel[i]
            seg = p.image_wave(i).reshape(-1)
            np.testing.assert_array_equal(wave[w0 + b["off"][k]: w0 + b["off"][k] + seg.size], seg)
        for j in range(b["n_evt"]):
            p, e = evts[e0 + j]
            assert b["evt"][j + 1] - b["evt"][j] == p.evt_off[e + 1] - p.evt_off[e]
