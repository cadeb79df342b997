"""The neighbour-peak window of the oracle (a pixel integrates its own samples
in the sliding window of the brightest pixel of its closed neighbourhood)
pinned to what its definition fixes: it reduces to the sliding window without
neighbours or for the brightest pixel; a dim pixel next to a bright pulse
integrates its own pulse in closed form where the sliding window would chase a
noise spike; ties; the order of the neighbour list; the choice is always the
neighbourhood's brightest window; and on pure noise next to bright pixels the
charge is unbiased where the sliding window is biased upwards."""
import numpy as np
import pytest

import oracle

SIGMA = 1.2


def unit_pulse(t0, S):
    k = np.arange(S)
    g = np.exp(-((k - t0) ** 2) / (2 * SIGMA ** 2))
    return g / np.exp(-(np.arange(-200, 201) ** 2) / (2 * SIGMA ** 2)).sum()


def ring_neighbours(P, K=6):
    """Pixel p's neighbours: p +- 1, +- 2, +- 3 on a ring (a stand-in lattice)."""
    nb = np.full((P, K), -1, np.int16)
    for p in range(P):
        for j, d in enumerate([1, -1, 2, -2, 3, -3][:K]):
            nb[p, j] = (p + d) % P
    return nb


def test_without_neighbours_it_is_the_sliding_window():
    rng = np.random.default_rng(1)
    P, S, W = 50, 30, 6
    wave = rng.integers(300, 700, (P, S)).astype(np.uint16)
    p16 = rng.integers(300 * 16, 500 * 16, P).astype(np.int32)
    scale = rng.uniform(0.005, 0.02, P).astype(np.float32)
    q0, t0, s0, _ = oracle.integrate(wave, p16, scale, True, 0, W)
    q1, t1, s1 = oracle.integrate_nbpeak(wave, p16, scale, np.full((P, 6), -1, np.int16), W)
    np.testing.assert_array_equal(q0, q1)
    np.testing.assert_array_equal(t0, t1)
    np.testing.assert_array_equal(s0, s1)


def test_the_brightest_pixel_keeps_its_window_and_the_choice_is_the_neighbourhood_peak():
    rng = np.random.default_rng(2)
    P, S, W = 80, 40, 6
    wave = rng.integers(380, 460, (P, S)).astype(np.uint16)
    for p in rng.choice(P, 12, replace=False):
        t = rng.integers(3, S - 4)
        wave[p, t - 1:t + 2] += np.uint16(rng.integers(50, 600))
    p16 = np.full(P, 400 * 16, np.int32)
    scale = rng.uniform(0.008, 0.012, P).astype(np.float32)
    nb = ring_neighbours(P)
    q0, _, s0, _ = oracle.integrate(wave, p16, scale, True, 0, W)
    q, t, s = oracle.integrate_nbpeak(wave, p16, scale, nb, W)
    for p in range(P):
        hood = [p] + [int(n) for n in nb[p] if n >= 0]
        best = max(q0[n] for n in hood)
        assert s[p] == min(s0[n] for n in hood if q0[n] == best)
        if q0[p] > max(q0[n] for n in hood[1:]):
            assert s[p] == s0[p]
        # the charge is the pixel's own flat sum at the chosen start, calibrated once
        num = 16 * int(wave[p, s[p]:s[p] + W].astype(np.int64).sum()) - W * int(p16[p])
        assert q[p] == np.float32(np.float32(num) * scale[p])


def test_a_dim_pixel_next_to_a_bright_pulse_integrates_its_own_pulse():
    """Pixel 1 carries a 30 pe pulse at the same time as its 2000 pe neighbour 0
    and a 120 pe noise spike 15 samples later. The sliding window takes the
    spike; the neighbour-peak window takes the pulse: charge 30 pe within ADC
    rounding (closed form)."""
    S, W, t_pulse, t_spike = 40, 6, 10.0, 25.0
    gain = 8.0
    g, h = unit_pulse(t_pulse, S), unit_pulse(t_spike, S)
    amp = np.stack([gain * 2000 * g, gain * 30 * g + gain * 120 * h, np.zeros(S)])
    wave = np.floor(400.0 + amp + 0.5).astype(np.uint16)
    kk = np.arange(-40, 41)
    gg = np.exp(-(kk ** 2) / (2 * SIGMA ** 2)) / np.exp(-(np.arange(-200, 201) ** 2) / (2 * SIGMA ** 2)).sum()
    f = max(gg[(kk >= s) & (kk < s + W)].sum() for s in range(-W, 1))
    p16 = np.full(3, 400 * 16, np.int32)
    scale = np.full(3, 1.0 / (16 * gain * f), np.float32)
    nb = np.array([[1, 2], [0, -1], [0, -1]], np.int16)
    qs, _, ss, _ = oracle.integrate(wave, p16, scale, True, 0, W)
    q, t, s = oracle.integrate_nbpeak(wave, p16, scale, nb, W)
    assert ss[1] > t_pulse + 5 and s[1] == ss[0]             # sliding chased the spike; nbpeak did not
    bound = (W * 0.5) / (gain * f) + 1e-6
    assert abs(q[1] - 30.0) <= bound, q[1]
    assert abs(qs[1] - 120.0) <= bound + 1.0                  # the spike's charge
    assert abs(q[0] - 2000.0) <= bound + 2000 * 1e-6          # the bright pixel keeps its own window
    assert s[2] == s[0] and abs(q[2]) <= bound                # an empty pixel next to the bright one: ~0


def test_ties_and_neighbour_order():
    S, W = 20, 4
    wave = np.full((4, S), 400, np.uint16)
    wave[1, 3:7] += 100          # neighbours 1 and 2 equally bright, 2 earlier
    wave[2, 1:5] += 100
    p16 = np.full(4, 400 * 16, np.int32)
    scale = np.ones(4, np.float32)
    for order in ([1, 2, -1], [2, 1, -1], [-1, 2, 1]):
        nb = np.array([order, [0, -1, -1], [0, -1, -1], [-1, -1, -1]], np.int16)
        q, t, s = oracle.integrate_nbpeak(wave, p16, scale, nb, W)
        assert s[0] == 1                 # equal charges: the earlier window
        assert s[3] == 0                 # no neighbours, flat: its own first window
    rng = np.random.default_rng(4)
    P = 60
    wave = rng.integers(350, 900, (P, 30)).astype(np.uint16)
    p16 = np.full(P, 400 * 16, np.int32)
    scale = rng.uniform(0.5, 1.5, P).astype(np.float32)
    nb = ring_neighbours(P)
    a = oracle.integrate_nbpeak(wave, p16, scale, nb, 6)
    b = oracle.integrate_nbpeak(wave, p16, scale, nb[:, rng.permutation(6)], 6)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_noise_next_to_bright_pixels_is_unbiased():
    """Pure-noise pixels: the sliding window's maximum over windows is biased
    upwards; a window placed by a bright neighbour is not."""
    rng = np.random.default_rng(5)
    n, S, W = 4000, 30, 6
    P = 2 * n
    wave = np.empty((P, S), np.uint16)
    wave[0::2] = np.floor(400 + rng.normal(0, 6, (n, S)) + 0.5).astype(np.uint16)       # noise
    tb = rng.integers(5, S - 6, n)
    bright = np.floor(400 + rng.normal(0, 6, (n, S)) + 0.5)
    for i in range(n):
        bright[i, tb[i] - 1:tb[i] + 2] += 800
    wave[1::2] = bright.astype(np.uint16)
    p16 = np.full(P, 400 * 16, np.int32)
    scale = np.full(P, 1.0 / 16, np.float32)
    nb = np.full((P, 1), -1, np.int16)
    nb[0::2, 0] = np.arange(1, P, 2)             # each noise pixel has one bright neighbour
    qs, _, _, _ = oracle.integrate(wave, p16, scale, True, 0, W)
    q, _, s = oracle.integrate_nbpeak(wave, p16, scale, nb, W)
    noise_sd = 6 * np.sqrt(W)
    assert abs(np.mean(q[0::2])) < 4 * noise_sd / np.sqrt(n)
    assert np.mean(qs[0::2]) > 1.0 * noise_sd
    assert np.std(q[0::2]) == pytest.approx(noise_sd, rel=0.1)
