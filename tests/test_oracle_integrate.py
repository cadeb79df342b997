"""Pins of the oracle's calibration + charge integration (signal extraction, Sec. 5).

The oracle is checked against things fixed independently of its code: brute
force over every window start, the charge a noiseless Gaussian pulse carries
(closed form), the centroid of a symmetric pulse, and pedestal-only statistics.
"""
import numpy as np
import pytest

import oracle

SIGMA = 1.5


def unit_pulse(t0, S):
    """Point-sampled Gaussian with sum over all integers equal to 1."""
    kk = np.arange(-200, 201)
    z = np.exp(-(kk ** 2) / (2 * SIGMA ** 2)).sum()
    k = np.arange(S)
    return np.exp(-((k - t0) ** 2) / (2 * SIGMA ** 2)) / z


def test_sliding_window_matches_brute_force_argmax():
    rng = np.random.default_rng(1)
    for S, W in [(40, 6), (30, 6), (25, 6), (16, 5), (7, 7), (6, 1)]:
        P = 300
        wave = rng.integers(0, 65536, size=(P, S), dtype=np.uint16)
        wave[:20] = rng.integers(0, 3, size=(20, S))       # many ties
        wave[20:25] = 1000                                 # all windows tie
        p16 = rng.integers(0, 16 * 1000, size=P).astype(np.int32)
        scale = rng.uniform(0.01, 1.0, size=P).astype(np.float32)
        q, t, ws, wsum = oracle.integrate(wave, p16, scale, True, 0, W)
        sums = np.lib.stride_tricks.sliding_window_view(wave.astype(np.int64), W, axis=1).sum(-1)
        exp_start = sums.argmax(1)          # numpy returns the first maximum
        np.testing.assert_array_equal(ws, exp_start)
        np.testing.assert_array_equal(wsum, sums.max(1))
        assert (ws[20:25] == 0).all()
        num = 16 * wsum - W * p16.astype(np.int64)
        np.testing.assert_array_equal(q, (num.astype(np.float32) * scale).astype(np.float32))


def test_fixed_window_sum():
    rng = np.random.default_rng(2)
    wave = rng.integers(0, 65536, size=(50, 16), dtype=np.uint16)
    p16 = np.full(50, 6400, np.int32)
    scale = np.ones(50, np.float32)
    q, t, ws, wsum = oracle.integrate(wave, p16, scale, False, 4, 5)
    np.testing.assert_array_equal(wsum, wave[:, 4:9].astype(np.int64).sum(1))
    assert (ws == 4).all()


@pytest.mark.parametrize("sliding,start,W,S,t0", [(False, 4, 5, 16, 6.0), (True, 0, 6, 40, 6.0),
                                                  (True, 0, 6, 40, 23.0), (True, 0, 6, 25, 6.0)])
@pytest.mark.parametrize("Q", [30.0, 500.0, 5000.0])
def test_noiseless_pulse_integrates_to_its_charge(sliding, start, W, S, t0, Q):
    """A pulse of Q pe on a pedestal gives q = Q up to ADC rounding (closed form)."""
    rng = np.random.default_rng(3)
    P = 64
    ped = 400 + rng.normal(0, 5, P)
    gain = 8 * (1 + rng.normal(0, 0.05, P))
    g = unit_pulse(t0, S)
    wave = np.floor(ped[:, None] + gain[:, None] * Q * g[None, :] + 0.5).astype(np.uint16)
    # window containment of an on-grid pulse, computed here from the pulse itself
    if sliding:
        kk = np.arange(-40, 41)
        gg = np.exp(-(kk ** 2) / (2 * SIGMA ** 2)) / np.exp(-(np.arange(-200, 201) ** 2) / (2 * SIGMA ** 2)).sum()
        f = max(gg[(kk >= s) & (kk < s + W)].sum() for s in range(-W, 1))
    else:
        f = g[start:start + W].sum()
    p16 = np.round(16 * ped).astype(np.int32)
    scale = (1.0 / (16 * gain * f)).astype(np.float32)
    q, t, ws, _ = oracle.integrate(wave, p16, scale, sliding, start, W)
    # ADC rounding: |err| <= W * 0.5 ADC; pedestal quantisation W/32 ADC
    bound = (W * 0.5 + W / 32.0) / (gain * f) + 1e-6 * Q
    assert np.all(np.abs(q - Q) <= bound), (q - Q, bound)
    if sliding:
        assert np.all(ws == int(t0) - W // 2), ws      # lowest of the two tied windows


def test_window_fraction_of_generator_matches_pulse():
    import synth
    g = unit_pulse(6.0, 16)
    assert synth.window_fraction(False, 4, 5) == pytest.approx(g[4:9].sum(), rel=1e-12)
    assert synth.window_fraction(False, 4, 5) == pytest.approx(0.910572, abs=1e-6)
    assert synth.window_fraction(True, 0, 6) == pytest.approx(0.946566, abs=1e-6)


def test_symmetric_pulse_time_is_its_peak():
    S = 16
    g = unit_pulse(6.0, S)
    wave = np.floor(400.0 + 8.0 * 1000 * g + 0.5).astype(np.uint16)[None, :]
    q, t, ws, _ = oracle.integrate(wave, np.array([6400], np.int32), np.ones(1, np.float32), False, 4, 5)
    assert t[0] == 6.0


@pytest.mark.parametrize("t0", [19.3, 20.0, 20.45, 21.7])
def test_pulse_time_is_window_centroid(t0):
    """t is the pedestal-subtracted sample centroid of the chosen window."""
    S, W = 40, 6
    g = unit_pulse(t0, S)
    amp = 8.0 * 2000 * g
    wave = np.floor(400.0 + amp + 0.5).astype(np.uint16)[None, :]
    q, t, ws, _ = oracle.integrate(wave, np.array([6400], np.int32), np.ones(1, np.float32), True, 0, W)
    s = int(ws[0])
    k = np.arange(s, s + W)
    centroid = (k * amp[k]).sum() / amp[k].sum()
    assert abs(t[0] - centroid) < 2e-3
    assert s <= t0 <= s + W - 1


def test_nonpositive_numerator_gives_window_centre():
    wave = np.full((1, 16), 390, np.uint16)
    q, t, ws, _ = oracle.integrate(wave, np.array([6400], np.int32), np.ones(1, np.float32), False, 4, 5)
    assert q[0] < 0 and t[0] == 4 + 2.0


def test_pedestal_only_statistics():
    """Pedestal + N(0,2) noise, fixed window: q ~ N(0, sqrt(W)*2/(gain f))."""
    rng = np.random.default_rng(5)
    P, S, W = 20000, 16, 5
    ped, gain = 400.3, 8.0
    wave = np.floor(ped + rng.normal(0, 2, (P, S)) + 0.5).astype(np.uint16)
    f = 0.910572
    q, t, _, _ = oracle.integrate(wave, np.full(P, round(16 * ped), np.int32),
                                  np.full(P, 1 / (16 * gain * f), np.float32), False, 4, W)
    sd = np.sqrt(W * (4 + 1 / 12)) / (gain * f)
    assert abs(q.mean()) < 5 * sd / np.sqrt(P) + W * (round(16 * ped) / 16 - ped) / (gain * f) + 1e-3
    assert q.std() == pytest.approx(sd, rel=0.03)


def test_bad_arguments_rejected():
    wave = np.zeros((2, 8), np.uint16)
    with pytest.raises(ValueError):
        oracle.integrate(wave, np.zeros(2, np.int32), np.ones(2, np.float32), True, 0, 9)
    with pytest.raises(ValueError):
        oracle.integrate(wave, np.zeros(2, np.int32), np.ones(2, np.float32), False, 5, 4)


# ---------------------------------------------------------------------------- digital-filter-style charge
def test_filter_with_unit_weights_is_the_window_sum():
    rng = np.random.default_rng(21)
    P, S, W = 64, 30, 6
    wave = rng.integers(300, 3000, size=(P, S)).astype(np.uint16)
    p16 = rng.integers(16 * 380, 16 * 420, size=P).astype(np.int32)
    scale = rng.uniform(0.004, 0.01, P).astype(np.float32)
    q0, t0, s0, _ = oracle.integrate(wave, p16, scale, True, 0, W)
    q1, t1, s1, _ = oracle.integrate(wave, p16, scale, True, 0, W, weights=[1] * W)
    np.testing.assert_array_equal(q0.view(np.uint32), q1.view(np.uint32))
    np.testing.assert_array_equal(t0, t1)
    np.testing.assert_array_equal(s0, s1)


def test_filter_is_linear_in_its_weights_and_blind_to_the_pedestal():
    """With scale = 1/16 and small integers every charge is exact, so charges of
    summed weights add exactly; a waveform at the pedestal gives zero for any
    weights; a single non-zero sample inside the window picks one weight."""
    rng = np.random.default_rng(22)
    P, S, W = 40, 25, 6
    wave = rng.integers(0, 200, size=(P, S)).astype(np.uint16)
    p16 = (16 * rng.integers(0, 50, size=P)).astype(np.int32)
    scale = np.full(P, 1.0 / 16.0, np.float32)
    c1 = np.array([1, 3, 5, 4, 2, 1])
    c2 = np.array([-1, 0, 2, 7, 0, 3])
    qa, _, sa, _ = oracle.integrate(wave, p16, scale, True, 0, W, weights=c1)
    qb, _, sb, _ = oracle.integrate(wave, p16, scale, True, 0, W, weights=c2)
    qc, _, sc, _ = oracle.integrate(wave, p16, scale, True, 0, W, weights=c1 + c2)
    assert (sa == sb).all() and (sa == sc).all()                 # the window does not depend on the weights
    np.testing.assert_array_equal(qc, qa + qb)
    ped = (p16 // 16).astype(np.uint16)
    flat = np.repeat(ped[:, None], S, axis=1)
    qp, _, _, _ = oracle.integrate(flat, p16, scale, True, 0, W, weights=c1)
    assert (qp == 0).all()
    for j in range(W):
        # the only signal at sample j < W: every window with start <= j ties, the
        # first (start 0) is chosen, so the sample meets weight j
        one = np.zeros((1, S), np.uint16)
        one[0, j] = 100
        q, _, st, _ = oracle.integrate(one, np.zeros(1, np.int32), np.ones(1, np.float32), True, 0, W,
                                       weights=c1)
        assert st[0] == 0 and q[0] == 16 * 100 * c1[j]
