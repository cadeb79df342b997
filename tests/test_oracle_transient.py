"""The transient-search oracle (on/off significance per sky bin on several
timescales) pinned to what the statistics and geometry fix: the Li & Ma
significance against a numerical Poisson likelihood-ratio test, its exact
special cases and Gaussian limit, the disk sum against a library convolution,
the window selection against a direct count, and a planted flare."""
import numpy as np
import pytest

import oracle

scipy = pytest.importorskip("scipy")
from scipy import ndimage, optimize, stats  # noqa: E402


def lr_significance(n_on, n_off, alpha):
    """sqrt(-2 ln lambda) of the Poisson on/off test, by numerical maximisation:
    free model mu_on = n_on, mu_off = n_off; null model mu_on = alpha b,
    mu_off = b with b fitted."""
    def nll0(b):
        return -(stats.poisson.logpmf(n_on, alpha * b) + stats.poisson.logpmf(n_off, b))
    hi = 10.0 * (n_on + n_off + 1.0) / min(alpha, 1.0)
    b = optimize.minimize_scalar(nll0, bounds=(1e-12, hi), method="bounded",
                                 options={"xatol": 1e-12 * hi, "maxiter": 2000}).x
    ll1 = stats.poisson.logpmf(n_on, max(n_on, 1e-300)) + stats.poisson.logpmf(n_off, max(n_off, 1e-300))
    s = np.sqrt(max(2.0 * (ll1 + nll0(b)), 0.0))
    return s if n_on >= alpha * n_off else -s


@pytest.mark.parametrize("n_on,n_off,alpha", [(12, 40, 0.1), (5, 60, 0.2), (40, 40, 0.5), (3, 90, 1 / 30.0),
                                               (300, 2000, 0.1), (0, 25, 0.25), (17, 0, 0.4), (1, 3, 1.0)])
def test_li_ma_equals_the_likelihood_ratio_test(n_on, n_off, alpha):
    assert oracle.li_ma(n_on, n_off, alpha) == pytest.approx(lr_significance(n_on, n_off, alpha), abs=2e-5)


def test_li_ma_special_cases():
    # no excess: n_on = alpha n_off gives exactly 0
    for n_off, alpha in [(40, 0.25), (90, 1 / 3), (7, 1.0), (60, 0.5)]:
        assert abs(float(oracle.li_ma(alpha * n_off, n_off, alpha))) < 1e-6
    # no off counts: the sum reduces to sqrt(2 n_on ln((1 + alpha) / alpha))
    for n_on, alpha in [(9, 0.1), (1, 1.0), (250, 0.05)]:
        assert float(oracle.li_ma(n_on, 0, alpha)) == pytest.approx(np.sqrt(2 * n_on * np.log((1 + alpha) / alpha)))
    # deficits are negative, excesses positive, nothing at all is zero
    assert oracle.li_ma(2, 100, 0.1) < 0 < oracle.li_ma(30, 100, 0.1)
    assert oracle.li_ma(0, 0, 0.3) == 0
    # grows with the excess at fixed background
    s = oracle.li_ma(np.arange(10, 60), 200, 0.1)
    assert (np.diff(s) > 0).all()


def test_li_ma_gaussian_limit():
    """For large counts the significance approaches the excess over its
    standard deviation sqrt(alpha (n_on + n_off)) (Li & Ma Eq. 9's regime)."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        alpha = rng.uniform(0.05, 1.0)
        n_off = rng.uniform(2e5, 1e6)
        n_on = alpha * n_off * (1 + rng.uniform(-0.01, 0.01))
        gauss = (n_on - alpha * n_off) / np.sqrt(alpha * (n_on + n_off))
        assert float(oracle.li_ma(n_on, n_off, alpha)) == pytest.approx(gauss, rel=0.03, abs=0.02)


@pytest.mark.parametrize("radius", [0, 1, 3, 5, 12])
def test_disk_sum_equals_a_convolution_with_a_disk(radius):
    rng = np.random.default_rng(radius)
    m = rng.integers(0, 5, size=(oracle.SKY_N, oracle.SKY_N))
    yy, xx = np.mgrid[-radius:radius + 1, -radius:radius + 1]
    disk = (xx * xx + yy * yy <= radius * radius).astype(np.int64)
    ref = ndimage.convolve(m, disk, mode="constant", cval=0)
    np.testing.assert_array_equal(oracle.disk_sum(m, radius), ref)


def test_windows_select_the_right_seconds_and_minutes():
    rng = np.random.default_rng(5)
    n = 4000
    now = 100_000
    sec = now - rng.integers(0, 3600, size=n)
    x = rng.uniform(-2.6, 2.6, n).astype(np.float32)
    y = rng.uniform(-2.6, 2.6, n).astype(np.float32)
    has = rng.uniform(size=n) < 0.95
    ix, iy = oracle.sky_bin(x), oracle.sky_bin(y)
    for on_s, off_s in [(1, 5), (5, 25), (10, 20), (60, 600), (300, 3300), (1800, 1800)]:
        _, d_on, d_off, alpha = oracle.transient_maps(x, y, has, sec, now, (on_s, off_s), 0)
        if on_s + off_s <= 30:
            t, nw, on, off = sec, now, on_s, off_s
        else:
            t, nw, on, off = sec // 60, now // 60, on_s // 60, off_s // 60
        n_on = sum(1 for k in range(n) if has[k] and ix[k] >= 0 and iy[k] >= 0 and nw - on < t[k] <= nw)
        n_off = sum(1 for k in range(n) if has[k] and ix[k] >= 0 and iy[k] >= 0 and nw - on - off < t[k] <= nw - on)
        assert d_on.sum() == n_on and d_off.sum() == n_off and alpha == on_s / off_s
    with pytest.raises(ValueError):
        oracle.transient_maps(x, y, has, sec, now, (20, 20), 0)       # 40 s: not whole minutes
    with pytest.raises(ValueError):
        oracle.transient_maps(x, y, has, sec, now, (60, 3600), 0)     # longer than the minute ring


def test_a_planted_flare_is_found_where_it_was_planted():
    rng = np.random.default_rng(11)
    now = 50_000
    # background: 20 events/s spread over the map for 30 s; a flare of 60 events
    # within 0.05 deg of (0.31, -0.47) deg in the last 5 s
    nb = 20 * 30
    xb, yb = rng.uniform(-2.5, 2.5, nb), rng.uniform(-2.5, 2.5, nb)
    sb = now - rng.integers(0, 30, nb)
    nf = 60
    xf, yf = 0.31 + rng.normal(0, 0.02, nf), -0.47 + rng.normal(0, 0.02, nf)
    sf = now - rng.integers(0, 5, nf)
    x = np.concatenate([xb, xf]).astype(np.float32)
    y = np.concatenate([yb, yf]).astype(np.float32)
    s = np.concatenate([sb, sf])
    has = np.ones(len(x), bool)
    alerts = oracle.transient_search(x, y, has, s, now, [(5, 25), (10, 20)], 5, 5.0)
    assert alerts, "the flare must give alerts"
    best = max(alerts, key=lambda a: a[6])
    assert abs(best[1] - int((0.31 + 2.56) * 50)) <= 3 and abs(best[2] - int((-0.47 + 2.56) * 50)) <= 3
    assert best[6] > 8
    # every alert lies near the flare
    for a in alerts:
        assert abs(a[1] - best[1]) <= 10 and abs(a[2] - best[2]) <= 10
