"""Transient search on the serving stream's sky map against the oracle: an hour
of background events added second by second, a 5-second flare and a 10-minute
flare, windows from one second to half an hour (both slab rings)."""
import numpy as np
import pytest

import oracle
import synth
import paper_1307_6489_gb300 as rta

from gpu_helpers import make_ctx, proc_args

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WINDOWS = [(1, 5), (5, 25), (10, 20), (60, 600), (300, 1800), (600, 3000), (1800, 1800)]
NOW_S = 1_000_000 * 60 + 37          # a second that is not on a minute boundary
RADIUS = 5
S_MIN = 4.0


def event_rows(x, y, has):
    rows = np.zeros((len(x), 8), np.float32)
    rows[:, 1], rows[:, 2] = x, y
    rows.view(np.uint32)[:, 5] = np.where(has, 0, rta.RTA_EF_NO_DIRECTION)
    return rows


@pytest.fixture(scope="module")
def sky():
    rng = np.random.default_rng(1307)
    secs = np.arange(NOW_S - 3599, NOW_S + 1)
    xs, ys, hs, ss = [], [], [], []
    for t in secs:
        n = int(rng.poisson(12))
        x = rng.uniform(-2.7, 2.7, n)
        y = rng.uniform(-2.7, 2.7, n)
        if t > NOW_S - 5:                                # 5-second flare
            k = int(rng.poisson(15))
            x = np.concatenate([x, 0.31 + rng.normal(0, 0.03, k)])
            y = np.concatenate([y, -0.47 + rng.normal(0, 0.03, k)])
        if t > NOW_S - 600 and t % 2 == 0:               # 10-minute flare, one event every other second
            x = np.concatenate([x, [-1.13 + rng.normal(0, 0.03)]])
            y = np.concatenate([y, [0.82 + rng.normal(0, 0.03)]])
        h = rng.uniform(size=len(x)) < 0.97
        xs.append(x.astype(np.float32)), ys.append(y.astype(np.float32)), hs.append(h), ss.append(np.full(len(x), t))
    wl = synth.make_workload(2, 5)
    ctx = make_ctx(wl)
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    st = rta.rta_stream_create(ctx.handle, 0, 64 << 20, 1, 1000, 1000, mode, start, W, t_hi, t_lo, core_nb, 0.5)
    cs = torch.cuda.current_stream().cuda_stream
    for x, y, h, s in zip(xs, ys, hs, ss):
        d = torch.from_numpy(event_rows(x, y, h).reshape(-1)).cuda()
        rta.rta_stream_add_events(st, d.data_ptr(), len(x), int(s[0]) * 1_000_000_000 + 123_456, cs)
    torch.cuda.synchronize()
    ev = dict(x=np.concatenate(xs), y=np.concatenate(ys), has=np.concatenate(hs), sec=np.concatenate(ss))
    yield st, ev
    rta.rta_stream_destroy(st)
    ctx.close()


@pytest.mark.parametrize("window", WINDOWS)
def test_significance_maps_match_the_oracle(sky, window):
    st, ev = sky
    sig, d_on, d_off = rta.rta_significance_map(st, NOW_S * 1_000_000_000 + 999, window, RADIUS)
    ref, r_on, r_off, alpha = oracle.transient_maps(ev["x"], ev["y"], ev["has"], ev["sec"], NOW_S, window, RADIUS)
    np.testing.assert_array_equal(d_on, r_on)
    np.testing.assert_array_equal(d_off, r_off)
    np.testing.assert_allclose(sig, ref, rtol=1e-12, atol=1e-12)
    assert r_on.sum() > 0 and r_off.sum() > 0


def test_alerts_match_the_oracle_and_find_the_flares(sky):
    st, ev = sky
    got = rta.rta_transient_search(st, NOW_S * 1_000_000_000 + 999, WINDOWS, RADIUS, S_MIN)
    ref = oracle.transient_search(ev["x"], ev["y"], ev["has"], ev["sec"], NOW_S, WINDOWS, RADIUS, S_MIN)
    key = lambda w, x, y: (int(w), int(x), int(y))
    gk = {key(a["window"], a["ix"], a["iy"]): a for a in got}
    rk = {key(r[0], r[1], r[2]): r for r in ref}
    # the same alerts, except bins whose significance sits on the threshold itself
    borderline = {k for k, r in rk.items() if abs(r[6] - S_MIN) < 1e-9}
    assert set(gk) - borderline == set(rk) - borderline
    for k in set(gk) & set(rk):
        a, r = gk[k], rk[k]
        assert (a["n_on"], a["n_off"]) == (r[3], r[4]) and a["alpha"] == r[5]
        assert abs(a["significance"] - r[6]) <= 1e-12 * max(1.0, abs(r[6]))
    order = [(a["window"], a["iy"], a["ix"]) for a in got]
    assert order == sorted(order)
    # the 5-second flare in the short windows, the 10-minute flare in the long ones
    fx, fy = int((0.31 + 2.56) * 50), int((-0.47 + 2.56) * 50)
    gx, gy = int((-1.13 + 2.56) * 50), int((0.82 + 2.56) * 50)
    short = [a for a in got if WINDOWS[a["window"]][0] <= 10]
    long_ = [a for a in got if WINDOWS[a["window"]][0] >= 300]
    assert any(abs(a["ix"] - fx) <= 3 and abs(a["iy"] - fy) <= 3 for a in short)
    assert any(abs(a["ix"] - gx) <= 3 and abs(a["iy"] - gy) <= 3 for a in long_)
    # a cap on the number returned keeps the first ones in order
    few = rta.rta_transient_search(st, NOW_S * 1_000_000_000 + 999, WINDOWS, RADIUS, S_MIN, max_alerts=3)
    assert len(few) == min(3, len(got)) and (few == got[: len(few)]).all()
    # ... and the number found is still the full count
    few, n_found = rta.rta_transient_search(st, NOW_S * 1_000_000_000 + 999, WINDOWS, RADIUS, S_MIN, max_alerts=3,
                                            with_total=True)
    assert n_found == len(got) and len(few) == min(3, len(got))


def test_windows_outside_the_rings_are_refused(sky):
    st, _ = sky
    for bad in [(20, 20), (60, 3600), (0, 10), (10, 0)]:
        with pytest.raises(rta.RtaError) as e:
            rta.rta_transient_search(st, NOW_S * 1_000_000_000, [bad], RADIUS, S_MIN)
        assert e.value.code == rta.RTA_E_INVALID
    with pytest.raises(rta.RtaError):
        rta.rta_transient_search(st, NOW_S * 1_000_000_000, [(5, 25)], rta.RTA_MAX_DISK_RADIUS + 1, S_MIN)
