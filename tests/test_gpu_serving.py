"""The serving stream: continuous batching under an HBM budget, results that are
the same alone and in a mix, the device path's results, and the sky map."""
import time

import numpy as np
import pytest

import oracle
import synth
import paper_1307_6489_gb300 as rta

from gpu_helpers import Dev, make_ctx, proc_args

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def pinned(a):
    a = np.ascontiguousarray(a)
    t = torch.empty(max(a.nbytes, 1), dtype=torch.uint8, pin_memory=True)
    v = t.numpy()[: a.nbytes].view(a.dtype).reshape(a.shape)
    v[...] = a
    return t, v


class HostBundle:
    def __init__(self, wl, arrival_ns):
        self.keep = []
        self.wave = self._pin(wl.wave)
        self.off = self._pin(wl.wave_off.astype(np.int64))
        self.tel = self._pin(wl.img_tel.astype(np.int32))
        self.evt = self._pin(wl.evt_off.astype(np.int32))
        self.events = self._pin(np.zeros(wl.n_evt * 32, np.uint8))
        self.b = rta.Bundle(self.wave.ctypes.data, self.wave.size, self.off.ctypes.data, self.tel.ctypes.data,
                            wl.n_img, self.evt.ctypes.data, wl.n_evt, arrival_ns, self.events.ctypes.data)

    def _pin(self, a):
        t, v = pinned(a)
        self.keep.append(t)
        return v


def make_bundles(wl, sizes):
    out, e = [], 0
    for n in sizes:
        out.append(synth.subset(wl, np.arange(e, e + n)))
        e += n
    return out


def serve(stream, bundles, arrival_ns, concurrent=True, times=None):
    hbs = [HostBundle(b, arrival_ns) for b in bundles]
    if concurrent:
        tickets = [rta.rta_stream_submit(stream, h.b) for h in hbs]
        rta.rta_stream_drain(stream, 120000)
    else:
        tickets = []
        for h in hbs:
            tickets.append(rta.rta_stream_submit(stream, h.b))
            rta.rta_stream_drain(stream, 120000)
    for t in tickets:           # a ticket is reported once
        if times is None:
            assert rta.rta_stream_poll(stream, t) is not None
        else:
            times.append(rta.rta_stream_poll_times(stream, t))
            assert times[-1] is not None
    return [h.events.copy() for h in hbs]


@pytest.fixture(scope="module")
def env():
    wl = synth.make_workload(2, 2400)
    ctx = make_ctx(wl)
    model = rta.rta_surrogate_create(ctx.handle, 5, np.array([0, 0.57, 0.0, -1.1] + [0] * 12, np.float32))
    yield wl, ctx, model
    rta.rta_surrogate_destroy(model)
    ctx.close()


@pytest.mark.parametrize("use_model", [True, False])
def test_results_are_the_same_alone_and_in_a_mix_and_equal_the_device_path(env, use_model):
    wl, ctx, model = env
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    bundles = make_bundles(wl, [700, 90, 400, 1, 650, 300, 259])
    st = rta.rta_stream_create(ctx.handle, model if use_model else 0, 3 << 30, 3, 20000, 2000, mode, start, W,
                               t_hi, t_lo, core_nb, 0.5)
    tm = []
    try:
        now = time.monotonic_ns()
        mixed = serve(st, bundles, now, concurrent=True, times=tm)
        alone = serve(st, bundles[:3], now, concurrent=False)
    finally:
        rta.rta_stream_destroy(st)
    # submitted together, bundles share passes: the device queue handed several to one pass
    print("bundles per pass:", [t.batch_bundles for t in tm])
    assert max(t.batch_bundles for t in tm) >= 2
    assert all(1 <= t.batch_bundles <= len(bundles) and t.ready_wait_ms >= 0 for t in tm)
    for a, m in zip(alone, mixed[:3]):
        np.testing.assert_array_equal(a, m)
    # the same rows as the device-resident calls
    for b, got in zip(bundles, mixed):
        dev = Dev(b)
        h = dev.hillas_buf()
        ctx.image_chain(dev.wave, dev.wave_off, dev.img_tel, mode, start, W, t_hi, t_lo, core_nb, h)
        if use_model:
            out = torch.zeros(b.n_evt * 32, dtype=torch.uint8, device="cuda")
            rta.rta_surrogate_infer(model, h.data_ptr(), dev.img_tel.data_ptr(), b.n_img, dev.evt_off.data_ptr(),
                                    b.n_evt, 0.5, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
            np.testing.assert_array_equal(got, out.cpu().numpy())
        else:
            s = dev.stereo_buf()
            ctx.stereo(h, dev.evt_off, dev.img_tel, s)
            sr = rta.stereo_to_numpy(s.cpu().numpy()[: b.n_evt * 8])
            ev = rta.events_to_numpy(got)
            np.testing.assert_array_equal(ev["dir_x"], sr["dir_x"])
            np.testing.assert_array_equal(ev["dir_y"], sr["dir_y"])
            np.testing.assert_array_equal((ev["flags"] & 1) != 0, (sr["flags"] & 1) != 0)
    ctx.check()


def test_admission_waits_for_the_budget(env):
    wl, ctx, model = env
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    bundles = make_bundles(wl, [600, 600, 600])
    need = max(b.wave_bytes for b in bundles)
    # room for one bundle at a time: the others are admitted as memory frees up
    st = rta.rta_stream_create(ctx.handle, 0, int(need * 1.3) + (8 << 20), 4, 20000, 3000, mode, start, W, t_hi,
                               t_lo, core_nb, 0.5)
    times = []
    try:
        res = serve(st, bundles, time.monotonic_ns(), times=times)
        big = synth.subset(wl, np.arange(0, 2400))
        with pytest.raises(rta.RtaError) as e:
            rta.rta_stream_submit(st, HostBundle(big, time.monotonic_ns()).b)
        assert e.value.code == rta.RTA_E_NOMEM
    finally:
        rta.rta_stream_destroy(st)
    st2 = rta.rta_stream_create(ctx.handle, 0, 4 << 30, 4, 20000, 2000, mode, start, W, t_hi, t_lo, core_nb, 0.5)
    try:
        ref = serve(st2, bundles, time.monotonic_ns())
    finally:
        rta.rta_stream_destroy(st2)
    for a, b in zip(res, ref):
        np.testing.assert_array_equal(a, b)
    # each bundle's times are ordered and its device durations positive; with room
    # for one bundle at a time, a later bundle is admitted only after an earlier one is done
    for t in times:
        assert t.arrival_ns <= t.submit_ns <= t.admit_ns <= t.done_ns
        assert t.h2d_ms > 0 and t.compute_ms > 0 and t.d2h_ms > 0 and 0 <= t.slot < 4
    assert max(t.admit_ns for t in times) >= min(t.done_ns for t in times)


def test_sky_map_matches_the_oracle():
    """Stage-isolated: synthetic directions (CPU) counted into one-second slabs."""
    wl = synth.make_workload(2, 5)
    ctx = make_ctx(wl)
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    st = rta.rta_stream_create(ctx.handle, 0, 64 << 20, 1, 1000, 1000, mode, start, W, t_hi, t_lo, core_nb, 0.5)
    rng = np.random.default_rng(2)
    xs, ys, hs, ss = [], [], [], []
    try:
        for sec in [1000 + s for s in [0, 0, 3, 10, 29, 30, 31, 45, 59, 60, 60, 61]]:
            n = int(rng.integers(8, 5000))
            x = rng.normal(0, 1.5, n).astype(np.float32)
            y = rng.normal(0, 1.5, n).astype(np.float32)
            edges = np.array([-2.56, 2.56, 0.02 * 7 - 2.56, np.nan, 2.5599999], np.float32)
            x[: len(edges)] = edges
            has = rng.uniform(size=n) < 0.9
            rows = np.zeros((n, 8), np.float32)
            rows[:, 1], rows[:, 2] = x, y
            rows.view(np.uint32)[:, 5] = np.where(has, 0, rta.RTA_EF_NO_DIRECTION)
            d = torch.from_numpy(rows.reshape(-1)).cuda()
            rta.rta_stream_add_events(st, d.data_ptr(), n, sec * 1_000_000_000 + 123,
                                      torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            xs.append(x), ys.append(y), hs.append(has), ss.append(np.full(n, sec))
            x_, y_, h_, s_ = (np.concatenate(v) for v in (xs, ys, hs, ss))
            for now in [sec, sec + 5]:
                got = rta.rta_skymap_read(st, now * 1_000_000_000 + 5)
                np.testing.assert_array_equal(got.astype(np.int64), oracle.skymap(x_, y_, h_, s_, now))
    finally:
        rta.rta_stream_destroy(st)
        ctx.close()


def test_submission_rejects_images_outside_the_bundle(env):
    """In a pass the image kernel addresses the whole arena, so each image must lie
    inside its own bundle's waveforms: rejected at submission otherwise."""
    wl, ctx, model = env
    mode, start, W, t_hi, t_lo, core_nb = proc_args(wl)
    b = make_bundles(wl, [50])[0]
    st = rta.rta_stream_create(ctx.handle, 0, 1 << 30, 2, 20000, 2000, mode, start, W, t_hi, t_lo, core_nb, 0.5)
    try:
        for change, code in [("past_end", rta.RTA_E_INVALID), ("misaligned", rta.RTA_E_ALIGN),
                             ("negative", rta.RTA_E_ALIGN)]:
            hb = HostBundle(b, time.monotonic_ns())
            if change == "past_end":
                hb.off[-1] = b.wave.size - 8          # the last image runs past the waveforms
            elif change == "misaligned":
                hb.off[1] += 4
            else:
                hb.off[0] = -8
            with pytest.raises(rta.RtaError) as e:
                rta.rta_stream_submit(st, hb.b)
            assert e.value.code == code, change
        # the stream still serves a good bundle afterwards
        res = serve(st, [b], time.monotonic_ns())
        assert len(res) == 1
    finally:
        rta.rta_stream_destroy(st)
