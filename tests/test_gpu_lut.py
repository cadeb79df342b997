"""Lookup-table reconstruction on the GPU (rta_lut_accumulate, rta_lut_finalize,
rta_lut_reconstruct) against the oracle. Stage-isolated: both sides get the
same FP32 Hillas and stereo rows, and the reconstruction gets the oracle's
tables. Per-event results are FP64 in a fixed order on both sides, so they are
compared bit for bit after the rounding to FP32; the training sums are atomic
(order varies), so cell means and deviations get 4 units in the last place."""
import numpy as np
import pytest

import oracle
import synth
import paper_1307_6489_gb300 as rta
from oracle import lut

from gpu_helpers import f32_rows_as_oracle, hillas_rows_as_f32, make_ctx

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZE_EDGES = np.float32(10.0) ** np.linspace(1.0, 5.0, 25, dtype=np.float32)
DIST_EDGES = np.linspace(0.0, 900.0, 19, dtype=np.float32)
CUTS = (-2.0, 1.5, -2.0, 2.0)


def stereo_rows_as_f32(srows):
    """Oracle stereo rows rounded to FP32 and packed as rta_stereo_t."""
    S = oracle.S
    buf = np.zeros((len(srows), 8), np.float32)
    for j, k in enumerate(["dir_x", "dir_y", "core_x", "core_y"]):
        buf[:, j] = srows[:, S[k]].astype(np.float32)
    ib = buf.view(np.int32)
    ib[:, 4] = srows[:, S["n_valid"]].astype(np.int32)
    ib[:, 5] = srows[:, S["flags"]].astype(np.int32)
    return buf


def f32_stereo_as_oracle(buf):
    S = oracle.S
    out = np.zeros((len(buf), 6))
    for j, k in enumerate(["dir_x", "dir_y", "core_x", "core_y"]):
        out[:, S[k]] = buf[:, j]
    out[:, S["n_valid"]] = buf.view(np.int32)[:, 4]
    out[:, S["flags"]] = buf.view(np.int32)[:, 5]
    return out


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def training():
    """Generated gamma and proton showers through the oracle's image and stereo steps."""
    wl = synth.make_workload(3, 1500, seed=81)
    r = oracle.reconstruct(wl)
    hbuf = hillas_rows_as_f32(r["hillas"])
    sbuf = stereo_rows_as_f32(r["stereo"])
    return wl, hbuf, sbuf


@pytest.fixture(scope="module")
def ctx_of(training):
    wl = training[0]
    ctx = make_ctx(wl)
    yield ctx
    ctx.close()


def gpu_build(ctx, wl, hbuf, use, min_count, split=1):
    n_cells = rta.RTA_MAX_CAMS * (len(SIZE_EDGES) - 1) * (len(DIST_EDGES) - 1)
    acc = torch.zeros(n_cells * 8, dtype=torch.float64, device="cuda")
    cells = torch.zeros(n_cells * 8, dtype=torch.float32, device="cuda")
    h, tel = dev(hbuf.reshape(-1)), dev(wl.img_tel)
    le = dev(np.log10(wl.truth[:, 0]).astype(np.float32))
    core = dev(wl.truth[:, 3:5].astype(np.float32).reshape(-1))
    u = dev(np.asarray(use, np.uint8)) if use is not None else None
    se, de = dev(SIZE_EDGES), dev(DIST_EDGES)
    # several batches add to the same sums
    bounds = np.linspace(0, wl.n_evt, split + 1).astype(int)
    for a, b in zip(bounds[:-1], bounds[1:]):
        off = dev(wl.evt_off[a:b + 1])
        rta.rta_lut_accumulate(ctx.handle, h.data_ptr(), tel.data_ptr(), wl.n_img, off.data_ptr(), b - a,
                               le[a:].data_ptr(), core[2 * a:].data_ptr(), 0 if u is None else u[a:].data_ptr(),
                               se.data_ptr(), len(SIZE_EDGES) - 1, de.data_ptr(), len(DIST_EDGES) - 1,
                               acc.data_ptr())
    rta.rta_lut_finalize(ctx.handle, acc.data_ptr(), n_cells, min_count, cells.data_ptr())
    torch.cuda.synchronize()
    return rta.lut_cells_to_numpy(cells.cpu().numpy()), acc.cpu().numpy().reshape(-1, 8)


def oracle_build(wl, hbuf, use, min_count):
    return lut.lut_build(f32_rows_as_oracle(hbuf), wl.img_tel, wl.evt_off, wl.tel_cam, wl.tel_xy,
                         np.log10(wl.truth[:, 0]).astype(np.float32), wl.truth[:, 3:5].astype(np.float32), use,
                         SIZE_EDGES, DIST_EDGES, min_count)


@pytest.mark.parametrize("split", [1, 3])
def test_tables_match_the_oracle_build(training, ctx_of, split):
    wl, hbuf, _ = training
    use = (wl.truth[:, 5] == 0).astype(np.uint8)
    g, acc = gpu_build(ctx_of, wl, hbuf, use, 5, split)
    ref, cnt = oracle_build(wl, hbuf, use, 5)
    np.testing.assert_array_equal(g["n"], cnt.astype(np.int32))
    np.testing.assert_array_equal(acc[:, 0], cnt.astype(np.float64))
    assert (cnt >= 5).sum() > 30
    for j, k in enumerate(rta.LUT_CELL_FIELDS[1:]):
        r = ref[:, 1 + j]
        tol = 4 * np.spacing(np.abs(r)) + 1e-30
        bad = np.abs(g[k] - r) > tol
        assert not bad.any(), (k, np.nonzero(bad)[0][:5], g[k][bad][:5], r[bad][:5])


def test_all_events_and_every_min_count(training, ctx_of):
    wl, hbuf, _ = training
    for mc in (1, 40):
        g, _ = gpu_build(ctx_of, wl, hbuf, None, mc)
        ref, cnt = oracle_build(wl, hbuf, None, mc)
        np.testing.assert_array_equal(g["n"], cnt.astype(np.int32))
        assert ((g["sigma_w"] > 0) <= (cnt >= mc)).all()
        np.testing.assert_array_equal(g["mean_w"] != 0, ref[:, 1] != 0)


def lookup_of(ctx, cells):
    """The table's lookup form on the device (rta_lut_prepare)."""
    cl = dev(np.ascontiguousarray(cells, np.float32).reshape(-1))
    n_cells = cl.numel() // 8
    lk = torch.zeros(n_cells * rta.LUT_LOOKUP_BYTES // 4, dtype=torch.float32, device="cuda")
    rta.rta_lut_prepare(ctx.handle, cl.data_ptr(), n_cells, lk.data_ptr())
    return lk


def gpu_reconstruct(ctx, hbuf, img_tel, evt_off, n_img, sbuf, cells, cuts=CUTS, edges=(SIZE_EDGES, DIST_EDGES),
                    expect_bits=0):
    n_evt = len(evt_off) - 1
    out = torch.zeros(max(n_evt, 1) * 8, dtype=torch.float32, device="cuda")
    h, tel, off, st = dev(hbuf.reshape(-1)), dev(img_tel), dev(evt_off), dev(sbuf.reshape(-1))
    lk = lookup_of(ctx, cells)
    se, de = dev(edges[0]), dev(edges[1])
    rta.rta_lut_reconstruct(ctx.handle, h.data_ptr(), tel.data_ptr(), n_img, off.data_ptr(), n_evt, st.data_ptr(),
                            lk.data_ptr(), se.data_ptr(), len(edges[0]) - 1, de.data_ptr(), len(edges[1]) - 1, cuts,
                            out.data_ptr())
    torch.cuda.synchronize()
    bits = 0
    try:
        ctx.check()
    except rta.RtaError as e:
        bits = getattr(e, "bits", -1)
    assert bits == expect_bits, bits
    return rta.lut_events_to_numpy(out.cpu().numpy()[: n_evt * 8])


def oracle_cells_as_struct(ref):
    return rta.lut_cells_from_numpy(ref[:, 0], *[ref[:, k] for k in range(1, 7)])


def compare_events(g, ref):
    """Bit-exact: n_used and flags, and the four values as FP32."""
    np.testing.assert_array_equal(g["n_used"], ref[:, 4].astype(np.int32))
    np.testing.assert_array_equal(g["flags"], ref[:, 5].astype(np.uint32))
    for j, k in enumerate(["log_energy", "sigma_log_energy", "mscw", "mscl"]):
        np.testing.assert_array_equal(g[k], ref[:, j].astype(np.float32), err_msg=k)


@pytest.mark.parametrize("n_evt", [1, 37, 700, 1500])
def test_events_match_the_oracle_bit_for_bit(training, ctx_of, n_evt):
    wl, hbuf, sbuf = training
    ref_cells, _ = oracle_build(wl, hbuf, (wl.truth[:, 5] == 0), 5)
    cells = oracle_cells_as_struct(ref_cells)
    off = wl.evt_off[: n_evt + 1]
    g = gpu_reconstruct(ctx_of, hbuf, wl.img_tel, off, wl.n_img, sbuf[:n_evt], cells)
    ref = lut.lut_reconstruct(f32_rows_as_oracle(hbuf), wl.img_tel, off, wl.n_img, wl.tel_cam, wl.tel_xy,
                              f32_stereo_as_oracle(sbuf[:n_evt]), ref_cells, SIZE_EDGES, DIST_EDGES, CUTS)
    compare_events(g, ref)
    if n_evt >= 700:
        assert (g["flags"] & rta.RTA_LF_GAMMA).sum() > 50 and (g["n_used"] >= 2).sum() > 100


def test_edge_cases_match_the_oracle(training, ctx_of):
    """Malformed ranges, stereo-invalid events, unknown telescopes, empty and
    bad-input images, NaN and edge-valued sizes, events without images, and one
    event of 3000 images (several staging pieces)."""
    wl, hbuf, sbuf = training
    ref_cells, _ = oracle_build(wl, hbuf, (wl.truth[:, 5] == 0), 5)
    cells = oracle_cells_as_struct(ref_cells)
    rng = np.random.default_rng(9)
    n0 = 400
    hb = hbuf[:n0].copy()
    tel = wl.img_tel[:n0].copy()
    tel[5], tel[17] = -3, 10 ** 6                                  # unknown telescopes
    hb.view(np.int32)[9, 11] = rta.RTA_HF_BAD_INPUT
    hb.view(np.int32)[11, 11] = rta.RTA_HF_EMPTY
    hb[13, 4] = np.nan                                             # NaN width
    hb[15, 0] = SIZE_EDGES[3]                                      # a size on an edge
    hb[19, 0] = SIZE_EDGES[-1]                                     # on the last edge: outside
    big = rng.integers(0, n0, 3000)
    hb = np.concatenate([hb, hb[big]])
    tel = np.concatenate([tel, tel[big]])
    n_img = len(hb)
    off = [0]
    while off[-1] < n0:
        off.append(min(n0, off[-1] + int(rng.integers(0, 9))))
    off.append(n_img)                                              # the 3000-image event
    off = np.array(off, np.int32)
    n_evt = len(off) - 1
    st = stereo_rows_as_f32(f32_stereo_as_oracle(sbuf[rng.integers(0, len(sbuf), n_evt)]))
    st.view(np.int32)[3, 5] |= oracle.FLAG_STEREO_INVALID
    st.view(np.int32)[-1, 5] &= ~oracle.FLAG_STEREO_INVALID
    bad = off.copy()
    bad[7] = bad[8] + 1          # event 6 overlaps event 8's first image, event 7 ends before it starts
    bad[20] = -5
    for o, bits in ((off, 0), (bad, rta.RTA_DEV_BAD_IMAGE)):
        g = gpu_reconstruct(ctx_of, hb, tel, o, n_img, st, cells, expect_bits=bits)
        ref = lut.lut_reconstruct(f32_rows_as_oracle(hb), tel, o, n_img, wl.tel_cam, wl.tel_xy,
                                  f32_stereo_as_oracle(st), ref_cells, SIZE_EDGES, DIST_EDGES, CUTS)
        compare_events(g, ref)
    assert g["n_used"][-1] > 100
    assert (g["flags"] & rta.RTA_LF_MALFORMED).any() and (g["flags"] & rta.RTA_LF_NO_CORE).any()


def test_full_bundle_matches_the_oracle(ctx_of):
    """The benchmark bundle's shape (10,000 events of the 2000-image array
    preset, its multiplicities and telescopes) with synthetic Hillas and
    stereo rows, in the launch configuration of that event count."""
    rng = np.random.default_rng(10)
    # a table with every cell drawn at random, a tenth of them unused
    n_cells = rta.RTA_MAX_CAMS * (len(SIZE_EDGES) - 1) * (len(DIST_EDGES) - 1)
    ref_cells = np.zeros((n_cells, 8), np.float32)
    ref_cells[:, 0] = rng.integers(1, 500, n_cells)
    ref_cells[:, 1:7] = rng.uniform(0.01, 0.3, (n_cells, 6))
    ref_cells[:, 5] = rng.uniform(-1.5, 2.0, n_cells)
    ref_cells[rng.uniform(size=n_cells) < 0.1, 2] = 0.0
    cells = oracle_cells_as_struct(ref_cells)
    big = synth.make_workload(2, 10000, seed=synth.BASE_SEED + 2, render=False)
    n_img = big.n_img
    hb = np.zeros((n_img, 16), np.float32)
    hb[:, 0] = 10.0 ** rng.uniform(1.0, 4.5, n_img)
    hb[:, 3] = rng.gamma(6, 0.03, n_img)
    hb[:, 4] = rng.gamma(4, 0.02, n_img)
    hb.view(np.int32)[:, 10] = rng.integers(0, 60, n_img)
    st = np.zeros((big.n_evt, 8), np.float32)
    st[:, 2:4] = rng.uniform(-900, 900, (big.n_evt, 2))
    st.view(np.int32)[:, 5] = (rng.uniform(size=big.n_evt) < 0.05).astype(np.int32)
    g = gpu_reconstruct(ctx_of, hb, big.img_tel, big.evt_off, n_img, st, cells)
    ref = lut.lut_reconstruct(f32_rows_as_oracle(hb), big.img_tel, big.evt_off, n_img, big.tel_cam, big.tel_xy,
                              f32_stereo_as_oracle(st), ref_cells, SIZE_EDGES, DIST_EDGES, CUTS)
    compare_events(g, ref)
    assert (g["n_used"] > 0).sum() > 5000


def test_bad_arguments_are_refused(training, ctx_of):
    wl, hbuf, sbuf = training
    h = dev(hbuf.reshape(-1))
    tel, off, st = dev(wl.img_tel), dev(wl.evt_off), dev(sbuf.reshape(-1))
    cells = torch.zeros(rta.RTA_MAX_CAMS * 24 * 18 * rta.LUT_LOOKUP_BYTES // 4, dtype=torch.float32, device="cuda")
    out = torch.zeros(wl.n_evt * 8 + 4, dtype=torch.float32, device="cuda")
    se, de = dev(SIZE_EDGES), dev(DIST_EDGES)
    args = lambda n_size, o: (ctx_of.handle, h.data_ptr(), tel.data_ptr(), wl.n_img, off.data_ptr(), wl.n_evt,
                              st.data_ptr(), cells.data_ptr(), se.data_ptr(), n_size, de.data_ptr(), 18, CUTS, o)
    for n_size, o, code in [(0, out.data_ptr(), rta.RTA_E_INVALID), (65, out.data_ptr(), rta.RTA_E_INVALID),
                            (24, out.data_ptr() + 4, rta.RTA_E_ALIGN)]:
        with pytest.raises(rta.RtaError) as e:
            rta.rta_lut_reconstruct(*args(n_size, o))
        assert e.value.code == code
    acc = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(rta.RtaError) as e:
        rta.rta_lut_finalize(ctx_of.handle, acc.data_ptr(), 1, 0, cells.data_ptr())
    assert e.value.code == rta.RTA_E_INVALID
    with pytest.raises(rta.RtaError) as e:
        rta.rta_lut_prepare(ctx_of.handle, cells.data_ptr(), 1, cells.data_ptr() + 8)
    assert e.value.code == rta.RTA_E_ALIGN
