#!/usr/bin/env python
"""Benchmark: waveform -> Hillas -> stereo reconstruction of the 69-telescope
array (three camera types, bundles of 10,000 events of multiplicity 2-40).

One step = one pass of the whole path over one bundle: the fused image kernel
(calibrate + integrate + clean + Hillas, all images) and the stereo kernel (all
events), on inputs already resident in HBM. `value` is events/s over all ranks;
`e2e` is the same metric through the host-buffer call (pinned host bundle in,
host event list out, copies inside the timed region). The roofline object
reports the fused image kernel against the measured HBM copy bandwidth.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--events E] [--impl ours|reference]

Under torchrun each rank reconstructs its own bundle (different seed); the
bundles are independent, so no collective touches the data path ("weak").
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "waveform→Hillas→stereo events/s and GB/s vs HBM peak; p99 bundle latency"
WORKLOAD = "69-telescope array bundle (4x1855px/40, 15x1764px/30, 50x2048px/25 samples), 10k gamma events"
PAPER_RATE = "paper requirement: 0.5-8 GB/s of DL0 input (abstract, Sec. 2.2)"
HILLAS_BYTES, STEREO_BYTES = 64, 32


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(rank: int) -> int:
    """Each rank reconstructs its own bundle: the generator's seed of rank r."""
    import synth
    return synth.BASE_SEED + 2 + 1000 * rank


def max_over_ranks(x: float, ws: int, device=None) -> float:
    """The largest value over all ranks (a step time, so that the slowest rank
    sets the job's time); x itself when there is one rank."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, ws: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank has its own bundle of the same size)."""
    return units_per_rank * ws / seconds


def make_bundle(n_events: int, seed: int, pinned: bool):
    import synth
    import torch
    wl = synth.make_workload(2, n_events, seed=seed, render=False)
    total = wl.n_samples_total
    if pinned:
        host = torch.empty(total, dtype=torch.int16, pin_memory=True)
        buf = host.numpy().view(np.uint16)
    else:
        host, buf = None, np.empty(total, np.uint16)
    synth.render_waves(wl, wave_out=buf)
    return wl, host


def cpu_baseline(wl, target_s: float = 10.0):
    """The oracle, as it stands, on a bounded sample of the same bundle (all host
    cores): whole passes over the bundle's first events until about target_s of work."""
    import oracle
    import synth
    cores = os.cpu_count() or 1
    n = min(wl.n_evt, 64)
    while True:
        sub = synth.subset(wl, np.arange(n))
        t0 = time.perf_counter()
        oracle.reconstruct(sub, threads=cores)
        dt = time.perf_counter() - t0
        if dt >= target_s / 4 or n >= wl.n_evt:
            break
        n = min(wl.n_evt, max(n * 2, int(n * target_s / 4 / max(dt, 1e-3))))
    reps, total = 1, dt
    while total < target_s:
        t0 = time.perf_counter()
        oracle.reconstruct(sub, threads=cores)
        total += time.perf_counter() - t0
        reps += 1
    return {"value": reps * n / total, "unit": "events/s", "cores": cores, "kind": "oracle",
            "sample": f"{reps} passes over the first {n} events ({sub.n_img} images, {sub.wave_bytes / 1e6:.0f} MB) "
                      f"of the bundle, {total:.1f} s on {cores} threads",
            "gbs": reps * sub.wave_bytes / total / 1e9}


# lookup-table binning: 32 size bins over 10..1e5 photoelectrons, 20 distance bins of 50 m
LUT_SIZE_EDGES = np.float32(10.0) ** np.linspace(1.0, 5.0, 33, dtype=np.float32)
LUT_DIST_EDGES = np.linspace(0.0, 1000.0, 21, dtype=np.float32)
LUT_CUTS = (-2.0, 0.9, -2.0, 2.0)      # gamma box: mscw_lo, mscw_hi, mscl_lo, mscl_hi


def stream_leg(ctx, wl, proc, stream, steps, e2e_steps, hil, ste, tune=True):
    """The bundle as a DL0 byte stream (the packet layout of include/rta.h),
    written by the generator into pinned host memory: rta_ingest alone (with and
    without the CRC check), the zero-copy rta_reconstruct_stream, and end to end
    per step: host-to-device copy of the stream, ingest with CRC, reconstruction,
    device-to-host copy of the Hillas and stereo rows. The stream path's image
    kernel gets its own launch configuration from rta_autotune_stream (outside
    the timed regions); the time under the contiguous bundle's configuration is
    reported beside it."""
    import torch
    import paper_1307_6489_gb300 as rta
    import synth
    sp = stream.cuda_stream
    plan = synth.stream_plan(wl)
    n_bytes = plan["n_bytes"]
    host = torch.empty(n_bytes, dtype=torch.uint8, pin_memory=True)
    buf, plan = synth.encode_stream(wl, out=host.numpy())
    n_pk = len(plan["img"])
    d_stream = torch.empty((n_bytes + 31) // 16 * 16, dtype=torch.uint8, device="cuda")
    d_seg = torch.empty(n_pk * 2, dtype=torch.int64, device="cuda")
    d_img_seg = torch.empty(wl.n_img + 1, dtype=torch.int32, device="cuda")
    d_img_tel = torch.empty(wl.n_img, dtype=torch.int32, device="cuda")
    d_evt_off = torch.empty(wl.n_evt + 1, dtype=torch.int32, device="cuda")
    d_evn = torch.empty(wl.n_evt, dtype=torch.int64, device="cuda")
    d_evt = torch.empty(wl.n_evt, dtype=torch.int64, device="cuda")
    d_cnt = torch.zeros(6, dtype=torch.int64, device="cuda")
    h2 = torch.empty_like(hil)
    s2 = torch.empty_like(ste)
    h = ctx.handle
    d_stream[:n_bytes].copy_(host, non_blocking=True)
    torch.cuda.synchronize()

    def ingest(crc):
        rta.rta_ingest(h, d_stream.data_ptr(), n_bytes, crc, d_seg.data_ptr(), n_pk, d_img_seg.data_ptr(),
                       d_img_tel.data_ptr(), wl.n_img, d_evt_off.data_ptr(), d_evn.data_ptr(), d_evt.data_ptr(),
                       wl.n_evt, d_cnt.data_ptr(), sp)

    def recon():
        rta.rta_reconstruct_stream(h, d_stream.data_ptr(), n_bytes, d_seg.data_ptr(), n_pk, d_img_seg.data_ptr(),
                                   d_img_tel.data_ptr(), wl.n_img, d_evt_off.data_ptr(), wl.n_evt, d_cnt.data_ptr(),
                                   *proc, h2.data_ptr(), s2.data_ptr(), sp)

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    ingest_ms = timed(lambda: ingest(0))
    ingest_crc_ms = timed(lambda: ingest(1))
    cnt = d_cnt.cpu().numpy()
    assert cnt[4] == 0 and cnt[0] == n_pk and cnt[1] == wl.n_img and cnt[2] == wl.n_evt, cnt
    recon_ms = timed(recon)
    ctx.check(sp)
    assert torch.equal(h2, hil) and torch.equal(s2, ste), "zero-copy rows differ from the bundle path"
    recon_bundle_cfg_ms, stream_cfg = recon_ms, None
    if tune:
        entries = rta.rta_autotune_stream(h, d_stream.data_ptr(), n_bytes, d_seg.data_ptr(), n_pk,
                                          d_img_seg.data_ptr(), d_img_tel.data_ptr(), wl.n_img, d_cnt.data_ptr(),
                                          *proc, h2.data_ptr(), reps=2, stream=sp)
        best = min(entries, key=lambda e: e["ms"])
        for e in sorted(entries, key=lambda e: e["ms"])[:6]:
            print("autotune_stream", json.dumps(e), file=sys.stderr)
        stream_cfg = {"variant": best["variant"], "n_stages": best["n_stages"], "ctas_per_sm": best["ctas_per_sm"],
                      "grid": best["grid"], "configs_measured": len(entries)}
        h2.zero_()
        s2.zero_()
        recon_ms = timed(recon)
        ctx.check(sp)
        assert torch.equal(h2, hil) and torch.equal(s2, ste), "zero-copy rows differ under the tuned configuration"
    # end to end from the pinned host stream: two device copies of the stream, so
    # that the next bundle's upload (copy stream) overlaps this bundle's ingest,
    # reconstruction and read-back (compute stream)
    hh = torch.empty(hil.numel(), dtype=torch.float32, pin_memory=True)
    hs = torch.empty(ste.numel(), dtype=torch.float32, pin_memory=True)
    bufs = [d_stream, torch.empty_like(d_stream)]
    cs = torch.cuda.Stream()
    up = [torch.cuda.Event(), torch.cuda.Event()]
    done = [torch.cuda.Event(), torch.cuda.Event()]
    for ev in done:
        ev.record(stream)

    def e2e_step(k):
        nonlocal d_stream
        b = k & 1
        cs.wait_event(done[b])
        with torch.cuda.stream(cs):
            bufs[b][:n_bytes].copy_(host, non_blocking=True)
        up[b].record(cs)
        stream.wait_event(up[b])
        d_stream = bufs[b]
        ingest(1)
        recon()
        with torch.cuda.stream(stream):
            hh.copy_(h2, non_blocking=True)
            hs.copy_(s2, non_blocking=True)
        done[b].record(stream)

    e2e_step(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        e2e_step(k)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    ctx.check(sp)
    assert torch.equal(hh, hil.cpu()), "end-to-end stream rows differ"
    hbm_peak, _ = peaks()
    return {"stream_bytes": n_bytes, "packets": n_pk, "ingest_ms": ingest_ms, "ingest_crc_ms": ingest_crc_ms,
            "ingest_crc_gbs": n_bytes / (ingest_crc_ms / 1e3) / 1e9,
            "ingest_crc_hbm_frac": n_bytes / (ingest_crc_ms / 1e3) / 1e9 / hbm_peak,
            "reconstruct_stream_ms": recon_ms,
            "reconstruct_stream_hbm_frac": n_bytes / (recon_ms / 1e3) / 1e9 / hbm_peak,
            "reconstruct_stream_ms_bundle_config": recon_bundle_cfg_ms,
            "stream_config": stream_cfg,
            "e2e": {"value": wl.n_evt / e2e_s, "unit": "events/s", "h2d_bytes_per_step": n_bytes,
                    "d2h_bytes_per_step": (hil.numel() + ste.numel()) * 4, "gbs": n_bytes / e2e_s / 1e9,
                    "call": "H2D stream + rta_ingest (CRC) + rta_reconstruct_stream + D2H rows, "
                            "next upload overlapped"}}


def config0_leg(steps, device, n_events=2000):
    """The small single camera: 2,000 events of the 16 x 16 square camera (16
    samples, fixed 5-sample window, tailcut 10/5): 16.4 MB, resident in L2, so
    its rate is not an HBM measurement. Reported: the image kernel's events/s,
    every event's image compared with the oracle (n_pix exact, size within 1e-4),
    and the oracle on all events (all host cores)."""
    import torch
    import oracle
    import paper_1307_6489_gb300 as rta
    import synth
    wl = synth.make_workload(0, n_events)
    ctx = rta.Context(device, hbm_budget_bytes=1 << 30)
    for c, cam in wl.cams.items():
        ctx.register_camera(c, cam.xy, cam.nb, cam.n_samples)
    ctx.register_array(wl.tel_cam, wl.tel_xy, wl.p16, wl.scale)
    p = wl.proc
    proc = (rta.RTA_WINDOW_SLIDING if p.sliding else rta.RTA_WINDOW_FIXED, p.start, p.W, p.t_hi, p.t_lo,
            p.core_needs_neighbour)
    dev = torch.device("cuda", device)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    wave = torch.from_numpy(wl.wave.view(np.int16)).to(dev)
    off = torch.from_numpy(np.ascontiguousarray(wl.wave_off)).to(dev)
    tel = torch.from_numpy(np.ascontiguousarray(wl.img_tel)).to(dev)
    hil = torch.zeros(wl.n_img * 16, dtype=torch.float32, device=dev)

    def chain():
        rta.rta_image_chain(ctx.handle, wave.data_ptr(), wave.numel(), off.data_ptr(), tel.data_ptr(), wl.n_img, *proc,
                            hil.data_ptr(), sp)

    for _ in range(3):
        chain()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        chain()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    ctx.check(sp)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    passes = 0
    while passes == 0 or time.perf_counter() - t0 < 2.0:      # whole passes, about 2 s of work
        ref = oracle.reconstruct(wl, do_stereo=False, threads=cores)
        passes += 1
    cpu_s = (time.perf_counter() - t0) / passes
    g = rta.hillas_to_numpy(hil.cpu().numpy())
    H = oracle.H
    nmatch = int(np.sum(g["n_pix"] == ref["hillas"][:, H["n_pix"]].astype(np.int32)))
    ok = ref["hillas"][:, H["n_pix"]] > 0
    rel = np.abs(g["size"][ok] - ref["hillas"][ok, H["size"]]) / ref["hillas"][ok, H["size"]]
    ctx.close()
    return {"workload": f"16x16 square camera, {wl.n_evt} events x 16 samples, {wl.wave_bytes / 1e6:.1f} MB "
                        "(L2-resident: not an HBM measurement)",
            "kernel": {"ms": ms, "events_per_s": wl.n_evt / (ms / 1e3)},
            "parity_all_events": {"events": wl.n_evt, "n_pix_equal": nmatch,
                                  "max_size_rel_err": float(rel.max()) if ok.any() else 0.0,
                                  "pass": bool(nmatch == wl.n_evt and (not ok.any() or rel.max() <= 1e-4))},
            "cpu_baseline": {"value": wl.n_evt / cpu_s, "unit": "events/s", "cores": cores, "kind": "oracle",
                             "sample": f"{passes} passes over all {wl.n_evt} events, {cpu_s * 1e3:.1f} ms each on "
                                       f"{cores} threads"}}


def config1_leg(n_events, hbm_peak, steps, device, cpu_events=20000, sample_events=300):
    """The single large camera streamed from host memory: n_events events of the
    1855-pixel hexagonal camera (40 samples, sliding 6-sample window, tailcut 8/4
    with the neighbour test), about 30 GB at 200,000 events, in a pinned host
    buffer. Reported: the image kernel's GB/s on one HBM-resident chunk (roofline
    fraction), the end-to-end rate of rta_reconstruct_host over the whole stream
    (its chunked, double-buffered host-to-device copies included), the oracle on
    the first cpu_events events (all host cores), and a sampled parity check of
    the streamed rows against the oracle."""
    import torch
    import oracle
    import paper_1307_6489_gb300 as rta
    import synth
    t_setup = time.perf_counter()
    wl = synth.make_workload(1, n_events, render=False)
    host = torch.empty(wl.n_samples_total, dtype=torch.int16, pin_memory=True)
    wave_h = host.numpy().view(np.uint16)
    synth.render_waves(wl, wave_out=wave_h)
    gen_s = time.perf_counter() - t_setup
    ctx = rta.Context(device, hbm_budget_bytes=8 << 30)
    for c, cam in wl.cams.items():
        ctx.register_camera(c, cam.xy, cam.nb, cam.n_samples)
    ctx.register_array(wl.tel_cam, wl.tel_xy, wl.p16, wl.scale)
    p = wl.proc
    proc = (rta.RTA_WINDOW_SLIDING if p.sliding else rta.RTA_WINDOW_FIXED, p.start, p.W, p.t_hi, p.t_lo,
            p.core_needs_neighbour)
    dev = torch.device("cuda", device)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    # the image kernel on one HBM-resident chunk of up to 20,000 events (~3 GB, larger than L2)
    n_c = min(wl.n_evt, 20000)
    i_c = int(wl.evt_off[n_c])
    s_c = int(wl.wave_off[i_c]) if i_c < wl.n_img else wl.n_samples_total
    wave_c = host[:s_c].to(dev)
    off_c = torch.from_numpy(np.ascontiguousarray(wl.wave_off[:i_c])).to(dev)
    tel_c = torch.from_numpy(np.ascontiguousarray(wl.img_tel[:i_c])).to(dev)
    hil_c = torch.zeros(i_c * 16, dtype=torch.float32, device=dev)
    h = ctx.handle

    def chain():
        rta.rta_image_chain(h, wave_c.data_ptr(), wave_c.numel(), off_c.data_ptr(), tel_c.data_ptr(), i_c, *proc,
                            hil_c.data_ptr(), sp)

    for _ in range(3):
        chain()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        chain()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    chain_ms = e0.elapsed_time(e1) / steps
    ctx.check(sp)
    alg = 2 * s_c + 64 * i_c
    kernel_gbs = alg / (chain_ms / 1e3) / 1e9
    del wave_c
    torch.cuda.empty_cache()
    # end to end: the whole host stream through rta_reconstruct_host
    hh = np.zeros(wl.n_img * 16, np.float32)
    hs = np.zeros(wl.n_evt * 8, np.float32)
    woff = np.ascontiguousarray(wl.wave_off)
    itel = np.ascontiguousarray(wl.img_tel)
    eoff = np.ascontiguousarray(wl.evt_off)
    ctx.reconstruct_host(wave_h, woff, itel, eoff, *proc, hh, hs)      # warm (staging buffers)
    passes = 2
    t0 = time.perf_counter()
    for _ in range(passes):
        ctx.reconstruct_host(wave_h, woff, itel, eoff, *proc, hh, hs)
    e2e_s = (time.perf_counter() - t0) / passes
    # the HBM-resident chunk and the streamed pass give the same rows
    assert np.array_equal(hh[: i_c * 16].view(np.uint32), hil_c.cpu().numpy().view(np.uint32)), "streamed rows differ"
    # sampled parity of the streamed rows against the oracle, over the whole stream
    rng = np.random.default_rng(5)
    ev = np.sort(rng.choice(wl.n_evt, min(sample_events, wl.n_evt), replace=False))
    sub = synth.subset(wl, ev)
    ref = oracle.reconstruct(sub, do_stereo=False)
    g = rta.hillas_to_numpy(hh.reshape(-1, 16)[ev].reshape(-1))
    H = oracle.H
    nmatch = int(np.sum(g["n_pix"] == ref["hillas"][:, H["n_pix"]].astype(np.int32)))
    ok = ref["hillas"][:, H["n_pix"]] > 0
    rel = np.abs(g["size"][ok] - ref["hillas"][ok, H["size"]]) / ref["hillas"][ok, H["size"]]
    parity = {"events": int(len(ev)), "n_pix_equal": nmatch, "max_size_rel_err": float(rel.max()) if ok.any() else 0.0,
              "pass": bool(nmatch == len(ev) and (not ok.any() or rel.max() <= 1e-4))}
    # the oracle on the first cpu_events events, all host cores
    cores = os.cpu_count() or 1
    n_o = min(cpu_events, wl.n_evt)
    sub_o = synth.subset(wl, np.arange(n_o))
    t0 = time.perf_counter()
    oracle.reconstruct(sub_o, do_stereo=False, threads=cores)
    cpu_s = time.perf_counter() - t0
    out = {"workload": f"1855-pixel hexagonal camera, {wl.n_evt} events x 40 samples, {wl.wave_bytes / 1e9:.2f} GB "
                       "in pinned host memory", "events": wl.n_evt, "bytes": wl.wave_bytes, "generate_s": gen_s,
           "kernel": {"events_on_device": n_c, "ms": chain_ms, "gbs": kernel_gbs, "hbm_frac": kernel_gbs / hbm_peak,
                      "events_per_s": n_c / (chain_ms / 1e3)},
           "e2e": {"value": wl.n_evt / e2e_s, "unit": "events/s", "gbs": wl.wave_bytes / e2e_s / 1e9,
                   "h2d_bytes_per_pass": wl.wave_bytes + wl.n_img * 12 + (wl.n_evt + 1) * 4,
                   "d2h_bytes_per_pass": wl.n_img * 64 + wl.n_evt * 32, "passes": passes,
                   "call": "rta_reconstruct_host (pinned host stream, chunked and double-buffered)"},
           "cpu_baseline": {"value": n_o / cpu_s, "unit": "events/s", "cores": cores, "kind": "oracle",
                            "sample": f"the first {n_o} events, {cpu_s:.1f} s on {cores} threads",
                            "gbs": sub_o.wave_bytes / cpu_s / 1e9},
           "parity_sampled": parity}
    ctx.close()
    del host
    return out


def cam_codes(wl):
    codes = np.zeros(16, np.float32)
    for c, cam in wl.cams.items():
        codes[c] = np.log10(cam.mirror_area) - 2.0
    return codes


def hillas_sets(ctx, calib_seed, proc, n_events, chunk=20000, seed0=1307064893):
    """Hillas rows of n_events events of the learned-surrogate preset (the array,
    gamma and proton showers) made the way a deployment makes them: waveforms
    rendered chunk by chunk into device memory (the generator's GPU renderer:
    same showers and noise as the host renderer, in FP32) and reconstructed by
    the image kernel; only the 64-byte rows stay (device). Returns rows,
    telescopes, event offsets, truth and camera codes."""
    import torch
    import synth
    plans = []
    k = 0
    while sum(p.n_evt for p in plans) < n_events:
        n = min(chunk, n_events - sum(p.n_evt for p in plans))
        plans.append(synth.make_workload(3, n, seed=seed0 + 7919 * k, render=False, calib_seed=calib_seed))
        k += 1
    n_img = sum(p.n_img for p in plans)
    rows = torch.zeros(n_img * 16, dtype=torch.float32, device="cuda")
    tel = torch.from_numpy(np.concatenate([p.img_tel for p in plans]).astype(np.int32)).cuda()
    dwave = torch.empty(max(p.n_samples_total for p in plans), dtype=torch.int16, device="cuda")
    i0 = 0
    for p in plans:
        keep = synth.render_waves_gpu(p, dwave, torch.cuda.current_stream().cuda_stream)
        off = torch.from_numpy(np.ascontiguousarray(p.wave_off)).cuda()
        ctx.image_chain(dwave[: p.n_samples_total], off, tel[i0:i0 + p.n_img], *proc,
                        rows[i0 * 16:(i0 + p.n_img) * 16])
        torch.cuda.synchronize()
        del keep
        i0 += p.n_img
    ctx.check()
    offs, base = [0], 0
    for p in plans:
        offs.extend((p.evt_off[1:] + base).tolist())
        base += p.n_img
    truth = np.concatenate([p.truth for p in plans])
    del dwave
    torch.cuda.empty_cache()
    return rows, tel, np.asarray(offs, np.int64), truth, cam_codes(plans[0])


def oracle_forward_baseline(tr, h_dev, tel_dev, evt_off, codes, n_evt):
    """The oracle's learned reconstruction (features and FP64 forward pass, numpy)
    on the first n_evt held-out events with the trained weights, timed on the
    host: the CPU baseline of the learned path."""
    import oracle
    import paper_1307_6489_gb300 as rta
    from oracle import mlp
    import synth
    n_img = int(evt_off[n_evt])
    g = rta.hillas_to_numpy(h_dev[: n_img * 16].cpu().numpy())
    H = oracle.H
    rows = np.zeros((n_img, 12))
    for k in rta.HILLAS_FIELDS:
        rows[:, H[k]] = g[k]
    rows[:, H["n_pix"]] = g["n_pix"]
    rows[:, H["flags"]] = g["flags"]
    tel = tel_dev[:n_img].cpu().numpy()
    tel_cam, tel_xy = np.zeros(69, np.int32), np.zeros(138, np.float32)
    synth._L().synth_array(synth._p(tel_cam), synth._p(tel_xy))
    params = rta.unpack_params(rta.rta_surrogate_get_params(tr.model, 0))
    params = {k: mlp.bf16_round(v) for k, v in params.items()}
    off = np.asarray(evt_off[: n_evt + 1], np.int64)
    t0 = time.perf_counter()
    X, used, base, n_used = mlp.features(rows, off, tel, tel_xy.reshape(-1, 2).astype(np.float64), codes[tel_cam])
    y, _ = mlp.forward(params, mlp.bf16_round(X), used, off)
    dt = time.perf_counter() - t0
    return {"value": n_evt / dt, "unit": "events/s", "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": f"features and FP64 forward pass of the first {n_evt} held-out events ({n_img} images), "
                      f"{dt:.1f} s (numpy; the matrix products may use the host's threads)"}


def surrogate_leg(ctx, wl, dev_b, proc, stream, steps, n_train, n_eval, train_epochs=0):
    """Train the deep-sets surrogate with the library's kernels on n_train mixed
    gamma/proton events and judge it, next to the geometric reconstruction and
    the lookup tables built from the same training events, on n_eval held-out
    events (setup, outside any timed region); then time the learned path on the
    benchmark bundle (image kernel + surrogate with geometric fallback) against
    the geometric path."""
    import torch
    import paper_1307_6489_gb300 as rta
    from paper_1307_6489_gb300 import train
    wave, wave_off, img_tel, evt_off, hil, ste = dev_b
    sp = stream.cuda_stream
    t_setup = time.perf_counter()
    rows, tel, offs, truth, codes = hillas_sets(ctx, wl.seed, proc, n_train + n_eval)
    gen_s = time.perf_counter() - t_setup
    i_tr = int(offs[n_train])
    h_tr, tel_tr, off_tr = rows[: i_tr * 16], tel[:i_tr], offs[: n_train + 1]
    h_ev, tel_ev = rows[i_tr * 16:].contiguous(), tel[i_tr:].contiguous()
    off_ev = (offs[n_train:] - i_tr).astype(np.int32)
    tr_truth, ev_truth = truth[:n_train], truth[n_train:]
    dev = wave.device
    logE = torch.from_numpy(np.log10(tr_truth[:, 0]).astype(np.float32)).to(dev)
    src = torch.from_numpy(tr_truth[:, 1:3].astype(np.float32).reshape(-1)).to(dev)
    gam = torch.from_numpy((tr_truth[:, 5] == 0).astype(np.uint8)).to(dev)
    tr = train.SurrogateTrainer(ctx, seed=1, cam_code=codes)
    t_fit = time.perf_counter()
    # about 6,000 Adam steps of 2,048 events whatever the training-set size (at least 3 epochs)
    epochs = train_epochs or max(3, int(round(6000 * 2048 / n_train)))
    losses = tr.fit(h_tr, tel_tr, off_tr, logE, src, gam, epochs=epochs, batch_events=2048, lr=2e-3, lr_end=5e-5)
    fit_s = time.perf_counter() - t_fit
    # lookup tables (calibration matrices) from the same training gammas at their true cores
    se_d = torch.from_numpy(LUT_SIZE_EDGES).to(dev)
    de_d = torch.from_numpy(LUT_DIST_EDGES).to(dev)
    n_cells = rta.RTA_MAX_CAMS * (len(LUT_SIZE_EDGES) - 1) * (len(LUT_DIST_EDGES) - 1)
    acc = torch.zeros(n_cells * 8, dtype=torch.float64, device=dev)
    cells = torch.zeros(n_cells * 8, dtype=torch.float32, device=dev)
    core_t = torch.from_numpy(tr_truth[:, 3:5].astype(np.float32).reshape(-1)).to(dev)
    devt_tr = torch.from_numpy(off_tr.astype(np.int32)).to(dev)
    rta.rta_lut_accumulate(ctx.handle, h_tr.data_ptr(), tel_tr.data_ptr(), i_tr, devt_tr.data_ptr(), n_train,
                           logE.data_ptr(), core_t.data_ptr(), gam.data_ptr(), se_d.data_ptr(),
                           len(LUT_SIZE_EDGES) - 1, de_d.data_ptr(), len(LUT_DIST_EDGES) - 1, acc.data_ptr(), sp)
    rta.rta_lut_finalize(ctx.handle, acc.data_ptr(), n_cells, 10, cells.data_ptr(), sp)
    lookup = torch.zeros(n_cells * rta.LUT_LOOKUP_BYTES // 4, dtype=torch.float32, device=dev)
    rta.rta_lut_prepare(ctx.handle, cells.data_ptr(), n_cells, lookup.data_ptr(), sp)
    # the held-out events: learned path, geometric path and lookup tables on the same rows
    n_ev_img = h_ev.numel() // 16
    devt_ev = torch.from_numpy(off_ev).to(dev)
    st_ev = torch.zeros(n_eval * 8, dtype=torch.float32, device=dev)
    lev_ev = torch.zeros(n_eval * 8, dtype=torch.float32, device=dev)
    sev = torch.zeros(n_eval * 32, dtype=torch.uint8, device=dev)
    rta.rta_stereo(ctx.handle, h_ev.data_ptr(), tel_ev.data_ptr(), n_ev_img, devt_ev.data_ptr(), n_eval,
                   st_ev.data_ptr(), sp)
    rta.rta_surrogate_infer(tr.model, h_ev.data_ptr(), tel_ev.data_ptr(), n_ev_img, devt_ev.data_ptr(), n_eval, 0.5,
                            sev.data_ptr(), sp)
    rta.rta_lut_reconstruct(ctx.handle, h_ev.data_ptr(), tel_ev.data_ptr(), n_ev_img, devt_ev.data_ptr(), n_eval,
                            st_ev.data_ptr(), lookup.data_ptr(), se_d.data_ptr(), len(LUT_SIZE_EDGES) - 1,
                            de_d.data_ptr(), len(LUT_DIST_EDGES) - 1, LUT_CUTS, lev_ev.data_ptr(), sp)
    torch.cuda.synchronize()
    ctx.check(sp)
    sev_np = rta.events_to_numpy(sev.cpu().numpy())
    held_out = train.evaluate(sev_np, rta.stereo_to_numpy(st_ev.cpu().numpy()), ev_truth)
    lt = rta.lut_events_to_numpy(lev_ev.cpu().numpy())
    ok_l = (lt["flags"] & (rta.RTA_LF_NO_CORE | rta.RTA_LF_NO_IMAGE | rta.RTA_LF_MALFORMED)) == 0
    g_ev = ev_truth[:, 5] == 0
    # the learned energy on exactly the gammas the tables give an energy for
    sub = ok_l & g_ev & ((sev_np["flags"] & rta.RTA_EF_NO_DIRECTION) == 0)
    d_s = sev_np["log_energy"][sub] - np.log10(ev_truth[sub, 0])
    held_out["energy_res_on_table_events"] = float(np.std(d_s)) if sub.any() else None
    held_out["energy_bias_on_table_events"] = float(np.mean(d_s)) if sub.any() else None
    d_le = lt["log_energy"][ok_l & g_ev] - np.log10(ev_truth[ok_l & g_ev, 0])
    lut_held_out = {"with_energy_frac": float(np.mean(ok_l[g_ev])) if g_ev.any() else None,
                    "energy_bias": float(np.mean(d_le)) if len(d_le) else None,
                    "energy_res": float(np.std(d_le)) if len(d_le) else None,
                    "gamma_pass": float(np.mean((lt["flags"][ok_l & g_ev] & rta.RTA_LF_GAMMA) != 0))
                    if (ok_l & g_ev).any() else None,
                    "proton_pass": float(np.mean((lt["flags"][ok_l & ~g_ev] & rta.RTA_LF_GAMMA) != 0))
                    if (ok_l & ~g_ev).any() else None}
    proton_pass = lut_held_out["proton_pass"]
    cpu_fwd = oracle_forward_baseline(tr, h_ev, tel_ev, off_ev, codes, min(100000, n_eval))
    del rows, h_tr, h_ev, st_ev, lev_ev, sev
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    # timed: image kernel + learned reconstruction on the bundle
    ev = torch.zeros(wl.n_evt * 32, dtype=torch.uint8, device=wave.device)
    h = ctx.handle

    def sur_step():
        # image kernel + learned reconstruction in one call (the inference kernel reads the
        # bundle's offsets and the weights while the image kernel finishes)
        rta.rta_reconstruct_learned(tr.model, wave.data_ptr(), wave.numel(), wave_off.data_ptr(), img_tel.data_ptr(),
                                    wl.n_img, evt_off.data_ptr(), wl.n_evt, *proc, 0.5, hil.data_ptr(), ev.data_ptr(),
                                    sp)

    def sur_step_nofb():
        rta.rta_reconstruct_learned(tr.model, wave.data_ptr(), wave.numel(), wave_off.data_ptr(), img_tel.data_ptr(),
                                    wl.n_img, evt_off.data_ptr(), wl.n_evt, *proc, 1e30, hil.data_ptr(), ev.data_ptr(),
                                    sp)

    for _ in range(3):
        sur_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        sur_step()
    e1.record(stream)
    torch.cuda.synchronize()
    sur_ms = e0.elapsed_time(e1) / steps
    ctx.check(sp)

    def infer_ms(bound):
        # the learned reconstruction alone on the Hillas rows of the bundle
        for _ in range(3):
            rta.rta_surrogate_infer(tr.model, hil.data_ptr(), img_tel.data_ptr(), wl.n_img, evt_off.data_ptr(),
                                    wl.n_evt, bound, ev.data_ptr(), sp)
        e0.record(stream)
        for _ in range(steps):
            rta.rta_surrogate_infer(tr.model, hil.data_ptr(), img_tel.data_ptr(), wl.n_img, evt_off.data_ptr(),
                                    wl.n_evt, bound, ev.data_ptr(), sp)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    infer_nofb_ms = infer_ms(1e30)
    infer_full_ms = infer_ms(0.5)

    # the non-learned path: image kernel + geometric stereo + lookup tables
    lev = torch.zeros(wl.n_evt * 8, dtype=torch.float32, device=wave.device)
    lut_args = (lookup.data_ptr(), se_d.data_ptr(), len(LUT_SIZE_EDGES) - 1, de_d.data_ptr(),
                len(LUT_DIST_EDGES) - 1, LUT_CUTS, lev.data_ptr(), sp)

    def lut_step():
        rta.rta_image_chain(h, wave.data_ptr(), wave.numel(), wave_off.data_ptr(), img_tel.data_ptr(), wl.n_img,
                            *proc, hil.data_ptr(), sp)
        rta.rta_stereo(h, hil.data_ptr(), img_tel.data_ptr(), wl.n_img, evt_off.data_ptr(), wl.n_evt, ste.data_ptr(), sp)
        rta.rta_lut_reconstruct(h, hil.data_ptr(), img_tel.data_ptr(), wl.n_img, evt_off.data_ptr(), wl.n_evt,
                                ste.data_ptr(), *lut_args)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    lut_path_ms = timed(lut_step)
    # the geometric step timed exactly like the learned one (the same loop, one call per step)
    geo_loop_ms = timed(lambda: rta.rta_reconstruct(h, wave.data_ptr(), wave.numel(), wave_off.data_ptr(),
                                                    img_tel.data_ptr(), wl.n_img, evt_off.data_ptr(), wl.n_evt, *proc,
                                                    hil.data_ptr(), ste.data_ptr(), sp))
    sur_nofb_ms = timed(sur_step_nofb)             # the learned step with the fallback switched off
    sur_ms = timed(sur_step)                       # again, next to it
    lut_ms = timed(lambda: rta.rta_lut_reconstruct(h, hil.data_ptr(), img_tel.data_ptr(), wl.n_img,
                                                   evt_off.data_ptr(), wl.n_evt, ste.data_ptr(), *lut_args))
    stereo_ms = timed(lambda: rta.rta_stereo(h, hil.data_ptr(), img_tel.data_ptr(), wl.n_img, evt_off.data_ptr(),
                                             wl.n_evt, ste.data_ptr(), sp))
    ctx.check(sp)
    le = rta.lut_events_to_numpy(lev.cpu().numpy())
    ok = (le["flags"] & (rta.RTA_LF_NO_CORE | rta.RTA_LF_NO_IMAGE | rta.RTA_LF_MALFORMED)) == 0
    g_b = wl.truth[:, 5] == 0
    d_le = le["log_energy"][ok & g_b] - np.log10(wl.truth[ok & g_b, 0])
    lut_out = {"ms_per_step": lut_path_ms, "events_per_s": wl.n_evt / (lut_path_ms / 1e3), "lut_ms": lut_ms,
               "stereo_ms": stereo_ms, "cuts": list(LUT_CUTS), "filled_cells": int((cells.view(torch.int32)[0::8] >= 10).sum()),
               "accuracy_on_bundle": {"with_energy_frac": float(np.mean(ok[g_b])) if g_b.any() else None,
                                      "energy_bias": float(np.mean(d_le)) if len(d_le) else None,
                                      "energy_res": float(np.std(d_le)) if len(d_le) else None,
                                      "gamma_pass": float(np.mean((le["flags"][ok & g_b] & rta.RTA_LF_GAMMA) != 0))
                                      if (ok & g_b).any() else None},
               "proton_pass_held_out": proton_pass}
    # accuracy on the bundle (gamma showers) against the geometric result of the same images
    rta.rta_stereo(h, hil.data_ptr(), img_tel.data_ptr(), wl.n_img, evt_off.data_ptr(), wl.n_evt, ste.data_ptr(), sp)
    torch.cuda.synchronize()
    res = train.evaluate(rta.events_to_numpy(ev.cpu().numpy()), rta.stereo_to_numpy(ste.cpu().numpy()), wl.truth)
    out = {"ms_per_step": sur_ms, "events_per_s": wl.n_evt / (sur_ms / 1e3),
           "geometric_same_loop_ms_per_step": geo_loop_ms,
           "learned_vs_geometric_events_per_s": geo_loop_ms / sur_ms,
           "ms_per_step_without_fallback": sur_nofb_ms,
           "infer_ms": infer_full_ms, "infer_without_fallback_ms": infer_nofb_ms, "train_events": n_train,
           "held_out_events": n_eval, "train_epochs": epochs, "train_steps": len(losses), "train_s": fit_s,
           "generate_and_reconstruct_s": gen_s, "setup_s": setup_s, "final_loss": float(np.mean(losses[-20:])),
           "held_out": held_out, "held_out_lookup_tables": lut_held_out, "cpu_baseline_forward": cpu_fwd,
           "accuracy_on_bundle": res, "lookup_tables": lut_out}
    return out, tr


def serving_feed(wl, n_events, rng, seg_events=5000, seed0=1307064895):
    """The telescope feed of the serving leg: n_events array events in one pinned
    host buffer, made of segments of seg_events events, each triggered on its own
    random sub-array of 20-69 telescopes (same array and calibration as wl),
    rendered on the GPU (the generator's GPU renderer) and copied out. A bundle
    is any contiguous event range of it, so bundles of 1k-50k events mix
    sub-arrays without copies of their own."""
    import torch
    import synth
    plans, k = [], 0
    while sum(p.n_evt for p in plans) < n_events:
        sub = rng.choice(len(wl.tel_cam), size=int(rng.integers(20, len(wl.tel_cam) + 1)), replace=False)
        plans.append(synth.make_workload(2, min(seg_events, n_events - sum(p.n_evt for p in plans)),
                                         seed=seed0 + 7919 * k, render=False, telescopes=sub, calib_seed=wl.seed))
        k += 1
    feed = feed_layout(plans)
    host = torch.empty(feed["n_samples"], dtype=torch.int16, pin_memory=True)
    dwave = torch.empty(max(p.n_samples_total for p in plans), dtype=torch.int16, device="cuda")
    for p, b0 in zip(plans, feed["seg_base"]):
        keep = synth.render_waves_gpu(p, dwave, torch.cuda.current_stream().cuda_stream)
        host[int(b0):int(b0) + p.n_samples_total].copy_(dwave[:p.n_samples_total])
        torch.cuda.synchronize()
        del keep
    del dwave
    torch.cuda.empty_cache()
    feed.update(host=host, wave=host.numpy().view(np.uint16))
    return feed


def feed_layout(plans):
    """The feed's tables: the segments' images one after another (sample offsets
    from the feed's start, telescopes, event CSR over all of them)."""
    sizes = np.array([p.n_samples_total for p in plans], np.int64)
    base = np.concatenate([[0], np.cumsum(sizes)])
    img_base = np.concatenate([[0], np.cumsum([p.n_img for p in plans])])
    evt_off = [0]
    for p, i0 in zip(plans, img_base[:-1]):
        evt_off.extend((p.evt_off[1:].astype(np.int64) + i0).tolist())
    wave_off = np.concatenate([p.wave_off + b0 for p, b0 in zip(plans, base[:-1])]).astype(np.int64)
    return dict(seg_base=base[:-1], n_samples=int(base[-1]), wave_off=wave_off,
                wave_end=np.append(wave_off[1:], base[-1]),
                img_tel=np.concatenate([p.img_tel for p in plans]).astype(np.int32),
                evt_off=np.asarray(evt_off, np.int64), n_evt=len(evt_off) - 1, segments=len(plans),
                bytes=int(2 * base[-1]))


def feed_bundles(feed, n_bundles, rng, lo=1000, hi=50000):
    """n_bundles contiguous event ranges of the feed, their event counts
    log-uniform in [lo, hi], with the tables a bundle carries (wave offsets from
    its first sample, telescopes, event CSR from 0)."""
    out = []
    hi = min(hi, feed["n_evt"])
    for _ in range(n_bundles):
        n = int(np.exp(rng.uniform(np.log(lo), np.log(hi + 1))))
        n = max(lo, min(hi, n))
        e0 = int(rng.integers(0, feed["n_evt"] - n + 1))
        i0, i1 = int(feed["evt_off"][e0]), int(feed["evt_off"][e0 + n])
        w0, w1 = int(feed["wave_off"][i0]), int(feed["wave_end"][i1 - 1])
        out.append(dict(ptr=feed["wave"][w0:].ctypes.data, n_wave=w1 - w0,
                        off=np.ascontiguousarray(feed["wave_off"][i0:i1] - w0),
                        tel=np.ascontiguousarray(feed["img_tel"][i0:i1]),
                        evt=np.ascontiguousarray(feed["evt_off"][e0:e0 + n + 1] - i0, dtype=np.int32),
                        n_img=i1 - i0, n_evt=n, bytes=2 * (w1 - w0)))
    return out


def arrival_schedule(pool_bytes, rate, duration_s, rng, min_arrivals=8, burst=24):
    """Arrivals [(ns after the start, pool index)] of bundles drawn from a pool at
    an aggregate rate (GB/s). rate = inf: a burst of `burst` bundles at the start.
    Otherwise Poisson arrivals -- exponential gaps, each with the mean its bundle's
    bytes give at this rate -- for at least duration_s and at least min_arrivals
    bundles (so that the low rates' percentiles are not those of one or two), the
    gaps then scaled by one factor so that the schedule offers exactly `rate`: its
    bytes over the time from the start to the last arrival."""
    n = len(pool_bytes)
    if not rate > 0:
        raise ValueError(f"arrival rate {rate} GB/s must be positive")
    if rate == float("inf"):
        return [(0, int(rng.integers(n))) for _ in range(burst)]
    picks, gaps, total = [], [], 0
    while total < rate * 1e9 * duration_s or len(picks) < min_arrivals:
        i = int(rng.integers(n))
        gaps.append(rng.exponential(pool_bytes[i] / (rate * 1e9)))
        picks.append(i)
        total += pool_bytes[i]
    scale = (total / (rate * 1e9)) / sum(gaps)
    out, t = [], 0.0
    for i, g in zip(picks, gaps):
        t += g * scale * 1e9
        out.append((int(t), i))
    return out


def hour_of_sky(st, now_s, rate_hz, rng, flare_xy=(0.31, -0.47), flare_s=20, flare_hz=30):
    """An hour of sky-map history before now_s, second by second, counted in
    through rta_stream_add_events: rate_hz background events a second, uniform
    in a 2.5 deg disk (3 % without a direction), and the last flare_s seconds
    flare_hz more a second in a 0.03 deg Gaussian at flare_xy."""
    import torch
    import paper_1307_6489_gb300 as rta
    cs = torch.cuda.current_stream().cuda_stream
    keep = []
    for t in range(now_s - 3599, now_s + 1):
        n = int(rng.poisson(rate_hz))
        r = 2.5 * np.sqrt(rng.uniform(size=n))
        a = rng.uniform(0, 2 * np.pi, n)
        x, y = r * np.cos(a), r * np.sin(a)
        if t > now_s - flare_s:
            k = int(rng.poisson(flare_hz))
            x = np.concatenate([x, flare_xy[0] + rng.normal(0, 0.03, k)])
            y = np.concatenate([y, flare_xy[1] + rng.normal(0, 0.03, k)])
        rows = np.zeros((len(x), 8), np.float32)
        rows[:, 1], rows[:, 2] = x, y
        rows.view(np.uint32)[:, 5] = np.where(rng.uniform(size=len(x)) < 0.97, 0, rta.RTA_EF_NO_DIRECTION)
        d = torch.from_numpy(rows.reshape(-1)).cuda(non_blocking=False)
        rta.rta_stream_add_events(st, d.data_ptr(), len(x), t * 1_000_000_000 + 250_000_000, cs)
        keep.append(d)
        if len(keep) > 64:
            torch.cuda.synchronize()
            keep.clear()
    torch.cuda.synchronize()


def transient_leg(ctx, proc, rate_hz=10000, seed=1307064896):
    """Transient search over an hour of history (its own stream): the time of one
    call for 1 s .. 30 min windows, and what it finds: the planted flare and any
    other alert."""
    import paper_1307_6489_gb300 as rta
    rng = np.random.default_rng(seed)
    windows = [(1, 5), (5, 25), (10, 20), (60, 600), (300, 1800), (600, 3000), (1800, 1800)]
    now_s = 2_000_000 * 60 + 23
    fx, fy = 0.31, -0.47
    st = rta.rta_stream_create(ctx.handle, 0, 64 << 20, 1, 1000, 1000, *proc, 0.5)
    try:
        t0 = time.perf_counter()
        hour_of_sky(st, now_s, rate_hz, rng, (fx, fy))
        fill_s = time.perf_counter() - t0
        now = now_s * 1_000_000_000 + 999_000_000
        rta.rta_transient_search(st, now, windows, 5, 5.0)          # warm (work buffers)
        t0 = time.perf_counter()
        for _ in range(10):
            alerts, n_found = rta.rta_transient_search(st, now, windows, 5, 5.0, with_total=True)
        search_ms = (time.perf_counter() - t0) / 10 * 1e3
    finally:
        rta.rta_stream_destroy(st)
    cx = (alerts["ix"] + 0.5) * 0.02 - 2.56
    cy = (alerts["iy"] + 0.5) * 0.02 - 2.56
    near = np.hypot(cx - fx, cy - fy) <= 0.15
    return {"history": f"3600 one-second slabs, Poisson {rate_hz} events/s uniform in a 2.5 deg disk, 3 % without "
                       f"direction; a 20 s flare of 30 events/s (0.03 deg Gaussian) at ({fx}, {fy}) deg",
            "fill_s": fill_s, "windows": len(windows), "radius_bins": 5, "s_min": 5.0, "ms_per_call": search_ms,
            "alerts": int(n_found), "flare_alerts": int(near.sum()),
            "flare_windows": sorted({windows[int(w)][0] for w in alerts["window"][near]}),
            "other_alerts": int((~near).sum()),
            "max_significance": float(alerts["significance"].max()) if len(alerts) else None}


def serving_leg(ctx, model, wl, proc, rates, duration_s, feed_events=60000, seed=1307064894):
    """Poisson arrivals of telescope bundles (1k-50k events, contiguous ranges of
    a GPU-rendered feed of mixed sub-arrays) at fixed aggregate rates through the
    serving stream (continuous batching under an HBM budget); per rate the
    sustained GB/s, the arrival-to-event-list latency percentiles and where each
    bundle's time went (queue wait before a slot and memory free up, copies in,
    device work, copy out)."""
    import torch
    import paper_1307_6489_gb300 as rta
    rng = np.random.default_rng(seed)
    feed = serving_feed(wl, feed_events, rng)
    pool = feed_bundles(feed, 64, rng)
    max_img = max(b["n_img"] for b in pool)
    max_evt = max(b["n_evt"] for b in pool)
    budget = 48 << 30
    st = rta.rta_stream_create(ctx.handle, model or 0, budget, 4, max_img, max_evt, *proc, 0.5)
    pct = lambda a, q: float(np.percentile(a, q)) if len(a) else None
    out = []
    try:
        # the offered rates, then a burst of 48 small bundles (1k-2k events) submitted at once,
        # where copies finish close together and the device queue hands several to one pass
        small = feed_bundles(feed, 48, rng, lo=1000, hi=2000)
        for rate in list(rates) + ["small_burst"]:
            t_start = time.monotonic_ns() + 50_000_000
            if rate == "small_burst":
                sched = [(t_start, b) for b in small]
            else:
                sched = [(t_start + dt, pool[i]) for dt, i in arrival_schedule([b["bytes"] for b in pool], rate,
                                                                               duration_s, rng, min_arrivals=6)]
            total = sum(b["bytes"] for _, b in sched)
            ev_all = torch.empty(sum(b["n_evt"] for _, b in sched) * 32, dtype=torch.uint8, pin_memory=True)
            ev_np = ev_all.numpy()
            pos, structs, tickets, arr = 0, [], [], []
            for t_arr, b in sched:
                bs = rta.Bundle(b["ptr"], b["n_wave"], b["off"].ctypes.data, b["tel"].ctypes.data,
                                b["n_img"], b["evt"].ctypes.data, b["n_evt"], t_arr, ev_np[pos:].ctypes.data)
                pos += b["n_evt"] * 32
                structs.append(bs)
            done = {}
            k = 0
            while len(done) < len(sched):
                now = time.monotonic_ns()
                while k < len(sched) and sched[k][0] <= now:
                    tickets.append(rta.rta_stream_submit(st, structs[k]))
                    arr.append(sched[k][0])
                    k += 1
                for j, tk in enumerate(tickets):
                    if j not in done:
                        d = rta.rta_stream_poll_times(st, tk)
                        if d is not None:
                            done[j] = d
                time.sleep(0.0002)
            T = [done[j] for j in range(len(sched))]
            lat = np.array([(t.done_ns - t.arrival_ns) / 1e6 for t in T])
            qwait = np.array([(t.admit_ns - t.arrival_ns) / 1e6 for t in T])
            h2d = np.array([t.h2d_ms for t in T])
            comp = np.array([t.compute_ms for t in T])
            d2h = np.array([t.d2h_ms for t in T])
            rwait = np.array([t.ready_wait_ms for t in T])
            per_pass = np.array([t.batch_bundles for t in T])
            nbytes = np.array([b["bytes"] for _, b in sched], np.float64)
            span = (max(t.done_ns for t in T) - t_start) / 1e9
            slowest = int(np.argmax(lat))
            out.append({"rate_gbs": rate if rate != float("inf") else "burst", "bundles": len(sched),
                        "bytes": int(total), "events": int(sum(b["n_evt"] for _, b in sched)),
                        "offered_gbs": (total / ((arr[-1] - t_start) / 1e9) / 1e9) if arr[-1] > t_start else None,
                        "sustained_gbs": total / span / 1e9, "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
                        "max_ms": float(lat.max()),
                        "queue_wait_ms": {"p50": pct(qwait, 50), "p99": pct(qwait, 99), "max": float(qwait.max())},
                        "h2d_ms": {"p50": pct(h2d, 50), "p99": pct(h2d, 99), "max": float(h2d.max()),
                                   "gbs_median": float(np.median(nbytes / (h2d * 1e6)))},
                        # the device queue: how long published data waited for a pass, and the pass
                        # (all bundles it took) each bundle was reconstructed in
                        "ready_wait_ms": {"p50": pct(rwait, 50), "p99": pct(rwait, 99), "max": float(rwait.max())},
                        "bundles_per_pass": {"mean": float(per_pass.mean()), "max": int(per_pass.max())},
                        "pass_device_ms": {"p50": pct(comp, 50), "p99": pct(comp, 99), "max": float(comp.max())},
                        "pass_output_ms": {"p50": pct(d2h, 50), "max": float(d2h.max())},
                        "slowest": {"events": int(sched[slowest][1]["n_evt"]), "gb": float(nbytes[slowest] / 1e9),
                                    "latency_ms": float(lat[slowest]), "queue_wait_ms": float(qwait[slowest]),
                                    "h2d_ms": float(h2d[slowest]), "ready_wait_ms": float(rwait[slowest]),
                                    "pass_device_ms": float(comp[slowest]),
                                    "bundles_in_pass": int(per_pass[slowest])}})
            del ev_all
    finally:
        rta.rta_stream_destroy(st)
    info = {"feed_events": feed["n_evt"], "feed_gb": feed["bytes"] / 1e9, "feed_segments": feed["segments"],
            "bundle_events": {"min": min(b["n_evt"] for b in pool), "median": int(np.median([b["n_evt"] for b in pool])),
                              "max": max(b["n_evt"] for b in pool)},
            "bundle_gb_max": max(b["bytes"] for b in pool) / 1e9, "hbm_budget_gb": budget / 2**30, "slots": 4}
    del feed
    return out, info


def run_reference(args, ws, rank):
    """The reference arm of this build is the CPU oracle, timed on the host cores."""
    if rank != 0:
        return
    import oracle
    import synth
    wl = synth.make_workload(2, args.events, seed=synth.BASE_SEED + 2)
    cores = os.cpu_count() or 1
    per_step = max(8, min(wl.n_evt, args.ref_events))
    rng = np.random.default_rng(0)
    times = []
    for k in range(args.warmup + args.steps):
        ev = np.sort(rng.choice(wl.n_evt, per_step, replace=False))
        sub = synth.subset(wl, ev)
        t0 = time.perf_counter()
        oracle.reconstruct(sub, threads=cores)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = per_step / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u16->f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + f"; each step {per_step} random events of it", "events": args.events,
                       "preset": 2},
            "cpu_baseline": {"value": value, "unit": "events/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} random events per step"},
            "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--events", type=int, default=10000)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-events", type=int, default=300)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=0, help="steps of the host-buffer leg (default: --steps)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-stream", action="store_true")
    ap.add_argument("--train-events", type=int, default=2000000)
    ap.add_argument("--eval-events", type=int, default=1000000)
    ap.add_argument("--train-epochs", type=int, default=0,
                    help="epochs of the surrogate's training (default: about 6,000 Adam steps)")
    ap.add_argument("--serve-rates", default="0.5,2,8,inf", help="aggregate arrival rates, GB/s (inf: a burst)")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--chain", default="", help="fixed image-kernel config 'variant,stages,ctas_per_sm'")
    ap.add_argument("--config1-events", type=int, default=200000,
                    help="events of the single-camera stream leg (1855 px x 40 samples; 0: skip)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if ws > 1:
        # several ranks measure the step's scaling: the single-GPU legs (learned path with its
        # training, serving, DL0 stream, the single-camera configurations) run only at N = 1
        args.no_surrogate = args.no_serving = args.no_stream = True
        args.config1_events = 0

    import torch
    import torch.distributed as dist

    import paper_1307_6489_gb300 as rta
    import synth

    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wl, host = make_bundle(args.events, rank_seed(rank), pinned=True)
    wave_h = host.numpy().view(np.uint16)

    ctx = rta.Context(local, hbm_budget_bytes=8 << 30)
    for c, cam in wl.cams.items():
        ctx.register_camera(c, cam.xy, cam.nb, cam.n_samples)
    ctx.register_array(wl.tel_cam, wl.tel_xy, wl.p16, wl.scale)
    p = wl.proc
    mode = rta.RTA_WINDOW_SLIDING if p.sliding else rta.RTA_WINDOW_FIXED
    proc = (mode, p.start, p.W, p.t_hi, p.t_lo, p.core_needs_neighbour)
    dev = torch.device("cuda", local)
    wave = host.to(dev)
    wave_off = torch.from_numpy(wl.wave_off).to(dev)
    img_tel = torch.from_numpy(wl.img_tel).to(dev)
    evt_off = torch.from_numpy(wl.evt_off).to(dev)
    hil = torch.zeros(wl.n_img * 16, dtype=torch.float32, device=dev)
    ste = torch.zeros(wl.n_evt * 8, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    h = ctx.handle
    nw = wave.numel()

    # the project's autotuner picks the fused kernel's tile shape, pipeline depth and
    # CTAs/SM on this bundle (setup, outside the timed region)
    tune = []
    if not args.no_autotune:
        tune = rta.rta_autotune(h, wave.data_ptr(), wave.numel(), wave_off.data_ptr(), img_tel.data_ptr(), wl.n_img,
                                *proc, hil.data_ptr(), reps=2, stream=sp)
        if rank == 0:
            for e in sorted(tune, key=lambda e: e["ms"])[:12]:
                print("autotune", json.dumps(e), file=sys.stderr)
    if args.chain:
        v, ns, cps = (int(x) for x in args.chain.split(","))
        ctx.set_chain_config(v, ns, cps)

    def step():
        rta.rta_reconstruct(h, wave.data_ptr(), nw, wave_off.data_ptr(), img_tel.data_ptr(), wl.n_img,
                            evt_off.data_ptr(), wl.n_evt, *proc, hil.data_ptr(), ste.data_ptr(), sp)

    for _ in range(args.warmup):
        step()
    ctx.check(sp)

    # ---------------- timed region (device-resident inputs; 5+ GB per bundle >> 129 MB L2)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)   # let the sampler start before the timed region
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        # one step: rta_reconstruct (image kernel, then the stereo kernel as its programmatic
        # dependent, with nothing between them on the stream)
        rta.rta_reconstruct(h, wave.data_ptr(), nw, wave_off.data_ptr(), img_tel.data_ptr(), wl.n_img,
                            evt_off.data_ptr(), wl.n_evt, *proc, hil.data_ptr(), ste.data_ptr(), sp)
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    if ws > 1:
        dist.barrier()
    # the same steps with events around each kernel: the kernels' own durations (the events
    # between the kernels cost the stereo kernel its early launch, so these steps are slower)
    for k in range(args.steps):
        e0, e1, e2 = ev[k]
        e0.record(stream)
        rta.rta_image_chain(h, wave.data_ptr(), nw, wave_off.data_ptr(), img_tel.data_ptr(), wl.n_img, *proc,
                            hil.data_ptr(), sp)
        e1.record(stream)
        rta.rta_stereo(h, hil.data_ptr(), img_tel.data_ptr(), wl.n_img, evt_off.data_ptr(), wl.n_evt, ste.data_ptr(),
                       sp)
        e2.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ctx.check(sp)
    total_ms = t_start.elapsed_time(t_end)
    chain_ms = [a.elapsed_time(b) for a, b, _ in ev]
    stereo_ms = [b.elapsed_time(c) for _, b, c in ev]
    total_ms = max_over_ranks(total_ms, ws, dev)
    ms_per_step = total_ms / args.steps
    events_all = wl.n_evt * ws
    value = job_rate(wl.n_evt, ws, ms_per_step / 1e3)

    # ---------------- the same step launched as one CUDA graph (captured at capacity)
    n_img_d = torch.tensor([wl.n_img], dtype=torch.int64, device=dev)
    n_evt_d = torch.tensor([wl.n_evt], dtype=torch.int64, device=dev)
    graph = rta.rta_graph_create(h, wave.data_ptr(), nw, wave_off.data_ptr(), img_tel.data_ptr(), n_img_d.data_ptr(),
                                 wl.n_img, evt_off.data_ptr(), n_evt_d.data_ptr(), wl.n_evt, *proc, hil.data_ptr(),
                                 ste.data_ptr())
    for _ in range(3):
        rta.rta_graph_launch(graph, sp)
    torch.cuda.synchronize(dev)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(args.steps):
        rta.rta_graph_launch(graph, sp)
    g1.record(stream)
    torch.cuda.synchronize(dev)
    graph_ms = g0.elapsed_time(g1) / args.steps
    rta.rta_graph_destroy(graph)
    ctx.check(sp)

    # ---------------- the digital-filter-style extractor on the same bundle (image kernel alone)
    # weights summing to W, so that the registered (flat-window) calibration
    # normalises the filter and the cleaning sees charges of the same scale
    filt_w = (0, 1, 2, 2, 1, 0)
    filt_ms = None
    if proc[2] == len(filt_w) and proc[0] != rta.RTA_WINDOW_FIXED:
        rta.rta_set_filter_weights(h, filt_w)
        fproc = (rta.RTA_WINDOW_FILTER,) + tuple(proc[1:])
        fhil = torch.empty_like(hil)
        for _ in range(3):
            rta.rta_image_chain(h, wave.data_ptr(), nw, wave_off.data_ptr(), img_tel.data_ptr(), wl.n_img, *fproc,
                                fhil.data_ptr(), sp)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            rta.rta_image_chain(h, wave.data_ptr(), nw, wave_off.data_ptr(), img_tel.data_ptr(), wl.n_img, *fproc,
                                fhil.data_ptr(), sp)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        filt_ms = f0.elapsed_time(f1) / args.steps
        ctx.check(sp)

    # ---------------- the neighbour-peak window on the same bundle (image kernel alone; its own
    # launch configuration, tuned by the autotuner in this mode outside the timed region)
    nbp_ms = None
    if proc[0] != rta.RTA_WINDOW_FIXED:
        nproc = (rta.RTA_WINDOW_NEIGHBOUR,) + tuple(proc[1:])
        nhil = torch.empty_like(hil)
        if not args.no_autotune and not args.chain:
            rta.rta_autotune(h, wave.data_ptr(), nw, wave_off.data_ptr(), img_tel.data_ptr(), wl.n_img, *nproc,
                             nhil.data_ptr(), reps=2, stream=sp)
        for _ in range(3):
            rta.rta_image_chain(h, wave.data_ptr(), nw, wave_off.data_ptr(), img_tel.data_ptr(), wl.n_img, *nproc,
                                nhil.data_ptr(), sp)
        n0, n1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0.record(stream)
        for _ in range(args.steps):
            rta.rta_image_chain(h, wave.data_ptr(), nw, wave_off.data_ptr(), img_tel.data_ptr(), wl.n_img, *nproc,
                                nhil.data_ptr(), sp)
        n1.record(stream)
        torch.cuda.synchronize(dev)
        nbp_ms = n0.elapsed_time(n1) / args.steps
        ctx.check(sp)
        del nhil

    # ---------------- roofline of the dominant kernel (fused image kernel)
    hbm_peak, peak_kind = peaks()
    alg_bytes = wl.wave_bytes + wl.n_img * HILLAS_BYTES
    chain_avg = statistics.mean(chain_ms)
    achieved = alg_bytes / (chain_avg / 1e3) / 1e9
    traffic = None
    prof = os.path.join(ROOT, "profiles", "image_chain_traffic.json")
    if os.path.exists(prof):
        try:
            tj = json.load(open(prof))
            if tj.get("kernel_hash") == _kernel_hash():
                traffic = tj["bytes_per_image"] * wl.n_img
        except Exception:
            traffic = None

    # ---------------- end to end through the host-buffer call
    e2e_steps = args.e2e_steps or args.steps
    hh = np.zeros(wl.n_img * 16, np.float32)
    hs = np.zeros(wl.n_evt * 8, np.float32)
    woff = np.ascontiguousarray(wl.wave_off)
    itel = np.ascontiguousarray(wl.img_tel)
    eoff = np.ascontiguousarray(wl.evt_off)
    ctx.reconstruct_host(wave_h, woff, itel, eoff, *proc, hh, hs)   # warm (allocates staging)
    if ws > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.reconstruct_host(wave_h, woff, itel, eoff, *proc, hh, hs)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, ws, dev)
    assert np.array_equal(hh.view(np.uint32), hil.cpu().numpy().view(np.uint32)), "host path differs"
    h2d = wl.wave_bytes + wl.n_img * 12 + (wl.n_evt + 1) * 4
    d2h = wl.n_img * HILLAS_BYTES + wl.n_evt * STEREO_BYTES

    # ---------------- the learned path (setup: training) and the serving loop
    sur, trainer, serving, pool_info = None, None, None, None
    if not args.no_surrogate:
        sur, trainer = surrogate_leg(ctx, wl, (wave, wave_off, img_tel, evt_off, hil, ste), proc, stream, args.steps,
                                     args.train_events, args.eval_events, args.train_epochs)
    if not args.no_serving:
        rates = [float(r) for r in args.serve_rates.split(",")]
        serving, pool_info = serving_leg(ctx, trainer.model if trainer else None, wl, proc, rates,
                                         args.serve_seconds)
        pool_info["transient_search"] = transient_leg(ctx, proc)
    if trainer:
        trainer.close()

    # ---------------- the DL0 byte stream: ingest and the zero-copy reconstruction (last:
    # its pinned and device copies of the stream stay out of the serving measurement)
    stream_out = None
    if not args.no_stream:
        stream_out = stream_leg(ctx, wl, proc, stream, args.steps, e2e_steps, hil, ste,
                                tune=not args.no_autotune)
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl)

    # ---------------- the single large camera streamed from host memory (last: ~30 GB pinned)
    cfg1 = None
    if args.config1_events > 0:
        del host, wave_h
        torch.cuda.empty_cache()
        cfg1 = config1_leg(args.config1_events, hbm_peak, args.steps, local)
    cfg0 = config0_leg(args.steps, local) if ws == 1 else None

    if rank == 0:
        cfg = ctx.chain_config()
        line = {
            "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u16->int32/f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "events_per_bundle": wl.n_evt, "images_per_bundle": wl.n_img,
                       "bundle_bytes": wl.wave_bytes, "mean_multiplicity": wl.n_img / wl.n_evt,
                       "l2": "inputs larger than L2 (bundle >> 129 MB), no flush",
                       "chain": cfg, "paper_context": PAPER_RATE,
                       "autotune": {"configs_measured": len(tune),
                                    "best_ms": min((e["ms"] for e in tune), default=None),
                                    "worst_ms": max((e["ms"] for e in tune), default=None)}},
            "gbs": wl.wave_bytes * ws / (ms_per_step / 1e3) / 1e9,
            "gbs_vs_hbm_peak": wl.wave_bytes / (ms_per_step / 1e3) / 1e9 / hbm_peak,
            "kernel_ms": {"image_chain": chain_avg, "stereo": statistics.mean(stereo_ms)},
            "extractors": {"sliding_window_ms": chain_avg, "digital_filter_ms": filt_ms, "filter_weights": list(filt_w),
                           "digital_filter_hbm_frac": (alg_bytes / (filt_ms / 1e3) / 1e9 / hbm_peak
                                                       if filt_ms else None),
                           "neighbour_peak_ms": nbp_ms,
                           "neighbour_peak_hbm_frac": (alg_bytes / (nbp_ms / 1e3) / 1e9 / hbm_peak
                                                       if nbp_ms else None)},
            "graph": {"ms_per_step": graph_ms, "events_per_s": events_all / (graph_ms / 1e3)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": "k_image_chain", "algorithmic_bytes_per_launch": alg_bytes},
            "e2e": {"value": events_all / e2e_s, "unit": "events/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "gbs": wl.wave_bytes * ws / e2e_s / 1e9,
                    "call": "rta_reconstruct_host (pinned host bundle)"},
            "paths": {"geometric": {"ms_per_step": ms_per_step, "events_per_s": wl.n_evt / (ms_per_step / 1e3)},
                      "surrogate": sur},
            "dl0_stream": stream_out,
            "single_camera_stream": cfg1,
            "single_camera_small": cfg0,
            "serving": {"rates": serving, "feed": pool_info,
                        "model": "surrogate" if trainer else "geometric"} if serving else None,
            "p99_bundle_latency_ms": next((r["p99_ms"] for r in serving if r["rate_gbs"] == 8.0), None)
            if serving else None,
            "gpu_launches": 2 * args.steps,   # timed region: k_image_chain + k_stereo per step
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(_finite(line)), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


def _finite(x):
    """NaN and infinities become null (strict JSON)."""
    if isinstance(x, float):
        return x if np.isfinite(x) else None
    if isinstance(x, dict):
        return {k: _finite(v) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [_finite(v) for v in x]
    return x


def _kernel_hash():
    import hashlib
    h = hashlib.sha1()
    for f in sorted(os.listdir(os.path.join(ROOT, "paper_1307_6489_gb300", "csrc"))):
        if f in ("k_image.cu", "k_image_lean.cu", "k_image_chain.cuh", "rta_device.cuh"):
            h.update(open(os.path.join(ROOT, "paper_1307_6489_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


if __name__ == "__main__":
    main()
