"""Seeded synthetic inputs (cameras, array, calibration table, showers, waveforms).

Input generation only: nothing here computes any step of the reconstruction.
The CUDA library and the CPU oracle both consume these arrays.  The C source
(``synth.c``) is compiled in-tree into ``libsynth.so`` on first use.

Workload presets (the paper gives requirements, not data; these stand in for
the Prod2 simulations its assessment used, Sec. 5):

  0  one 16x16 square camera (0.1 deg), 16 samples, sizes log-U(50, 5000) pe,
     fixed 5-sample window at samples 4..8, tailcut 10/5 pe, no neighbour test
  1  one 1855-pixel hexagonal camera (0.1 deg), 40 samples, sizes
     log-U(30, 20000) pe, sliding 6-sample max-sum, tailcut 8/4 + neighbour test
  2  the 69-telescope array (4 x 1855 px / 40 samples, 15 x 1764 px / 30,
     50 x 2048 px / 25), gamma showers E^-2.5 on 0.03-100 TeV, multiplicity
     2-40, processing as preset 1
  3  preset 2 with half proton-like showers (for the learned reconstruction)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None

BASE_SEED = 1307064890
N_CAM = 4
CAM_NAMES = {0: "square256", 1: "large1855", 2: "medium1764", 3: "small2048"}


def build(force: bool = False) -> str:
    """Compile libsynth.so in-tree (gcc, a few seconds)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, u64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        lib.synth_lattice.argtypes = [i32, i32, f64, i32, P, P]
        lib.synth_camera_info.argtypes = [i32, P, P]
        lib.synth_camera.argtypes = [i32, P, P]
        lib.synth_array.argtypes = [P, P]
        lib.synth_window_fraction.argtypes = [i32, i32, i32]
        lib.synth_window_fraction.restype = f64
        lib.synth_calibration.argtypes = [u64, i32, P, P, f64, P, P, P, P]
        lib.synth_plan_single.argtypes = [u64, i64, f64, f64, P, P]
        lib.synth_plan_array.argtypes = [u64, i64, f64, i32, P, P, i64, P, P, P, P, P]
        lib.synth_plan_array.restype = i64
        lib.synth_render.argtypes = [u64, i64, P, P, P, P, P, P, P, P, P, P, P, i32, i32]
        lib.synth_test_uniforms.argtypes = [u64, i32, P]
        lib.synth_test_normals.argtypes = [u64, i32, P]
        lib.synth_test_poisson.argtypes = [u64, f64, i32, P]
        lib.synth_philox_block.argtypes = [P, P, P]
        lib.synth_crc16.argtypes = [P, i64]
        lib.synth_crc16.restype = ctypes.c_uint16
        lib.synth_write_stream.argtypes = [i64, P, P, P, P, P, P, P, P, P, P, P, P, P, P, i32]
        _lib = lib
    return _lib


_GPU_SRC = os.path.join(_HERE, "synth_gpu.cu")
_GPU_LIB = os.path.join(_HERE, "libsynth_gpu.so")
_gpu_lib = None


def build_gpu(force: bool = False) -> str:
    """Compile libsynth_gpu.so in-tree (nvcc, sm_103a): the GPU renderer for bulk inputs."""
    if force or not os.path.exists(_GPU_LIB) or os.path.getmtime(_GPU_LIB) < os.path.getmtime(_GPU_SRC):
        tmp = _GPU_LIB + f".tmp{os.getpid()}"
        subprocess.check_call([os.environ.get("NVCC", "nvcc"), "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                               "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-o", tmp, _GPU_SRC])
        os.replace(tmp, _GPU_LIB)
    return _GPU_LIB


class _RenderGpuArgs(ctypes.Structure):
    P = ctypes.c_void_p
    _fields_ = [("seed", ctypes.c_uint64), ("n_img", ctypes.c_int64), ("img_evt", P), ("img_tel", P),
                ("tel_cam", P), ("tel_pix_off", P), ("ped", P), ("gain", P), ("ell", P), ("n_ell", P),
                ("cam_xy", P * 16), ("cam_pix", ctypes.c_int * 16), ("cam_samp", ctypes.c_int * 16),
                ("cam_area", ctypes.c_float * 16), ("wave_off", P), ("wave", P), ("inv_norm", ctypes.c_float)]


def _GL():
    global _gpu_lib
    if _gpu_lib is None:
        build_gpu()
        lib = ctypes.CDLL(_GPU_LIB)
        lib.synth_render_gpu.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
        if lib.synth_render_gpu_args_size() != ctypes.sizeof(_RenderGpuArgs):
            raise RuntimeError("libsynth_gpu argument block does not match")
        _gpu_lib = lib
    return _gpu_lib


def render_waves_gpu(wl: "Workload", d_wave, stream: int = 0):
    """Render the workload's waveforms on the GPU into the device buffer d_wave (a
    torch CUDA tensor of at least n_samples_total 16-bit values), asynchronously on
    `stream`. The same model and random streams as render_waves, in FP32: the
    samples follow the same distributions but are not equal to the host
    renderer's bit for bit (bulk training and evaluation sets only; parity tests
    use render_waves). Returns the tensors the kernel reads, which must stay alive
    until it has run."""
    import torch
    dev = d_wave.device
    assert d_wave.numel() >= wl.n_samples_total and d_wave.element_size() == 2
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(dev, non_blocking=False)
    keep = [t(wl.img_evt, np.int32), t(wl.img_tel, np.int32), t(wl.tel_cam, np.int32), t(wl.tel_pix_off, np.int64),
            t(wl.ped, np.float32), t(wl.gain, np.float32), t(wl.ell.reshape(len(wl.img_tel), -1), np.float32),
            t(wl.n_ell, np.int32), t(wl.wave_off, np.int64)]
    a = _RenderGpuArgs()
    a.seed = wl.seed
    a.n_img = wl.n_img
    a.img_evt, a.img_tel, a.tel_cam, a.tel_pix_off, a.ped, a.gain, a.ell, a.n_ell, a.wave_off = \
        [k.data_ptr() for k in keep]
    for c, cam in wl.cams.items():
        xy = t(cam.xy, np.float32)
        keep.append(xy)
        a.cam_xy[c] = xy.data_ptr()
        a.cam_pix[c] = cam.n_pix
        a.cam_samp[c] = cam.n_samples
        a.cam_area[c] = cam.pix_area
    a.wave = d_wave.data_ptr()
    k = np.arange(-60, 61, dtype=np.float64)
    a.inv_norm = float(1.0 / np.exp(-k * k / (2 * 1.5 * 1.5)).sum())
    rc = _GL().synth_render_gpu(ctypes.byref(a), int(min(wl.n_img, 1 << 20)), stream)
    if rc != 0:
        raise RuntimeError(f"synth_render_gpu failed: CUDA error {rc}")
    return keep


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# cameras and array
# --------------------------------------------------------------------------
@dataclass
class Camera:
    cam_id: int
    n_pix: int
    n_samples: int
    K: int
    pitch: float
    pix_area: float
    mirror_area: float
    xy: np.ndarray  # (P, 2) float32, degrees
    nb: np.ndarray  # (P, K) int16, -1 padded


_cam_cache: dict = {}


def camera(cam_id: int) -> Camera:
    if cam_id in _cam_cache:
        return _cam_cache[cam_id]
    lib = _L()
    info = np.zeros(4, np.int32)
    finfo = np.zeros(3, np.float64)
    if lib.synth_camera_info(cam_id, _p(info), _p(finfo)) != 0:
        raise ValueError(f"unknown camera id {cam_id}")
    P, S, K = int(info[0]), int(info[1]), int(info[2])
    xy = np.zeros((P, 2), np.float32)
    nb = np.zeros((P, K), np.int16)
    if lib.synth_camera(cam_id, _p(xy), _p(nb)) != 0:
        raise RuntimeError("synth_camera failed")
    cam = Camera(cam_id, P, S, K, float(finfo[0]), float(finfo[1]), float(finfo[2]), xy, nb)
    _cam_cache[cam_id] = cam
    return cam


def lattice(kind: str, n_pix: int, pitch: float):
    """Pixel centres and neighbour table of a custom lattice ('grid', 'hex', 'square')."""
    k = {"grid": 0, "hex": 1, "square": 2}[kind]
    K = 6 if kind == "hex" else 4
    xy = np.zeros((n_pix, 2), np.float32)
    nb = np.zeros((n_pix, K), np.int16)
    if _L().synth_lattice(k, n_pix, pitch, K, _p(xy), _p(nb)) != 0:
        raise ValueError("bad lattice arguments")
    return xy, nb


def array_layout():
    tel_cam = np.zeros(128, np.int32)
    tel_xy = np.zeros((128, 2), np.float32)
    n = _L().synth_array(_p(tel_cam), _p(tel_xy))
    return tel_cam[:n].copy(), tel_xy[:n].copy()


def window_fraction(sliding: bool, start: int, W: int) -> float:
    return float(_L().synth_window_fraction(int(sliding), int(start), int(W)))


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
@dataclass
class Processing:
    """Per-workload processing parameters (window and tailcut). weights: integer
    weights of the digital-filter-style charge over the sliding window (None:
    the flat window sum). nbpeak: the neighbour-peak window (a pixel takes the
    window of the brightest pixel of its closed neighbourhood)."""
    sliding: bool
    start: int
    W: int
    t_hi: float
    t_lo: float
    core_needs_neighbour: bool
    weights: tuple = None
    nbpeak: bool = False


PRESET_PROCESSING = {
    0: Processing(False, 4, 5, 10.0, 5.0, False),
    1: Processing(True, 0, 6, 8.0, 4.0, True),
    2: Processing(True, 0, 6, 8.0, 4.0, True),
    3: Processing(True, 0, 6, 8.0, 4.0, True),
}


@dataclass
class Workload:
    preset: int
    seed: int
    proc: Processing
    cams: dict                 # cam id -> Camera
    tel_cam: np.ndarray        # (n_tel,) int32
    tel_xy: np.ndarray         # (n_tel, 2) float32, metres
    tel_pix_off: np.ndarray    # (n_tel + 1,) int64: calibration row of each telescope's pixel 0
    ped: np.ndarray            # truth, float64 per calibration row
    gain: np.ndarray
    p16: np.ndarray            # int32 per calibration row
    scale: np.ndarray          # float32 per calibration row
    evt_off: np.ndarray        # (n_evt + 1,) int32 CSR of images per event
    img_tel: np.ndarray        # (n_img,) int32
    img_evt: np.ndarray        # (n_img,) int32
    wave_off: np.ndarray       # (n_img,) int64, sample offset of each image
    pix_off: np.ndarray        # (n_img + 1,) int64, pixel offset of each image
    ell: np.ndarray            # (n_img, 3, 6) float32 generated ellipses
    n_ell: np.ndarray          # (n_img,) int32
    truth: np.ndarray          # (n_evt, 8) float64
    wave: np.ndarray | None = None  # flat uint16
    extra: dict = field(default_factory=dict)

    @property
    def n_evt(self) -> int:
        return len(self.evt_off) - 1

    @property
    def n_img(self) -> int:
        return len(self.img_tel)

    @property
    def n_samples_total(self) -> int:
        return int(self.pix_off_samples()[-1])

    def pix_off_samples(self) -> np.ndarray:
        P = np.array([self.cams[int(self.tel_cam[t])].n_pix for t in self.img_tel], np.int64)
        S = np.array([self.cams[int(self.tel_cam[t])].n_samples for t in self.img_tel], np.int64)
        return np.concatenate([[0], np.cumsum(P * S)])

    @property
    def wave_bytes(self) -> int:
        return 2 * self.n_samples_total

    def image_wave(self, i: int) -> np.ndarray:
        cam = self.cams[int(self.tel_cam[self.img_tel[i]])]
        o = int(self.wave_off[i])
        return self.wave[o:o + cam.n_pix * cam.n_samples].reshape(cam.n_pix, cam.n_samples)

    def image_calib(self, i: int):
        t = int(self.img_tel[i])
        a, b = int(self.tel_pix_off[t]), int(self.tel_pix_off[t + 1])
        return self.p16[a:b], self.scale[a:b]

    def image_cam(self, i: int) -> Camera:
        return self.cams[int(self.tel_cam[self.img_tel[i]])]


def _calibration(seed, tel_cam, proc: Processing, cams):
    n_tel = len(tel_cam)
    npix = np.array([cams[int(c)].n_pix for c in tel_cam], np.int64)
    tel_pix_off = np.concatenate([[0], np.cumsum(npix)]).astype(np.int64)
    rows = int(tel_pix_off[-1])
    ped = np.zeros(rows, np.float64)
    gain = np.zeros(rows, np.float64)
    p16 = np.zeros(rows, np.int32)
    scale = np.zeros(rows, np.float32)
    f = window_fraction(proc.sliding, proc.start, proc.W)
    tc = np.ascontiguousarray(tel_cam, np.int32)
    if _L().synth_calibration(seed, n_tel, _p(tc), _p(tel_pix_off), f, _p(ped), _p(gain), _p(p16), _p(scale)) != 0:
        raise RuntimeError("synth_calibration failed")
    return tel_pix_off, ped, gain, p16, scale


def make_workload(preset: int, n_events: int, seed: int | None = None, *, render: bool = True,
                  threads: int | None = None, wave_out: np.ndarray | None = None, flags: int = 0,
                  proton_frac: float | None = None, telescopes=None, calib_seed: int | None = None) -> Workload:
    """Plan (and optionally render) ``n_events`` events of a preset.

    ``wave_out`` may supply the destination buffer (e.g. a pinned host array) of
    at least the workload's sample count; ``flags`` bit0 turns off electronic
    noise and bit1 turns off night-sky background (used by tests);
    ``telescopes`` (array presets) restricts triggering to a sub-array of
    telescope ids (the calibration table still covers the whole array);
    ``calib_seed`` draws pedestals and gains from another seed, e.g. to make
    more events for the same physical array as an earlier workload."""
    if preset not in PRESET_PROCESSING:
        raise ValueError(f"unknown preset {preset}")
    seed = BASE_SEED + preset if seed is None else int(seed)
    proc = PRESET_PROCESSING[preset]
    lib = _L()
    if preset in (0, 1):
        cam_id = 0 if preset == 0 else 1
        cams = {cam_id: camera(cam_id)}
        tel_cam = np.array([cam_id], np.int32)
        tel_xy = np.zeros((1, 2), np.float32)
        lo, hi = (50.0, 5000.0) if preset == 0 else (30.0, 20000.0)
        ell = np.zeros((n_events, 3, 6), np.float32)
        n_ell = np.zeros(n_events, np.int32)
        lib.synth_plan_single(seed, n_events, lo, hi, _p(ell), _p(n_ell))
        evt_off = np.arange(n_events + 1, dtype=np.int32)
        img_tel = np.zeros(n_events, np.int32)
        truth = np.zeros((n_events, 8), np.float64)
        truth[:, 6] = 1
    else:
        tel_cam, tel_xy = array_layout()
        cams = {c: camera(c) for c in (1, 2, 3)}
        pf = (0.0 if preset == 2 else 0.5) if proton_frac is None else float(proton_frac)
        max_img = n_events * 40
        evt_off = np.zeros(n_events + 1, np.int32)
        img_tel = np.zeros(max_img, np.int32)
        ell = np.zeros((max_img, 3, 6), np.float32)
        n_ell = np.zeros(max_img, np.int32)
        truth = np.zeros((n_events, 8), np.float64)
        sub = np.arange(len(tel_cam)) if telescopes is None else np.asarray(sorted(set(int(t) for t in telescopes)))
        sub_cam = np.ascontiguousarray(tel_cam[sub], np.int32)
        sub_xy = np.ascontiguousarray(tel_xy[sub], np.float32)
        n_img = lib.synth_plan_array(seed, n_events, pf, len(sub), _p(sub_cam), _p(sub_xy), max_img,
                                     _p(evt_off), _p(img_tel), _p(ell), _p(n_ell), _p(truth))
        if n_img < 0:
            raise RuntimeError("synth_plan_array failed")
        img_tel = sub[img_tel[:n_img]].astype(np.int32)
        ell = ell[:n_img].copy()
        n_ell = n_ell[:n_img].copy()
    tel_pix_off, ped, gain, p16, scale = _calibration(seed if calib_seed is None else int(calib_seed), tel_cam, proc,
                                                      cams)
    img_evt = np.repeat(np.arange(len(evt_off) - 1, dtype=np.int32), np.diff(evt_off)).astype(np.int32)
    P = np.array([cams[int(tel_cam[t])].n_pix for t in img_tel], np.int64)
    S = np.array([cams[int(tel_cam[t])].n_samples for t in img_tel], np.int64)
    wave_off = np.concatenate([[0], np.cumsum(P * S)[:-1]]).astype(np.int64) if len(P) else np.zeros(0, np.int64)
    pix_off = np.concatenate([[0], np.cumsum(P)]).astype(np.int64)
    wl = Workload(preset, seed, proc, cams, tel_cam, tel_xy, tel_pix_off, ped, gain, p16, scale, evt_off,
                  img_tel, img_evt, wave_off, pix_off, ell, n_ell, truth)
    if render:
        render_waves(wl, threads=threads, wave_out=wave_out, flags=flags)
    return wl


def render_waves(wl: Workload, threads: int | None = None, wave_out: np.ndarray | None = None, flags: int = 0):
    total = wl.n_samples_total
    if wave_out is None:
        wave = np.empty(total, np.uint16)
    else:
        if wave_out.dtype != np.uint16 or wave_out.size < total:
            raise ValueError("wave_out too small or not uint16")
        wave = wave_out.reshape(-1)
    cam_xy = (ctypes.c_void_p * N_CAM)()
    keep = []
    for c, cam in wl.cams.items():
        cam_xy[c] = _p(cam.xy).value
        keep.append(cam.xy)
    threads = threads or os.cpu_count() or 1
    _L().synth_render(wl.seed, wl.n_img, _p(wl.img_evt), _p(wl.img_tel), _p(wl.tel_cam), _p(wl.tel_pix_off),
                      _p(wl.ped), _p(wl.gain), _p(wl.ell), _p(wl.n_ell), ctypes.cast(cam_xy, ctypes.c_void_p),
                      _p(wl.wave_off), _p(wave), int(flags), int(threads))
    wl.wave = wave[:total] if wave_out is None else wave
    return wl.wave


def subset(wl: Workload, events) -> Workload:
    """A workload holding only the given event indices (waves copied)."""
    events = np.asarray(events, np.int64)
    imgs = np.concatenate([np.arange(wl.evt_off[e], wl.evt_off[e + 1]) for e in events]).astype(np.int64) \
        if len(events) else np.zeros(0, np.int64)
    counts = np.diff(wl.evt_off)[events]
    evt_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    img_tel = wl.img_tel[imgs].copy()
    P = np.array([wl.cams[int(wl.tel_cam[t])].n_pix for t in img_tel], np.int64)
    S = np.array([wl.cams[int(wl.tel_cam[t])].n_samples for t in img_tel], np.int64)
    wave_off = np.concatenate([[0], np.cumsum(P * S)[:-1]]).astype(np.int64) if len(P) else np.zeros(0, np.int64)
    pix_off = np.concatenate([[0], np.cumsum(P)]).astype(np.int64)
    wave = None
    if wl.wave is not None:
        wave = np.empty(int(np.sum(P * S)), np.uint16)
        for k, i in enumerate(imgs):
            n = int(P[k] * S[k])
            wave[wave_off[k]:wave_off[k] + n] = wl.wave[wl.wave_off[i]:wl.wave_off[i] + n]
    return Workload(wl.preset, wl.seed, wl.proc, wl.cams, wl.tel_cam, wl.tel_xy, wl.tel_pix_off, wl.ped, wl.gain,
                    wl.p16, wl.scale, evt_off, img_tel, np.repeat(np.arange(len(events), dtype=np.int32), counts),
                    wave_off, pix_off, wl.ell[imgs].copy(), wl.n_ell[imgs].copy(), wl.truth[events].copy(), wave)


# ----------------------------------------------------------------------------- DL0 byte stream
PKT_MAX_BYTES = 65536


def max_segment_pixels(S: int) -> int:
    """Largest pixel count of one packet for S samples: 48 + 2 n S <= 65536 and
    n S a multiple of 8."""
    n = (PKT_MAX_BYTES - 48) // (2 * S)
    while (n * S) % 8:
        n -= 1
    return n


def stream_plan(wl: Workload, seg_pixels=None):
    """Packets of a workload in stream order (events in order, images of an event
    in order, segments of an image in pixel order): arrays img, first, n, flags
    (3 whole, 1 first, 0 continuation, 2 last), count (per telescope, mod 2^14) and
    the byte offset of each packet. seg_pixels: {camera id: pixels per segment}
    (default: the largest that fits)."""
    img, first, npx, flags = [], [], [], []
    for i in range(wl.n_img):
        cam = wl.image_cam(i)
        P, S = cam.n_pix, cam.n_samples
        seg = (seg_pixels or {}).get(int(wl.tel_cam[wl.img_tel[i]]), max_segment_pixels(S))
        assert (seg * S) % 8 == 0 and 48 + 2 * seg * S <= PKT_MAX_BYTES
        starts = list(range(0, P, seg))
        for j, f in enumerate(starts):
            n = min(seg, P - f)
            img.append(i)
            first.append(f)
            npx.append(n)
            whole, last = len(starts) == 1, j == len(starts) - 1
            flags.append(3 if whole else (1 if j == 0 else (2 if last else 0)))
    img = np.array(img, np.int32)
    first = np.array(first, np.int32)
    npx = np.array(npx, np.int32)
    flags = np.array(flags, np.int32)
    S_of = np.array([wl.image_cam(i).n_samples for i in range(wl.n_img)], np.int32)
    size = 48 + 2 * npx.astype(np.int64) * S_of[img]
    off = np.concatenate([[0], np.cumsum(size)[:-1]]).astype(np.int64)
    tel = wl.img_tel[img]
    count = np.zeros(len(img), np.int32)
    seen = {}
    for k, t in enumerate(tel):
        c = seen.get(int(t), 0)
        count[k] = c % 16384
        seen[int(t)] = c + 1
    return dict(img=img, first=first, n=npx, flags=flags, count=count, off=off, size=size,
                n_bytes=int(size.sum()))


def encode_stream(wl: Workload, event_numbers=None, times_ns=None, seg_pixels=None, threads: int | None = None,
                  out: np.ndarray | None = None):
    """The workload as a DL0 byte stream (the layout of include/rta.h). Returns
    (uint8 array, plan). event_numbers / times_ns: per event (defaults 1000 + e
    and 1 ms apart from 1.7e18 ns)."""
    plan = stream_plan(wl, seg_pixels)
    n_evt = wl.n_evt
    evnum = np.asarray(event_numbers if event_numbers is not None else 1000 + np.arange(n_evt), np.uint64)
    t_ns = np.asarray(times_ns if times_ns is not None else 1_700_000_000_000_000_000 + 1_000_000 * np.arange(n_evt),
                      np.int64)
    evt_of_img = np.repeat(np.arange(n_evt), np.diff(wl.evt_off))
    img_evnum = np.ascontiguousarray(evnum[evt_of_img])
    img_time = np.ascontiguousarray(t_ns[evt_of_img])
    img_P = np.array([wl.image_cam(i).n_pix for i in range(wl.n_img)], np.int32)
    img_S = np.array([wl.image_cam(i).n_samples for i in range(wl.n_img)], np.int32)
    buf = out if out is not None else np.empty(plan["n_bytes"], np.uint8)
    assert buf.size >= plan["n_bytes"]
    _L().synth_write_stream(len(plan["img"]), _p(plan["img"]), _p(plan["first"]), _p(plan["n"]), _p(plan["flags"]),
                            _p(plan["count"]), _p(plan["off"]), _p(np.ascontiguousarray(wl.wave)),
                            _p(np.ascontiguousarray(wl.wave_off)), _p(np.ascontiguousarray(wl.img_tel)), _p(img_P),
                            _p(img_S), _p(img_evnum), _p(img_time), _p(buf), int(threads or os.cpu_count() or 1))
    plan["event_numbers"] = evnum
    plan["times_ns"] = t_ns
    return buf[: plan["n_bytes"]], plan
