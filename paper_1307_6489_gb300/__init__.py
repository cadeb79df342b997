"""Python binding of librta, the GB300 real-time reconstruction library.

Argument marshalling only: every step runs in the CUDA kernels of
``librta.so`` (built in-tree for sm_103a by ``_build.py``).  The functions
below carry the C-ABI names of ``include/rta.h`` and take device pointers as
integers (e.g. ``tensor.data_ptr()``) and streams as integers
(``torch.cuda.current_stream().cuda_stream``).  ``Context`` is a convenience
wrapper that accepts torch tensors and checks their dtype and device.

There is no CPU fallback: if the library cannot be built or loaded, importing
works but every call raises ``RtaUnavailable``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

RTA_OK = 0
RTA_E_INVALID = -1
RTA_E_ALIGN = -2
RTA_E_NOMEM = -3
RTA_E_CUDA = -4
RTA_E_BUSY = -5
RTA_E_TIMEOUT = -6
RTA_E_DEVICE = -7
RTA_WINDOW_FIXED = 0
RTA_WINDOW_SLIDING = 1
RTA_WINDOW_FILTER = 2
RTA_WINDOW_NEIGHBOUR = 3
RTA_HF_EMPTY = 1
RTA_HF_NO_TIME = 2
RTA_HF_BAD_INPUT = 4
RTA_SF_INVALID = 1
RTA_DEV_BAD_IMAGE = 1
RTA_DEV_TIMEOUT = 2

HILLAS_FIELDS = ["size", "x", "y", "length", "width", "psi", "r", "phi", "time_grad", "time_mean"]
HILLAS_BYTES = 64
STEREO_BYTES = 32

_lib = None


class RtaUnavailable(RuntimeError):
    pass


class RtaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"librta error {code}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load(build: bool = True) -> ctypes.CDLL:
    """Load librta.so (building it first if needed and allowed)."""
    global _lib
    if _lib is not None:
        return _lib
    try:
        if build:
            _build.build()
        lib = ctypes.CDLL(_build.LIB)
    except Exception as e:  # no nvcc, no library: fail loudly, never fall back
        raise RtaUnavailable(f"librta is not available: {e}") from e
    P, i32, i64, f32, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t
    sig = {
        "rta_version": ([], i32),
        "rta_last_error": ([], ctypes.c_char_p),
        "rta_create": ([P, i32, sz], i32),
        "rta_destroy": ([P], i32),
        "rta_register_camera": ([P, i32, i32, i32, P, P, i32], i32),
        "rta_register_array": ([P, i32, P, P, P, P], i32),
        "rta_check": ([P, P, P], i32),
        "rta_set_chain_config": ([P, i32, i32, i32], i32),
        "rta_get_chain_config": ([P, P, P, P, P, P], i32),
        "rta_chain_variant_info": ([i32, P, P], i32),
        "rta_autotune": ([P, P, i64, P, P, i64, i32, i32, i32, f32, f32, i32, P, i32, P, i32, P, P], i32),
        "rta_calibrate_integrate": ([P, P, i64, P, P, P, i64, i32, i32, i32, P, P, i64, P], i32),
        "rta_clean": ([P, P, i64, P, P, i64, f32, f32, i32, P, P], i32),
        "rta_hillas": ([P, P, P, P, i64, P, P, i64, P, P], i32),
        "rta_image_chain": ([P, P, i64, P, P, i64, i32, i32, i32, f32, f32, i32, P, P], i32),
        "rta_image_chain_masks": ([P, P, i64, P, P, P, i64, i32, i32, i32, f32, f32, i32, P, i64, P, P], i32),
        "rta_stereo": ([P, P, P, i64, P, i64, P, P], i32),
        "rta_reconstruct": ([P, P, i64, P, P, i64, P, i64, i32, i32, i32, f32, f32, i32, P, P, P], i32),
        "rta_reconstruct_host": ([P, P, i64, P, P, i64, P, i64, i32, i32, i32, f32, f32, i32, P, P], i32),
        "rta_graph_create": ([P, P, i64, P, P, P, i64, P, P, i64, i32, i32, i32, f32, f32, i32, P, P, P], i32),
        "rta_graph_launch": ([P, P], i32),
        "rta_graph_destroy": ([P], i32),
        "rta_surrogate_num_params": ([], i32),
        "rta_surrogate_create": ([P, ctypes.c_uint64, P, P], i32),
        "rta_surrogate_destroy": ([P], i32),
        "rta_surrogate_set_params": ([P, P], i32),
        "rta_surrogate_get_params": ([P, i32, P], i32),
        "rta_surrogate_get_state": ([P, P, P, P, P], i32),
        "rta_surrogate_set_state": ([P, P, P, P, i64], i32),
        "rta_surrogate_forward": ([P, P, P, i64, P, i64, P, P, P], i32),
        "rta_surrogate_train_step": ([P, P, P, i64, P, i64, P, P, P, f32, i32, P, P], i32),
        "rta_surrogate_infer": ([P, P, P, i64, P, i64, f32, P, P], i32),
        "rta_reconstruct_learned": ([P, P, i64, P, P, i64, P, i64, i32, i32, i32, f32, f32, i32, f32, P, P, P], i32),
        "rta_stream_create": ([P, P, sz, i32, i64, i64, i32, i32, i32, f32, f32, i32, f32, P], i32),
        "rta_stream_submit": ([P, P, P], i32),
        "rta_stream_poll": ([P, ctypes.c_uint64, P], i32),
        "rta_stream_poll_times": ([P, ctypes.c_uint64, P, P], i32),
        "rta_stream_drain": ([P, i32], i32),
        "rta_skymap_read": ([P, i64, P], i32),
        "rta_stream_add_events": ([P, P, i64, i64, P], i32),
        "rta_stream_destroy": ([P], i32),
        "rta_set_filter_weights": ([P, P, i32], i32),
        "rta_transient_search": ([P, i64, P, i32, i32, ctypes.c_double, P, i32, P], i32),
        "rta_significance_map": ([P, i64, Window, i32, P, P, P], i32),
        "rta_selftest_wait_timeout": ([P, i32, P, P], i32),
        "rta_ingest": ([P, P, i64, i32, P, i64, P, P, i64, P, P, P, i64, P, P], i32),
        "rta_autotune_stream": ([P, P, i64, P, i64, P, P, i64, P, i32, i32, i32, f32, f32, i32, P, i32, P, i32, P, P],
                                i32),
        "rta_reconstruct_stream": ([P, P, i64, P, i64, P, P, i64, P, i64, P, i32, i32, i32, f32, f32, i32, P, P, P],
                                   i32),
        "rta_lut_accumulate": ([P, P, P, i64, P, i64, P, P, P, P, i32, P, i32, P, P], i32),
        "rta_lut_finalize": ([P, P, i64, i32, P, P], i32),
        "rta_lut_prepare": ([P, P, i64, P, P], i32),
        "rta_lut_reconstruct": ([P, P, P, i64, P, i64, P, P, P, i32, P, i32, f32, f32, f32, f32, P, P], i32),
        "rta_image_chain_noalloc": ([P, i32, P, P, i32, P, P, i64, P, i64, P, P, i64, i32, i32, i32, f32, f32, i32,
                                     P, P, P], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def exported_symbols():
    return [l.split("(")[0].split()[-1].lstrip("*") for l in _header_decls()]


def _header_decls():
    """Function declarations of include/rta.h (one string each)."""
    path = os.path.join(_build.INCLUDE, "rta.h")
    text = open(path).read()
    out, cur = [], ""
    for line in text.splitlines():
        s = line.strip()
        if s.startswith(("int rta_", "const char* rta_", "void rta_")) or cur:
            cur += " " + s
            if s.endswith(";"):
                out.append(cur.strip())
                cur = ""
    return out


def _check(rc: int):
    if rc != RTA_OK:
        raise RtaError(rc, load().rta_last_error().decode())


# ----------------------------------------------------------------------------- C-ABI names
def rta_version() -> int:
    return load().rta_version()


def rta_last_error() -> str:
    return load().rta_last_error().decode()


def rta_create(device: int = 0, hbm_budget_bytes: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load().rta_create(ctypes.byref(h), device, hbm_budget_bytes))
    return h.value


def rta_destroy(ctx: int):
    _check(load().rta_destroy(ctx))


def _np(a, dtype):
    a = np.ascontiguousarray(a, dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def rta_register_camera(ctx: int, cam: int, n_pix: int, n_samples: int, pix_xy, nb, K: int):
    xy, pxy = _np(pix_xy, np.float32)
    nbv, pnb = _np(nb, np.int16)
    _check(load().rta_register_camera(ctx, cam, n_pix, n_samples, pxy, pnb, K))


def rta_register_array(ctx: int, n_tel: int, tel_cam, tel_xy, p16, scale):
    a, pa = _np(tel_cam, np.int32)
    b, pb = _np(tel_xy, np.float32)
    c, pc = _np(p16, np.int32)
    d, pd = _np(scale, np.float32)
    _check(load().rta_register_array(ctx, n_tel, pa, pb, pc, pd))


def rta_check(ctx: int, stream: int = 0) -> int:
    """Synchronise and return the device status bits; raises RtaError(RTA_E_DEVICE) when non-zero."""
    bits = ctypes.c_uint32(0)
    rc = load().rta_check(ctx, stream, ctypes.byref(bits))
    if rc not in (RTA_OK, RTA_E_DEVICE):
        _check(rc)
    if rc == RTA_E_DEVICE:
        err = RtaError(rc, rta_last_error())
        err.bits = bits.value
        raise err
    return bits.value


RTA_CHAIN_VARIANTS = 5


class TuneEntry(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("n_stages", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("grid", ctypes.c_int), ("ms", ctypes.c_float)]


def rta_selftest_wait_timeout(ctx: int, timeout_ms: int, stream: int = 0) -> int:
    """Run the bounded-wait self-test; returns the device-measured wait in ns."""
    w = ctypes.c_uint64()
    _check(load().rta_selftest_wait_timeout(ctx, timeout_ms, ctypes.byref(w), stream))
    return w.value


def rta_set_filter_weights(ctx: int, weights):
    """Integer weights of the RTA_WINDOW_FILTER extractor (empty: clear)."""
    w = np.ascontiguousarray(np.asarray(weights, np.int32).reshape(-1))
    _check(load().rta_set_filter_weights(ctx, w.ctypes.data_as(ctypes.c_void_p) if len(w) else None, len(w)))


def rta_set_chain_config(ctx: int, variant: int, n_stages: int, ctas_per_sm: int):
    _check(load().rta_set_chain_config(ctx, variant, n_stages, ctas_per_sm))


def rta_get_chain_config(ctx: int):
    v, ns, cps, grid, smem = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
    _check(load().rta_get_chain_config(ctx, ctypes.byref(v), ctypes.byref(ns), ctypes.byref(cps), ctypes.byref(grid),
                                       ctypes.byref(smem)))
    return dict(variant=v.value, n_stages=ns.value, ctas_per_sm=cps.value, grid=grid.value, smem_bytes=smem.value)


def rta_chain_variant_info(variant: int):
    w, p = ctypes.c_int(), ctypes.c_int()
    _check(load().rta_chain_variant_info(variant, ctypes.byref(w), ctypes.byref(p)))
    return dict(integrator_warps=w.value, pixels_per_thread=p.value)


def rta_autotune(ctx, d_wave, n_wave, d_wave_off, d_img_tel, n_img, window_mode, start, W, t_hi, t_lo,
                 core_needs_neighbour, d_out, reps=3, stream=0):
    """Sweep the fused kernel's launch configurations on a bundle; keeps the fastest. Returns all measurements."""
    cap = 256
    entries = (TuneEntry * cap)()
    n = ctypes.c_int()
    _check(load().rta_autotune(ctx, d_wave, n_wave, d_wave_off, d_img_tel, n_img, window_mode, start, W, t_hi, t_lo,
                               int(core_needs_neighbour), d_out, reps, entries, cap, ctypes.byref(n), stream))
    return [dict(variant=e.variant, n_stages=e.n_stages, ctas_per_sm=e.ctas_per_sm, grid=e.grid, ms=e.ms)
            for e in entries[: min(n.value, cap)]]


def rta_calibrate_integrate(ctx, d_wave, n_wave, d_wave_off, d_img_tel, d_pix_off, n_img, window_mode, start, W,
                            d_q, d_t, n_q, stream=0):
    _check(load().rta_calibrate_integrate(ctx, d_wave, n_wave, d_wave_off, d_img_tel, d_pix_off, n_img, window_mode,
                                          start, W, d_q, d_t, n_q, stream))


def rta_clean(ctx, d_q, n_q, d_img_tel, d_pix_off, n_img, t_hi, t_lo, core_needs_neighbour, d_mask, stream=0):
    _check(load().rta_clean(ctx, d_q, n_q, d_img_tel, d_pix_off, n_img, t_hi, t_lo, int(core_needs_neighbour),
                            d_mask, stream))


def rta_hillas(ctx, d_q, d_t, d_mask, n_q, d_img_tel, d_pix_off, n_img, d_out, stream=0):
    _check(load().rta_hillas(ctx, d_q, d_t, d_mask, n_q, d_img_tel, d_pix_off, n_img, d_out, stream))


def rta_image_chain(ctx, d_wave, n_wave, d_wave_off, d_img_tel, n_img, window_mode, start, W, t_hi, t_lo,
                    core_needs_neighbour, d_out, stream=0):
    _check(load().rta_image_chain(ctx, d_wave, n_wave, d_wave_off, d_img_tel, n_img, window_mode, start, W, t_hi,
                                  t_lo, int(core_needs_neighbour), d_out, stream))


def rta_image_chain_masks(ctx, d_wave, n_wave, d_wave_off, d_img_tel, d_pix_off, n_img, window_mode, start, W, t_hi,
                          t_lo, core_needs_neighbour, d_mask, n_q, d_out, stream=0):
    _check(load().rta_image_chain_masks(ctx, d_wave, n_wave, d_wave_off, d_img_tel, d_pix_off, n_img, window_mode,
                                        start, W, t_hi, t_lo, int(core_needs_neighbour), d_mask, n_q, d_out, stream))


def rta_stereo(ctx, d_hillas, d_img_tel, n_img, d_evt_off, n_evt, d_out, stream=0):
    _check(load().rta_stereo(ctx, d_hillas, d_img_tel, n_img, d_evt_off, n_evt, d_out, stream))


def rta_reconstruct(ctx, d_wave, n_wave, d_wave_off, d_img_tel, n_img, d_evt_off, n_evt, window_mode, start, W, t_hi,
                    t_lo, core_needs_neighbour, d_hillas, d_stereo, stream=0):
    _check(load().rta_reconstruct(ctx, d_wave, n_wave, d_wave_off, d_img_tel, n_img, d_evt_off, n_evt, window_mode,
                                  start, W, t_hi, t_lo, int(core_needs_neighbour), d_hillas, d_stereo, stream))


def rta_reconstruct_host(ctx, h_wave, n_wave, h_wave_off, h_img_tel, n_img, h_evt_off, n_evt, window_mode, start, W,
                         t_hi, t_lo, core_needs_neighbour, h_hillas, h_stereo):
    _check(load().rta_reconstruct_host(ctx, h_wave, n_wave, h_wave_off, h_img_tel, n_img, h_evt_off, n_evt,
                                       window_mode, start, W, t_hi, t_lo, int(core_needs_neighbour), h_hillas,
                                       h_stereo))


def rta_graph_create(ctx, d_wave, n_wave, d_wave_off, d_img_tel, d_n_img, max_img, d_evt_off, d_n_evt, max_evt,
                     window_mode, start, W, t_hi, t_lo, core_needs_neighbour, d_hillas, d_stereo) -> int:
    g = ctypes.c_void_p()
    _check(load().rta_graph_create(ctx, d_wave, n_wave, d_wave_off, d_img_tel, d_n_img, max_img, d_evt_off, d_n_evt,
                                   max_evt, window_mode, start, W, t_hi, t_lo, int(core_needs_neighbour), d_hillas,
                                   d_stereo, ctypes.byref(g)))
    return g.value


def rta_graph_launch(graph: int, stream: int = 0):
    _check(load().rta_graph_launch(graph, stream))


def rta_graph_destroy(graph: int):
    _check(load().rta_graph_destroy(graph))


RTA_EF_NO_DIRECTION = 1
RTA_EF_FALLBACK = 2
EVENT_BYTES = 32


def rta_surrogate_num_params() -> int:
    return load().rta_surrogate_num_params()


def rta_surrogate_create(ctx: int, seed: int = 0, cam_code=None) -> int:
    m = ctypes.c_void_p()
    codes = None
    if cam_code is not None:
        codes, _ = _np(np.resize(np.asarray(cam_code, np.float32), 16), np.float32)
    _check(load().rta_surrogate_create(ctx, seed, None if codes is None else codes.ctypes.data_as(ctypes.c_void_p),
                                       ctypes.byref(m)))
    return m.value


def rta_surrogate_destroy(model: int):
    _check(load().rta_surrogate_destroy(model))


def rta_surrogate_set_params(model: int, params):
    a, pa = _np(params, np.float32)
    assert a.size == rta_surrogate_num_params()
    _check(load().rta_surrogate_set_params(model, pa))


def rta_surrogate_get_params(model: int, which: int = 0) -> np.ndarray:
    out = np.zeros(rta_surrogate_num_params(), np.float32)
    _check(load().rta_surrogate_get_params(model, which, out.ctypes.data_as(ctypes.c_void_p)))
    return out


def rta_surrogate_get_state(model: int):
    """(parameters, first moments, second moments, Adam steps taken) as float32 arrays and an int."""
    n = rta_surrogate_num_params()
    p, m, v = (np.zeros(n, np.float32) for _ in range(3))
    step = ctypes.c_int64(0)
    _check(load().rta_surrogate_get_state(model, p.ctypes.data, m.ctypes.data, v.ctypes.data, ctypes.byref(step)))
    return p, m, v, int(step.value)


def rta_surrogate_set_state(model: int, params, m, v, step: int):
    n = rta_surrogate_num_params()
    p, m, v = (np.ascontiguousarray(x, np.float32).reshape(-1) for x in (params, m, v))
    if not (p.size == m.size == v.size == n):
        raise ValueError(f"state arrays must hold {n} floats each")
    _check(load().rta_surrogate_set_state(model, p.ctypes.data, m.ctypes.data, v.ctypes.data, int(step)))


def rta_surrogate_forward(model, d_hillas, d_img_tel, n_img, d_evt_off, n_evt, d_y, d_base, stream=0):
    _check(load().rta_surrogate_forward(model, d_hillas, d_img_tel, n_img, d_evt_off, n_evt, d_y, d_base, stream))


def rta_surrogate_train_step(model, d_hillas, d_img_tel, n_img, d_evt_off, n_evt, d_log_energy, d_src_xy, d_is_gamma,
                             lr, apply_update=1, d_loss=0, stream=0):
    _check(load().rta_surrogate_train_step(model, d_hillas, d_img_tel, n_img, d_evt_off, n_evt, d_log_energy, d_src_xy,
                                           d_is_gamma, lr, int(apply_update), d_loss, stream))


def rta_surrogate_infer(model, d_hillas, d_img_tel, n_img, d_evt_off, n_evt, fallback_deg, d_out, stream=0):
    _check(load().rta_surrogate_infer(model, d_hillas, d_img_tel, n_img, d_evt_off, n_evt, fallback_deg, d_out, stream))


def rta_reconstruct_learned(model, d_wave, n_wave, d_wave_off, d_img_tel, n_img, d_evt_off, n_evt, window_mode, start,
                            W, t_hi, t_lo, core_needs_neighbour, fallback_deg, d_hillas, d_events, stream=0):
    _check(load().rta_reconstruct_learned(model, d_wave, n_wave, d_wave_off, d_img_tel, n_img, d_evt_off, n_evt,
                                          window_mode, start, W, t_hi, t_lo, core_needs_neighbour, fallback_deg,
                                          d_hillas, d_events, stream))


def events_to_numpy(raw: np.ndarray) -> dict:
    """Decode rows of rta_event_t (n*32 bytes)."""
    raw = np.ascontiguousarray(raw).view(np.uint8).reshape(-1, EVENT_BYTES)
    f = raw.view(np.float32).reshape(-1, 8)
    i = raw.view(np.int32).reshape(-1, 8)
    return dict(log_energy=f[:, 0].copy(), dir_x=f[:, 1].copy(), dir_y=f[:, 2].copy(), gammaness=f[:, 3].copy(),
                n_used=i[:, 4].copy(), flags=i[:, 5].view(np.uint32).copy(), base_x=f[:, 6].copy(),
                base_y=f[:, 7].copy())


RTA_DEV_BAD_STREAM = 4
RTA_STREAM_OK, RTA_STREAM_FRAMING, RTA_STREAM_HEADER, RTA_STREAM_CAMERA, RTA_STREAM_SEGMENT, RTA_STREAM_CRC, \
    RTA_STREAM_CAPACITY = range(7)
SEGMENT_DTYPE = np.dtype([("offset", "<i8"), ("first_pixel", "<i4"), ("n_pixels", "<i4")])


def rta_ingest(ctx, d_stream, n_bytes, verify_crc, d_seg, seg_cap, d_img_seg, d_img_tel, img_cap, d_evt_off,
               d_evt_number, d_evt_time_ns, evt_cap, d_counts, stream=0):
    """Directory of a device-resident DL0 byte stream (see include/rta.h); d_counts
    (6 int64) receives n_segments, n_img, n_evt, n_samples, error, error offset."""
    _check(load().rta_ingest(ctx, d_stream, n_bytes, int(verify_crc), d_seg, seg_cap, d_img_seg, d_img_tel, img_cap,
                             d_evt_off, d_evt_number, d_evt_time_ns, evt_cap, d_counts, stream))


def rta_reconstruct_stream(ctx, d_stream, n_bytes, d_seg, max_seg, d_img_seg, d_img_tel, max_img, d_evt_off, max_evt,
                           d_counts, window_mode, start, W, t_hi, t_lo, core_needs_neighbour, d_hillas, d_stereo,
                           stream=0):
    _check(load().rta_reconstruct_stream(ctx, d_stream, n_bytes, d_seg, max_seg, d_img_seg, d_img_tel, max_img,
                                         d_evt_off, max_evt, d_counts, window_mode, start, W, t_hi, t_lo,
                                         int(core_needs_neighbour), d_hillas, d_stereo, stream))


def rta_autotune_stream(ctx, d_stream, n_bytes, d_seg, max_seg, d_img_seg, d_img_tel, max_img, d_counts, window_mode,
                        start, W, t_hi, t_lo, core_needs_neighbour, d_hillas, reps=3, stream=0):
    """Sweep the byte-stream image kernel's launch configurations; keeps the fastest. Returns all measurements."""
    cap = 256
    entries = (TuneEntry * cap)()
    n = ctypes.c_int()
    _check(load().rta_autotune_stream(ctx, d_stream, n_bytes, d_seg, max_seg, d_img_seg, d_img_tel, max_img, d_counts,
                                      window_mode, start, W, t_hi, t_lo, int(core_needs_neighbour), d_hillas, reps,
                                      entries, cap, ctypes.byref(n), stream))
    return [dict(variant=e.variant, n_stages=e.n_stages, ctas_per_sm=e.ctas_per_sm, grid=e.grid, ms=e.ms)
            for e in entries[: min(n.value, cap)]]


RTA_MAX_CAMS = 16
RTA_LUT_MAX_BINS = 64
RTA_LF_GAMMA = 1
RTA_LF_NO_CORE = 2
RTA_LF_NO_IMAGE = 4
RTA_LF_MALFORMED = 8
LUT_CELL_BYTES = 32
LUT_LOOKUP_BYTES = 64
LUT_EVENT_BYTES = 32
LUT_CELL_FIELDS = ["n", "mean_w", "sigma_w", "mean_l", "sigma_l", "mean_e", "sigma_e"]


def rta_lut_accumulate(ctx, d_hillas, d_img_tel, n_img, d_evt_off, n_evt, d_log_energy, d_core_xy, d_use,
                       d_size_edges, n_size, d_dist_edges, n_dist, d_acc, stream=0):
    _check(load().rta_lut_accumulate(ctx, d_hillas, d_img_tel, n_img, d_evt_off, n_evt, d_log_energy, d_core_xy, d_use,
                                     d_size_edges, n_size, d_dist_edges, n_dist, d_acc, stream))


def rta_lut_finalize(ctx, d_acc, n_cells, min_count, d_cells, stream=0):
    _check(load().rta_lut_finalize(ctx, d_acc, n_cells, min_count, d_cells, stream))


def rta_lut_prepare(ctx, d_cells, n_cells, d_lookup, stream=0):
    """The lookup form of a table (n_cells * LUT_LOOKUP_BYTES bytes at d_lookup)."""
    _check(load().rta_lut_prepare(ctx, d_cells, n_cells, d_lookup, stream))


def rta_lut_reconstruct(ctx, d_hillas, d_img_tel, n_img, d_evt_off, n_evt, d_stereo, d_lookup, d_size_edges, n_size,
                        d_dist_edges, n_dist, cuts, d_out, stream=0):
    """cuts = (mscw_lo, mscw_hi, mscl_lo, mscl_hi); d_lookup from rta_lut_prepare."""
    c = [float(v) for v in cuts]
    _check(load().rta_lut_reconstruct(ctx, d_hillas, d_img_tel, n_img, d_evt_off, n_evt, d_stereo, d_lookup,
                                      d_size_edges, n_size, d_dist_edges, n_dist, c[0], c[1], c[2], c[3], d_out,
                                      stream))


def lut_cells_to_numpy(raw: np.ndarray) -> dict:
    """Decode rows of rta_lut_cell_t (n*32 bytes)."""
    raw = np.ascontiguousarray(raw).view(np.uint8).reshape(-1, LUT_CELL_BYTES)
    f = raw.view(np.float32).reshape(-1, 8)
    out = {k: f[:, j].copy() for j, k in enumerate(LUT_CELL_FIELDS) if j}
    out["n"] = raw.view(np.int32).reshape(-1, 8)[:, 0].copy()
    return out


def lut_cells_from_numpy(n, mean_w, sigma_w, mean_l, sigma_l, mean_e, sigma_e) -> np.ndarray:
    """Pack per-cell columns into rta_lut_cell_t rows (float32 array of n_cells x 8)."""
    n = np.asarray(n)
    out = np.zeros((len(n), 8), np.float32)
    out.view(np.int32)[:, 0] = n.astype(np.int32)
    for j, v in enumerate([mean_w, sigma_w, mean_l, sigma_l, mean_e, sigma_e]):
        out[:, 1 + j] = np.asarray(v, np.float32)
    return out


def lut_events_to_numpy(raw: np.ndarray) -> dict:
    """Decode rows of rta_lut_event_t (n*32 bytes)."""
    raw = np.ascontiguousarray(raw).view(np.uint8).reshape(-1, LUT_EVENT_BYTES)
    f = raw.view(np.float32).reshape(-1, 8)
    i = raw.view(np.int32).reshape(-1, 8)
    return dict(log_energy=f[:, 0].copy(), sigma_log_energy=f[:, 1].copy(), mscw=f[:, 2].copy(), mscl=f[:, 3].copy(),
                n_used=i[:, 4].copy(), flags=i[:, 5].view(np.uint32).copy())


# packed parameter layout of the surrogate (name, shape), row-major
SURROGATE_LAYOUT = [("W1", (12, 128)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)), ("V1", (256, 256)),
                    ("c1", (256,)), ("V2", (256, 4)), ("c2", (4,))]


def pack_params(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[k], np.float32).reshape(-1) for k, _ in SURROGATE_LAYOUT])


def unpack_params(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for k, shp in SURROGATE_LAYOUT:
        n = int(np.prod(shp))
        out[k] = np.asarray(flat[o:o + n]).reshape(shp)
        o += n
    return out


RTA_SKY_N = 256
RTA_SKY_SLABS = 30


class Window(ctypes.Structure):
    """rta_window_t: on window of on_s seconds ending at the search time, off window of off_s seconds before it."""
    _fields_ = [("on_s", ctypes.c_int32), ("off_s", ctypes.c_int32)]


ALERT_DTYPE = np.dtype([("window", np.int32), ("ix", np.int32), ("iy", np.int32), ("pad", np.int32),
                        ("n_on", np.int64), ("n_off", np.int64), ("alpha", np.float64), ("significance", np.float64)])
RTA_SKY_MIN_SLABS = 60
RTA_MAX_DISK_RADIUS = 32


class Bundle(ctypes.Structure):
    """rta_bundle_t: one bundle in host memory for the serving stream."""
    _fields_ = [("h_wave", ctypes.c_void_p), ("n_wave", ctypes.c_int64), ("h_wave_off", ctypes.c_void_p),
                ("h_img_tel", ctypes.c_void_p), ("n_img", ctypes.c_int64), ("h_evt_off", ctypes.c_void_p),
                ("n_evt", ctypes.c_int64), ("arrival_ns", ctypes.c_int64), ("h_events", ctypes.c_void_p)]


def rta_stream_create(ctx, model, hbm_budget_bytes, max_inflight, max_img, max_evt, window_mode, start, W, t_hi, t_lo,
                      core_needs_neighbour, fallback_deg=0.5) -> int:
    h = ctypes.c_void_p()
    _check(load().rta_stream_create(ctx, model or None, hbm_budget_bytes, max_inflight, max_img, max_evt, window_mode,
                                    start, W, t_hi, t_lo, int(core_needs_neighbour), fallback_deg, ctypes.byref(h)))
    return h.value


def rta_stream_submit(stream: int, bundle: Bundle) -> int:
    t = ctypes.c_uint64()
    _check(load().rta_stream_submit(stream, ctypes.byref(bundle), ctypes.byref(t)))
    return t.value


def rta_stream_poll(stream: int, ticket: int):
    """Completion time (ns) once done, else None."""
    done = ctypes.c_int64()
    rc = load().rta_stream_poll(stream, ticket, ctypes.byref(done))
    if rc == RTA_E_BUSY:
        return None
    _check(rc)
    return done.value


class BundleTimes(ctypes.Structure):
    """rta_bundle_times_t: host instants (ns) of a bundle's arrival, submission, admission and completion,
    the device durations (ms) of its copies in, its pass's device work and output, the wait of its
    published data for that pass, and the number of bundles in the pass."""
    _fields_ = [("arrival_ns", ctypes.c_int64), ("submit_ns", ctypes.c_int64), ("admit_ns", ctypes.c_int64),
                ("done_ns", ctypes.c_int64), ("h2d_ms", ctypes.c_float), ("compute_ms", ctypes.c_float),
                ("d2h_ms", ctypes.c_float), ("slot", ctypes.c_int32), ("ready_wait_ms", ctypes.c_float),
                ("batch_bundles", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def rta_stream_poll_times(stream: int, ticket: int):
    """The bundle's BundleTimes once done, else None."""
    done = ctypes.c_int64()
    t = BundleTimes()
    rc = load().rta_stream_poll_times(stream, ticket, ctypes.byref(done), ctypes.byref(t))
    if rc == RTA_E_BUSY:
        return None
    _check(rc)
    return t


def rta_stream_drain(stream: int, timeout_ms: int = 60000):
    _check(load().rta_stream_drain(stream, timeout_ms))


def rta_skymap_read(stream: int, now_ns: int) -> np.ndarray:
    out = np.zeros((RTA_SKY_N, RTA_SKY_N), np.uint32)
    _check(load().rta_skymap_read(stream, now_ns, out.ctypes.data_as(ctypes.c_void_p)))
    return out


def rta_stream_add_events(stream: int, d_events: int, n_evt: int, arrival_ns: int, cuda_stream: int = 0):
    _check(load().rta_stream_add_events(stream, d_events, n_evt, arrival_ns, cuda_stream))


def rta_stream_destroy(stream: int):
    _check(load().rta_stream_destroy(stream))


def rta_transient_search(stream: int, now_ns: int, windows, radius_bins: int, s_min: float,
                         max_alerts: int = 65536, with_total: bool = False):
    """Alerts (ALERT_DTYPE rows sorted by window, iy, ix) of the windows [(on_s, off_s), ...]; the
    first max_alerts of them, and with with_total=True also the number found (which may be larger)."""
    w = np.ascontiguousarray(np.asarray(windows, np.int32).reshape(-1, 2))
    out = np.zeros(max(max_alerts, 1), ALERT_DTYPE)
    n = ctypes.c_int(0)
    _check(load().rta_transient_search(stream, now_ns, w.ctypes.data_as(ctypes.c_void_p), len(w), radius_bins,
                                       float(s_min), out.ctypes.data_as(ctypes.c_void_p), max_alerts, ctypes.byref(n)))
    rows = out[: min(n.value, max_alerts)].copy()
    return (rows, int(n.value)) if with_total else rows


def rta_significance_map(stream: int, now_ns: int, window, radius_bins: int):
    """(significance, disk on counts, disk off counts) maps [iy, ix] of one window (on_s, off_s)."""
    sig = np.zeros((RTA_SKY_N, RTA_SKY_N), np.float64)
    on = np.zeros((RTA_SKY_N, RTA_SKY_N), np.int64)
    off = np.zeros((RTA_SKY_N, RTA_SKY_N), np.int64)
    _check(load().rta_significance_map(stream, now_ns, Window(int(window[0]), int(window[1])), radius_bins,
                                       sig.ctypes.data_as(ctypes.c_void_p), on.ctypes.data_as(ctypes.c_void_p),
                                       off.ctypes.data_as(ctypes.c_void_p)))
    return sig, on, off


RTA_NOALLOC_MAX_CAMS = 16
RTA_NOALLOC_MAX_TEL = 1024


class CameraDesc(ctypes.Structure):
    """rta_camera_desc_t: one camera type whose tables live in caller-owned device memory."""
    _fields_ = [("n_pix", ctypes.c_int), ("n_samples", ctypes.c_int), ("K", ctypes.c_int),
                ("d_pix_xy", ctypes.c_void_p), ("d_nb8", ctypes.c_void_p)]


def rta_image_chain_noalloc(cams, tel_cam, tel_row, d_p16, d_scale, n_calib_rows, d_wave, n_wave, d_wave_off,
                            d_img_tel, n_img, window_mode, start, W, t_hi, t_lo, core_needs_neighbour, d_out,
                            d_status=0, stream=0):
    """For callers that cannot allocate device memory: the fused image kernel with
    caller-owned buffers only (see include/rta.h). `cams` is a sequence of
    CameraDesc (or (n_pix, n_samples, K, d_pix_xy, d_nb8) tuples)."""
    arr = (CameraDesc * max(1, len(cams)))()
    for i, c in enumerate(cams):
        arr[i] = c if isinstance(c, CameraDesc) else CameraDesc(*c)
    tc, ptc = _np(tel_cam, np.int32)
    tr, ptr = _np(tel_row, np.int64)
    _check(load().rta_image_chain_noalloc(arr, len(cams), ptc, ptr, len(tc), d_p16, d_scale, n_calib_rows, d_wave,
                                          n_wave, d_wave_off, d_img_tel, n_img, window_mode, start, W, t_hi, t_lo,
                                          int(core_needs_neighbour), d_out, d_status, stream))


# ----------------------------------------------------------------------------- row decoding
def hillas_to_numpy(raw: np.ndarray) -> dict:
    """Decode rows of rta_hillas_t (a uint8/float32 buffer of n*64 bytes) into named arrays."""
    raw = np.ascontiguousarray(raw).view(np.uint8).reshape(-1, HILLAS_BYTES)
    f = raw.view(np.float32).reshape(-1, 16)
    i = raw.view(np.int32).reshape(-1, 16)
    out = {k: f[:, j].copy() for j, k in enumerate(HILLAS_FIELDS)}
    out["n_pix"] = i[:, 10].copy()
    out["flags"] = i[:, 11].view(np.uint32).copy()
    return out


def stereo_to_numpy(raw: np.ndarray) -> dict:
    raw = np.ascontiguousarray(raw).view(np.uint8).reshape(-1, STEREO_BYTES)
    f = raw.view(np.float32).reshape(-1, 8)
    i = raw.view(np.int32).reshape(-1, 8)
    return dict(dir_x=f[:, 0].copy(), dir_y=f[:, 1].copy(), core_x=f[:, 2].copy(), core_y=f[:, 3].copy(),
                n_valid=i[:, 4].copy(), flags=i[:, 5].view(np.uint32).copy())


# ----------------------------------------------------------------------------- convenience wrapper
class Context:
    """Owns an rta_ctx; methods take torch tensors (device pointers are read from them)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.device = device
        self.handle = rta_create(device, hbm_budget_bytes)

    def close(self):
        if self.handle:
            rta_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def register_camera(self, cam: int, pix_xy, nb, n_samples: int):
        nb = np.asarray(nb)
        rta_register_camera(self.handle, cam, nb.shape[0], n_samples, pix_xy, nb, nb.shape[1])

    def register_array(self, tel_cam, tel_xy, p16, scale):
        rta_register_array(self.handle, len(tel_cam), tel_cam, tel_xy, p16, scale)

    def check(self, stream: int = 0) -> int:
        return rta_check(self.handle, stream)

    def set_chain_config(self, variant: int, n_stages: int, ctas_per_sm: int):
        rta_set_chain_config(self.handle, variant, n_stages, ctas_per_sm)

    def autotune(self, wave, wave_off, img_tel, window_mode, start, W, t_hi, t_lo, core_needs_neighbour, out, reps=3,
                 stream=None):
        return rta_autotune(self.handle, wave.data_ptr(), wave.numel(), wave_off.data_ptr(), img_tel.data_ptr(),
                            img_tel.numel(), window_mode, start, W, t_hi, t_lo, core_needs_neighbour, out.data_ptr(),
                            reps, self._stream(stream))

    def chain_config(self) -> dict:
        return rta_get_chain_config(self.handle)

    @staticmethod
    def _stream(stream):
        if stream is None:
            import torch
            return torch.cuda.current_stream().cuda_stream
        return int(stream)

    def calibrate_integrate(self, wave, wave_off, img_tel, pix_off, window_mode, start, W, q, t=None, stream=None):
        if t is not None:
            assert t.numel() == q.numel()
        rta_calibrate_integrate(self.handle, wave.data_ptr(), wave.numel(), wave_off.data_ptr(), img_tel.data_ptr(),
                                pix_off.data_ptr(), img_tel.numel(), window_mode, start, W, q.data_ptr(),
                                0 if t is None else t.data_ptr(), q.numel(), self._stream(stream))

    def clean(self, q, img_tel, pix_off, t_hi, t_lo, core_needs_neighbour, mask, stream=None):
        assert mask.numel() == q.numel()
        rta_clean(self.handle, q.data_ptr(), q.numel(), img_tel.data_ptr(), pix_off.data_ptr(), img_tel.numel(),
                  t_hi, t_lo, core_needs_neighbour, mask.data_ptr(), self._stream(stream))

    def hillas(self, q, t, mask, img_tel, pix_off, out, stream=None):
        assert mask.numel() == q.numel() and (t is None or t.numel() == q.numel())
        rta_hillas(self.handle, q.data_ptr(), 0 if t is None else t.data_ptr(), mask.data_ptr(), q.numel(),
                   img_tel.data_ptr(), pix_off.data_ptr(), img_tel.numel(), out.data_ptr(), self._stream(stream))

    def image_chain(self, wave, wave_off, img_tel, window_mode, start, W, t_hi, t_lo, core_needs_neighbour, out,
                    stream=None):
        rta_image_chain(self.handle, wave.data_ptr(), wave.numel(), wave_off.data_ptr(), img_tel.data_ptr(),
                        img_tel.numel(), window_mode, start, W, t_hi, t_lo, core_needs_neighbour, out.data_ptr(),
                        self._stream(stream))

    def image_chain_masks(self, wave, wave_off, img_tel, pix_off, window_mode, start, W, t_hi, t_lo,
                          core_needs_neighbour, mask, out, stream=None):
        rta_image_chain_masks(self.handle, wave.data_ptr(), wave.numel(), wave_off.data_ptr(), img_tel.data_ptr(),
                              pix_off.data_ptr(), img_tel.numel(), window_mode, start, W, t_hi, t_lo,
                              core_needs_neighbour, mask.data_ptr(), mask.numel(), out.data_ptr(),
                              self._stream(stream))

    def stereo(self, hillas, evt_off, img_tel, out, stream=None):
        rta_stereo(self.handle, hillas.data_ptr(), img_tel.data_ptr(), img_tel.numel(), evt_off.data_ptr(),
                   evt_off.numel() - 1, out.data_ptr(), self._stream(stream))

    def reconstruct(self, wave, wave_off, img_tel, evt_off, window_mode, start, W, t_hi, t_lo, core_needs_neighbour,
                    hillas, stereo, stream=None):
        rta_reconstruct(self.handle, wave.data_ptr(), wave.numel(), wave_off.data_ptr(), img_tel.data_ptr(),
                        img_tel.numel(), evt_off.data_ptr(), evt_off.numel() - 1, window_mode, start, W, t_hi, t_lo,
                        core_needs_neighbour, hillas.data_ptr(), stereo.data_ptr(), self._stream(stream))

    def reconstruct_host(self, wave: np.ndarray, wave_off: np.ndarray, img_tel: np.ndarray, evt_off: np.ndarray,
                         window_mode, start, W, t_hi, t_lo, core_needs_neighbour, hillas: np.ndarray,
                         stereo: np.ndarray):
        """Host buffers in, host rows out (hillas: n_img*64 bytes, stereo: n_evt*32 bytes)."""
        ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        for a in (wave, wave_off, img_tel, evt_off, hillas, stereo):
            assert a.flags["C_CONTIGUOUS"]
        rta_reconstruct_host(self.handle, ptr(wave), wave.size, ptr(wave_off), ptr(img_tel), len(img_tel), ptr(evt_off),
                             len(evt_off) - 1, window_mode, start, W, t_hi, t_lo, core_needs_neighbour, ptr(hillas),
                             ptr(stereo))
