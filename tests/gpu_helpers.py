"""Shared helpers of the GPU parity tests: device copies of a workload, a
registered librta context, row decoding, and the comparison rules.

Tolerances (floating point; integer and byte outputs are compared bit-exact):
  charges q            bit-exact (integer window sums, one FP32 multiply on both sides)
  peak times t         |dt| <= 1e-3 samples (FP32 division of exact integers vs FP64)
  cleaning masks       bit-exact (FP32 comparisons of bit-exact charges)
  size                 relative 1e-4
  x, y, length, width  |d| / max(|ref|, 0.1 deg) <= 1e-4
  psi                  1e-4 rad modulo pi, where (length - width) / length > 1e-2
  time gradient        |d| <= 1e-3 + 1e-4 |ref| where n_pix >= 5 and elongated as above,
                       with the sign taken along the GPU's psi orientation
  stereo direction     1e-3 deg; core 0.05 m + 2e-6 |core| (stage-isolated: both sides get the
                       same FP32 rows; the relative term is FP32 rounding of the core itself,
                       which for events with nearly parallel axes lies hundreds of km away)
"""
import numpy as np
import torch

import paper_1307_6489_gb300 as rta

REL_MOM = 1e-4
FLOOR_DEG = 0.1
PSI_ABS = 1e-4
T_ABS = 1e-3
TG_ABS, TG_REL = 1e-3, 1e-4
DIR_DEG = 1e-3
CORE_M = 0.05
CORE_REL = 2e-6


def core_ok(gx, gy, rx, ry):
    """Stage-isolated core parity: |d| <= CORE_M + CORE_REL |ref| per event."""
    return np.hypot(gx - rx, gy - ry) <= CORE_M + CORE_REL * np.hypot(rx, ry)


def make_ctx(wl, device=0):
    ctx = rta.Context(device)
    for c, cam in wl.cams.items():
        ctx.register_camera(c, cam.xy, cam.nb, cam.n_samples)
    ctx.register_array(wl.tel_cam, wl.tel_xy, wl.p16, wl.scale)
    if getattr(wl.proc, "weights", None) is not None:
        rta.rta_set_filter_weights(ctx.handle, wl.proc.weights)
    return ctx


class Dev:
    """Device copies of a synth.Workload (torch tensors; raw uint16 bytes as int16)."""

    def __init__(self, wl, device="cuda"):
        self.wave = torch.from_numpy(wl.wave.view(np.int16)).to(device)
        self.wave_off = torch.from_numpy(np.ascontiguousarray(wl.wave_off)).to(device)
        self.img_tel = torch.from_numpy(np.ascontiguousarray(wl.img_tel)).to(device)
        self.pix_off = torch.from_numpy(np.ascontiguousarray(wl.pix_off[:-1])).to(device)
        self.evt_off = torch.from_numpy(np.ascontiguousarray(wl.evt_off)).to(device)
        self.n_img = wl.n_img
        self.n_evt = wl.n_evt
        self.n_pix = int(wl.pix_off[-1])

    def hillas_buf(self):
        return torch.zeros(max(self.n_img, 1) * 16, dtype=torch.float32, device=self.wave.device)

    def stereo_buf(self):
        return torch.zeros(max(self.n_evt, 1) * 8, dtype=torch.float32, device=self.wave.device)


def proc_args(wl):
    p = wl.proc
    if getattr(p, "nbpeak", False):
        mode = rta.RTA_WINDOW_NEIGHBOUR
    elif getattr(p, "weights", None) is not None:
        mode = rta.RTA_WINDOW_FILTER
    else:
        mode = rta.RTA_WINDOW_SLIDING if p.sliding else rta.RTA_WINDOW_FIXED
    return (mode, p.start, p.W, p.t_hi, p.t_lo, p.core_needs_neighbour)


def hillas_rows(buf, n):
    return rta.hillas_to_numpy(buf.cpu().numpy()[: n * 16])


def stereo_rows(buf, n):
    return rta.stereo_to_numpy(buf.cpu().numpy()[: n * 8])


def compare_hillas(g, ref, what=""):
    """g: decoded GPU rows; ref: oracle rows (n, 12). Asserts every tolerance; returns max errors."""
    import oracle
    H = oracle.H
    n = len(ref)
    assert len(g["size"]) == n
    np.testing.assert_array_equal(g["n_pix"], ref[:, H["n_pix"]].astype(np.int32), err_msg=what + " n_pix")
    np.testing.assert_array_equal(g["flags"], ref[:, H["flags"]].astype(np.uint32), err_msg=what + " flags")
    ok = ref[:, H["n_pix"]] > 0
    errs = {}
    rs = ref[ok, H["size"]]
    errs["size"] = np.max(np.abs(g["size"][ok] - rs) / np.abs(rs), initial=0)
    for k in ["x", "y", "length", "width"]:
        r = ref[ok, H[k]]
        errs[k] = np.max(np.abs(g[k][ok] - r) / np.maximum(np.abs(r), FLOOR_DEG), initial=0)
    L, W = ref[:, H["length"]], ref[:, H["width"]]
    elong = ok & (L > 0) & ((L - W) / np.where(L > 0, L, 1) > 1e-2)
    d = np.abs(g["psi"][elong] - ref[elong, H["psi"]]) % np.pi
    errs["psi"] = np.max(np.minimum(d, np.pi - d), initial=0)
    tg = elong & (ref[:, H["n_pix"]] >= 5)
    r = ref[tg, H["time_grad"]]
    # the gradient is signed along psi; psi lives in (-pi/2, pi/2], so where an
    # axis sits at the +-pi/2 branch cut rounding may pick the other end of it
    orient = np.sign(np.cos(g["psi"][tg].astype(np.float64) - ref[tg, H["psi"]]))
    errs["time_grad"] = np.max(np.abs(orient * g["time_grad"][tg] - r) - TG_REL * np.abs(r), initial=0)
    r = ref[ok, H["time_mean"]]
    errs["time_mean"] = np.max(np.abs(g["time_mean"][ok] - r), initial=0)
    assert errs["size"] <= REL_MOM, (what, errs)
    for k in ["x", "y", "length", "width"]:
        assert errs[k] <= REL_MOM, (what, k, errs)
    assert errs["psi"] <= PSI_ABS, (what, errs)
    assert errs["time_grad"] <= TG_ABS, (what, errs)
    assert errs["time_mean"] <= T_ABS, (what, errs)
    return errs


def hillas_rows_as_f32(ref):
    """Oracle Hillas rows rounded to FP32 and packed as rta_hillas_t bytes."""
    import oracle
    H = oracle.H
    n = len(ref)
    buf = np.zeros((n, 16), np.float32)
    for j, k in enumerate(rta.HILLAS_FIELDS):
        buf[:, j] = ref[:, H[k]].astype(np.float32)
    ib = buf.view(np.int32)
    ib[:, 10] = ref[:, H["n_pix"]].astype(np.int32)
    ib[:, 11] = ref[:, H["flags"]].astype(np.int32)
    return buf


def f32_rows_as_oracle(buf):
    """The FP32 rows back as oracle rows (doubles), so both sides see identical inputs."""
    import oracle
    H = oracle.H
    n = buf.shape[0]
    ref = np.zeros((n, 12))
    for j, k in enumerate(rta.HILLAS_FIELDS):
        ref[:, H[k]] = buf[:, j].astype(np.float64)
    ib = buf.view(np.int32)
    ref[:, H["n_pix"]] = ib[:, 10]
    ref[:, H["flags"]] = ib[:, 11]
    return ref
