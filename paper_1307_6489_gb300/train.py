"""Host-side driver for training and evaluating the deep-sets surrogate.

Marshalling only: batching, learning-rate schedule and bookkeeping on the host;
every computation (image reconstruction, features, forward, backward, Adam,
inference) runs in librta's kernels through the C-ABI calls of the binding.
"""
from __future__ import annotations

import numpy as np

from . import (RTA_WINDOW_FIXED, RTA_WINDOW_SLIDING, Context, rta_surrogate_create, rta_surrogate_destroy,
               rta_surrogate_get_state, rta_surrogate_set_state,
               rta_surrogate_infer, rta_surrogate_train_step, events_to_numpy, hillas_to_numpy, stereo_to_numpy)


def reconstruct_images(ctx: Context, wave, wave_off, img_tel, evt_off, proc, stream=None):
    """Hillas rows (device, float32 view of n_img*16) of a device-resident bundle.

    wave/wave_off/img_tel/evt_off are torch CUDA tensors; proc = (window_mode,
    start, W, t_hi, t_lo, core_needs_neighbour)."""
    import torch
    h = torch.zeros(img_tel.numel() * 16, dtype=torch.float32, device=wave.device)
    ctx.image_chain(wave, wave_off, img_tel, *proc, h, stream=stream)
    return h


class SurrogateTrainer:
    """Trains an rta_model on a device-resident set of events.

    hillas: float32 CUDA tensor of n_img*16 (rta_hillas_t rows); img_tel: int32
    CUDA tensor; evt_off: int64 numpy array (n_evt+1, CSR of images); labels:
    log_energy (float32, n_evt), src_xy (float32, n_evt*2), is_gamma (uint8).
    """

    def __init__(self, ctx: Context, seed: int = 0, cam_code=None, model: int | None = None):
        self.ctx = ctx
        self.cam_code = np.zeros(16, np.float32) if cam_code is None else np.asarray(cam_code, np.float32)
        self.model = model if model is not None else rta_surrogate_create(ctx.handle, seed, cam_code)
        self.own = model is None

    def save(self, path: str):
        """Checkpoint: parameters, Adam moments, steps taken and camera codes."""
        p, m, v, step = rta_surrogate_get_state(self.model)
        write_checkpoint(path, p, m, v, step, self.cam_code)

    @classmethod
    def resume(cls, ctx: Context, path: str) -> "SurrogateTrainer":
        """A trainer whose model continues from a checkpoint exactly where it stopped."""
        p, m, v, step, codes = read_checkpoint(path)
        tr = cls(ctx, seed=0, cam_code=codes)
        rta_surrogate_set_state(tr.model, p, m, v, step)
        return tr

    def close(self):
        if self.own and self.model:
            rta_surrogate_destroy(self.model)
        self.model = None

    def fit(self, hillas, img_tel, evt_off, log_energy, src_xy, is_gamma, epochs=10, batch_events=4096, lr=2e-3,
            lr_end=2e-4, seed=0, stream=None):
        """Adam over shuffled batches of consecutive events. Nothing waits for the
        device inside the loop: every batch's event offsets are uploaded once, and
        each step's loss goes to its own slot of a device array read at the end."""
        import torch
        dev = hillas.device
        stream = torch.cuda.current_stream(dev).cuda_stream if stream is None else int(stream)
        evt_off = np.asarray(evt_off, np.int64)
        n_evt = len(evt_off) - 1
        starts = np.arange(0, n_evt, batch_events)
        rng = np.random.default_rng(seed)
        steps = epochs * len(starts)
        # per batch b: its events' image offsets relative to its first image (CSR)
        offs = np.zeros((len(starts), batch_events + 1), np.int32)
        for b, e0 in enumerate(starts):
            e1 = min(n_evt, e0 + batch_events)
            offs[b, : e1 - e0 + 1] = evt_off[e0:e1 + 1] - evt_off[e0]
        d_offs = torch.from_numpy(offs).to(dev)
        d_loss = torch.zeros(max(steps, 1), dtype=torch.float32, device=dev)
        torch.cuda.synchronize(dev)          # the uploads above ran on torch's stream
        k = 0
        for ep in range(epochs):
            for b in rng.permutation(len(starts)):
                e0 = int(starts[b])
                e1 = min(n_evt, e0 + batch_events)
                i0, i1 = int(evt_off[e0]), int(evt_off[e1])
                rate = lr * (lr_end / lr) ** (k / max(1, steps - 1))
                rta_surrogate_train_step(self.model, hillas.data_ptr() + 64 * i0, img_tel.data_ptr() + 4 * i0, i1 - i0,
                                         d_offs[b].data_ptr(), e1 - e0, log_energy.data_ptr() + 4 * e0,
                                         src_xy.data_ptr() + 8 * e0, is_gamma.data_ptr() + e0, rate, 1,
                                         d_loss[k].data_ptr(), stream)
                k += 1
        torch.cuda.synchronize(dev)
        return d_loss[:steps].cpu().numpy().astype(np.float64).tolist()

    def infer(self, hillas, img_tel, evt_off_dev, fallback_deg=0.5, stream=None):
        """rta_event_t rows (uint8 CUDA tensor n_evt*32) for a device-resident set."""
        import torch
        n_evt = evt_off_dev.numel() - 1
        out = torch.zeros(n_evt * 32, dtype=torch.uint8, device=hillas.device)
        stream = torch.cuda.current_stream(hillas.device).cuda_stream if stream is None else int(stream)
        rta_surrogate_infer(self.model, hillas.data_ptr(), img_tel.data_ptr(), img_tel.numel(), evt_off_dev.data_ptr(),
                            n_evt, fallback_deg, out.data_ptr(), stream)
        return out


def containment68(d):
    d = np.asarray(d)
    return float(np.percentile(d, 68)) if len(d) else float("nan")


def roc_auc(score_pos, score_neg):
    """Area under the ROC curve (probability a positive outranks a negative; ties count half)."""
    s = np.concatenate([score_pos, score_neg])
    order = np.argsort(s, kind="mergesort")
    ranks = np.empty(len(s))
    sorted_s = s[order]
    i = 0
    while i < len(s):
        j = i
        while j + 1 < len(s) and sorted_s[j + 1] == sorted_s[i]:
            j += 1
        ranks[order[i:j + 1]] = 0.5 * (i + j) + 1
        i = j + 1
    n1, n0 = len(score_pos), len(score_neg)
    return float((ranks[:n1].sum() - n1 * (n1 + 1) / 2) / (n1 * n0)) if n1 and n0 else float("nan")


def evaluate(events: dict, stereo: dict, truth: np.ndarray):
    """Resolution of the learned and the geometric reconstruction against the
    generated truth (truth rows: E TeV, src_x, src_y, core_x, core_y, is_proton, m, attempts)."""
    gam = truth[:, 5] == 0
    ok_s = (events["flags"] & 1) == 0
    ok_g = (stereo["flags"] & 1) == 0
    both = gam & ok_s & ok_g
    d_s = np.hypot(events["dir_x"] - truth[:, 1], events["dir_y"] - truth[:, 2])
    d_g = np.hypot(stereo["dir_x"] - truth[:, 1], stereo["dir_y"] - truth[:, 2])
    le = events["log_energy"] - np.log10(truth[:, 0])
    out = dict(n_events=int(len(truth)), n_gamma_both=int(both.sum()),
               r68_surrogate_deg=containment68(d_s[both]), r68_geometric_deg=containment68(d_g[both]),
               energy_bias=float(np.mean(le[gam & ok_s])) if (gam & ok_s).any() else float("nan"),
               energy_res=float(np.std(le[gam & ok_s])) if (gam & ok_s).any() else float("nan"),
               fallback_frac=float(np.mean((events["flags"] & 2) != 0)),
               auc_gamma_hadron=roc_auc(events["gammaness"][gam & ok_s], events["gammaness"][~gam & ok_s]))
    out["r68_ratio"] = out["r68_surrogate_deg"] / out["r68_geometric_deg"]
    return out


# Checkpoint file: the magic bytes, then little-endian uint32 version, uint32 parameter
# count n, int64 Adam steps taken, 16 float32 camera codes, and the float32 parameters,
# first moments and second moments (n each, the packed order of rta_surrogate_set_params).
CHECKPOINT_MAGIC = b"RTASURR1"
CHECKPOINT_VERSION = 1


def write_checkpoint(path: str, params, m, v, step: int, cam_code):
    p, m, v = (np.ascontiguousarray(x, "<f4").reshape(-1) for x in (params, m, v))
    codes = np.zeros(16, "<f4")
    c = np.asarray(cam_code, "<f4").reshape(-1)[:16]
    codes[: len(c)] = c
    if not (p.size == m.size == v.size):
        raise ValueError("parameters and moments differ in size")
    with open(path, "wb") as f:
        f.write(CHECKPOINT_MAGIC)
        f.write(np.array([CHECKPOINT_VERSION, p.size], "<u4").tobytes())
        f.write(np.array([step], "<i8").tobytes())
        f.write(codes.tobytes())
        for x in (p, m, v):
            f.write(x.tobytes())


def read_checkpoint(path: str):
    """(parameters, first moments, second moments, steps, camera codes); ValueError on a
    file of another kind or a truncated one."""
    with open(path, "rb") as f:
        raw = f.read()
    head = len(CHECKPOINT_MAGIC) + 8 + 8 + 64
    if len(raw) < head or raw[: len(CHECKPOINT_MAGIC)] != CHECKPOINT_MAGIC:
        raise ValueError(f"{path}: not a surrogate checkpoint")
    o = len(CHECKPOINT_MAGIC)
    version, n = np.frombuffer(raw, "<u4", 2, o)
    if version != CHECKPOINT_VERSION:
        raise ValueError(f"{path}: checkpoint version {version}, expected {CHECKPOINT_VERSION}")
    step = int(np.frombuffer(raw, "<i8", 1, o + 8)[0])
    codes = np.frombuffer(raw, "<f4", 16, o + 16).copy()
    if len(raw) != head + 12 * int(n):
        raise ValueError(f"{path}: truncated or padded checkpoint")
    arrs = [np.frombuffer(raw, "<f4", int(n), head + 4 * int(n) * k).copy() for k in range(3)]
    return arrs[0], arrs[1], arrs[2], step, codes
