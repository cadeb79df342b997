"""CPU oracle of the learned deep-sets surrogate -- TEST INFRASTRUCTURE ONLY.

Plain numpy in FP64. Only the tests, the smoke check and the benchmark's CPU
baseline load it; the CUDA library never does.

The paper asks RT-RECO for energy reconstruction and gamma/hadron separation
next to the direction (Sec. 4.1), as a speed-reduced version of the offline
reconstruction (Sec. 4.2). This surrogate is the reading of that step used
here; every definition below is what the CUDA kernels implement:

Features (per image, from its Hillas row and telescope):
  an image is used when it has >= 3 pixels (and is not empty or skipped);
  the event baseline b is the axis intersection of its two brightest used
  images (ties to the lower index) when |sin(psi_2 - psi_1)| >= 0.1, else the
  size-weighted mean centroid of its used images, else (0, 0);
  x = [log10 size, x - b_x, y - b_y, length, width, cos 2psi, sin 2psi,
       time_grad / 10, |c - b|, type code of the camera, T_x / 1000 m, T_y / 1000 m]
Network (deep sets):
  phi:  h1 = relu(x W1 + b1) (12 -> 128), h2 = relu(h1 W2 + b2) (128 -> 128)
  pool: p = [sum_used h2 / 40, sum_used h2 / max(1, n_used)]   (256)
  rho:  g = relu(p V1 + c1) (256 -> 256), y = g V2 + c2 (256 -> 4)
  y = (log10 E / TeV, dx, dy (deg, offsets from b), gammaness logit)
Loss (mean over the events of a batch):
  gamma events: (y0 - log10 E)^2 + ((y1 - dx)^2 + (y2 - dy)^2) / 0.1^2
  every event:  BCE(sigmoid(y3), is_gamma)
Adam: beta = (0.9, 0.999), eps = 1e-8, bias-corrected, FP32 master weights on the GPU.
"""
from __future__ import annotations

import numpy as np

N_FEAT = 12
POOL_DIV = 40.0
DIR_SIGMA = 0.1
BASE_MIN_SIN = 0.1
LAYERS = [("W1", (12, 128)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)),
          ("V1", (256, 256)), ("c1", (256,)), ("V2", (256, 4)), ("c2", (4,))]

# Hillas row layout of oracle.H
_SIZE, _X, _Y, _L, _W, _PSI, _R, _PHI, _TG, _TM, _NPIX, _FLAGS = range(12)


def used_images(h):
    return (h[:, _NPIX] >= 3) & ((h[:, _FLAGS].astype(np.int64) & 5) == 0)


def baseline(h, used):
    """Event baseline direction from one event's Hillas rows (see module doc)."""
    idx = np.nonzero(used)[0]
    if len(idx) == 0:
        return np.zeros(2)
    if len(idx) >= 2:
        order = sorted(idx, key=lambda i: (-h[i, _SIZE], i))
        a, c = order[0], order[1]
        s = np.sin(h[c, _PSI] - h[a, _PSI])
        if abs(s) >= BASE_MIN_SIN:
            ua = np.array([np.cos(h[a, _PSI]), np.sin(h[a, _PSI])])
            uc = np.array([np.cos(h[c, _PSI]), np.sin(h[c, _PSI])])
            d = h[c, [_X, _Y]] - h[a, [_X, _Y]]
            k = (d[0] * uc[1] - d[1] * uc[0]) / s
            return h[a, [_X, _Y]] + k * ua
    w = h[idx, _SIZE]
    return (w[:, None] * h[idx][:, [_X, _Y]]).sum(0) / w.sum()


def features(hrows, evt_off, img_tel, tel_xy, tel_code):
    """Per-image features (n_img, 12), used mask, per-event baselines (n_evt, 2), used counts."""
    hrows = np.asarray(hrows, np.float64)
    n_img, n_evt = len(hrows), len(evt_off) - 1
    X = np.zeros((n_img, N_FEAT))
    used = used_images(hrows)
    base = np.zeros((n_evt, 2))
    n_used = np.zeros(n_evt, np.int64)
    for e in range(n_evt):
        a, b = evt_off[e], evt_off[e + 1]
        h = hrows[a:b]
        base[e] = baseline(h, used[a:b])
        n_used[e] = used[a:b].sum()
        for k in range(b - a):
            i = a + k
            t = img_tel[i]
            dx, dy = h[k, _X] - base[e, 0], h[k, _Y] - base[e, 1]
            X[i] = [np.log10(max(h[k, _SIZE], 1e-3)), dx, dy, h[k, _L], h[k, _W], np.cos(2 * h[k, _PSI]),
                    np.sin(2 * h[k, _PSI]), h[k, _TG] / 10.0, np.hypot(dx, dy), tel_code[t], tel_xy[t, 0] / 1000.0,
                    tel_xy[t, 1] / 1000.0]
    return X, used, base, n_used


def relu(x):
    return np.maximum(x, 0.0)


def forward(params, X, used, evt_off):
    """Deep-sets forward pass. Returns y (n_evt, 4) and the cache for backward."""
    W1, b1, W2, b2, V1, c1, V2, c2 = (params[k] for k, _ in LAYERS)
    z1 = X @ W1 + b1
    h1 = relu(z1)
    z2 = h1 @ W2 + b2
    h2 = relu(z2)
    n_evt = len(evt_off) - 1
    H = h2.shape[1]
    pool = np.zeros((n_evt, 2 * H))
    cnt = np.zeros(n_evt)
    for e in range(n_evt):
        a, b = evt_off[e], evt_off[e + 1]
        m = used[a:b]
        s = h2[a:b][m].sum(0) if m.any() else np.zeros(H)
        cnt[e] = m.sum()
        pool[e, :H] = s / POOL_DIV
        pool[e, H:] = s / max(1.0, cnt[e])
    zg = pool @ V1 + c1
    g = relu(zg)
    y = g @ V2 + c2
    cache = dict(X=X, z1=z1, h1=h1, z2=z2, h2=h2, pool=pool, cnt=cnt, zg=zg, g=g, used=used, evt_off=evt_off)
    return y, cache


def loss(y, logE, ddir, is_gamma):
    """Mean loss over the batch and its gradient dL/dy."""
    n = len(y)
    gam = is_gamma.astype(np.float64)
    r0 = y[:, 0] - logE
    r1 = y[:, 1] - ddir[:, 0]
    r2 = y[:, 2] - ddir[:, 1]
    sig = 1.0 / (1.0 + np.exp(-y[:, 3]))
    bce = np.logaddexp(0.0, y[:, 3]) - gam * y[:, 3]        # -log sigmoid / -log(1 - sigmoid)
    L = (gam * (r0 ** 2 + (r1 ** 2 + r2 ** 2) / DIR_SIGMA ** 2) + bce).sum() / n
    dy = np.zeros_like(y)
    dy[:, 0] = 2 * gam * r0 / n
    dy[:, 1] = 2 * gam * r1 / DIR_SIGMA ** 2 / n
    dy[:, 2] = 2 * gam * r2 / DIR_SIGMA ** 2 / n
    dy[:, 3] = (sig - gam) / n
    return L, dy


def backward(params, cache, dy):
    """Gradients of the loss with respect to every parameter, by the chain rule."""
    W1, b1, W2, b2, V1, c1, V2, c2 = (params[k] for k, _ in LAYERS)
    g, zg, pool = cache["g"], cache["zg"], cache["pool"]
    grads = {}
    grads["V2"] = g.T @ dy
    grads["c2"] = dy.sum(0)
    dg = dy @ V2.T
    dzg = dg * (zg > 0)
    grads["V1"] = pool.T @ dzg
    grads["c1"] = dzg.sum(0)
    dpool = dzg @ V1.T
    h2, z2, h1, z1, X = cache["h2"], cache["z2"], cache["h1"], cache["z1"], cache["X"]
    H = h2.shape[1]
    dh2 = np.zeros_like(h2)
    evt_off, used, cnt = cache["evt_off"], cache["used"], cache["cnt"]
    for e in range(len(evt_off) - 1):
        a, b = evt_off[e], evt_off[e + 1]
        gsum = dpool[e, :H] / POOL_DIV + dpool[e, H:] / max(1.0, cnt[e])
        dh2[a:b] = used[a:b, None] * gsum[None, :]
    dz2 = dh2 * (z2 > 0)
    grads["W2"] = h1.T @ dz2
    grads["b2"] = dz2.sum(0)
    dh1 = dz2 @ W2.T
    dz1 = dh1 * (z1 > 0)
    grads["W1"] = X.T @ dz1
    grads["b1"] = dz1.sum(0)
    return grads


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam update (Kingma and Ba 2015); returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a32 = np.ascontiguousarray(a, np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed: int, scale: float = 1.0):
    """He-style random weights (test fixtures; not the GPU's own initialiser)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in LAYERS:
        if len(shape) == 2:
            p[name] = rng.normal(0, scale * np.sqrt(2.0 / shape[0]), shape)
        else:
            p[name] = rng.normal(0, 0.05 * scale, shape)
    return p
